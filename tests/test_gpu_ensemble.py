"""The batched ensemble at full size: 512 independent magnetized plasmas with volume
source and elastic + ionization + charge-exchange collisions (about 5e8 particles), run
as one batch in the configuration bench.py times.  Sixteen sampled instances are
checked particle by particle against the oracle, and two against the same instance run
alone (bit-identical).

Tolerance.  FP64: every particle within 1e-12 at every cell count (the oracle's
density and field phases are exact to within one final rounding, binary128 sums and
Thomas solve, like the GPU's fixed-point deposit and integer solve).  FP32: 1e-5, but
an ionization gives both outgoing electrons the speed sqrt((E - E_iz)/m), which near
threshold amplifies the FP32 rounding of the incident velocity by E/(E - E_iz); the
electron that ionized and both products are held to 100x.  Measured: instance 96 of
this ensemble has an ionization participant at 1.07e-5 after 10 steps; every other
particle is held to the flat 1e-5."""
import concurrent.futures as cf

import numpy as np
import pytest

from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W
from tests.gpu_common import (assert_same_clocks, by_id, ensure_built,
                              oracle_with_ionization_record, participant_mask, particle_errors,
                              requires_gpu, run_oracle, velocity_errors)

pytestmark = [pytest.mark.gpu, requires_gpu]

SAMPLE = list(range(0, 512, 32))  # 16 instances spread over the size range


@pytest.fixture(scope="module")
def ensemble():
    phys = W.ensemble()
    with cf.ThreadPoolExecutor(8) as ex:
        loads = list(ex.map(lambda ip: W.initial_load(ip[1], seed=ip[0] + 1), enumerate(phys)))
    return phys, loads


def _run_batch(phys, loads, precision, steps, sample):
    sim = capi.Sim(phys, precision=precision, sort_interval=20)
    for i, ld in enumerate(loads):
        sim.load_all(ld, inst=i)
    sim.step(steps)
    out = {i: ([sim.particles(i, s) for s in range(2)], sim.moments(i)) for i in sample}
    sim.close()
    return out


@pytest.mark.parametrize("precision,steps,tol", [(capi.FP32, 10, 1e-5), (capi.FP64, 20, 1e-12)])
def test_ensemble_sampled_instances_match_oracle(ensemble, precision, steps, tol):
    ensure_built()
    phys, loads = ensemble
    sample = SAMPLE if precision == capi.FP32 else SAMPLE[::4]
    got = _run_batch(phys, loads, precision, steps, sample)
    for i in sample:
        g, gm = got[i]
        if precision == capi.FP64:
            o, om = run_oracle(phys[i], loads[i], steps)
        else:
            o, om, n0, parents = oracle_with_ionization_record(phys[i], loads[i], steps)
        np.testing.assert_array_equal(gm["live"], om["live"])
        if precision == capi.FP64:
            np.testing.assert_array_equal(gm["collisions"], om["collisions"])
            np.testing.assert_array_equal(gm["wall_count"], om["wall_count"])
        for s, (ex, ev) in enumerate(particle_errors(phys[i], g, o)):
            assert ex < tol, (i, s, ex)
            if precision == capi.FP64:
                assert ev < tol, (i, s, ev)
            else:
                e = velocity_errors(phys[i], g[s], o[s], s)
                part = participant_mask(o[s], n0, parents)
                assert e[~part].max(initial=0.0) < tol, (i, s, e[~part].max())
                assert e[part].max(initial=0.0) < 100 * tol, (i, s, e[part].max())
        assert_same_clocks(g, o)


def test_ensemble_instance_in_batch_equals_alone(ensemble):
    ensure_built()
    phys, loads = ensemble
    picks = [5, 300]
    got = _run_batch(phys, loads, capi.FP32, 25, picks)
    for i in picks:
        sim = capi.Sim(phys[i], precision=capi.FP32, sort_interval=20)
        sim.load_all(loads[i])
        sim.step(25)
        alone = [by_id(sim.particles(0, s)) for s in range(2)]
        sim.close()
        for a, b in zip(alone, got[i][0]):
            b = by_id(b)
            for k in a:
                np.testing.assert_array_equal(a[k], b[k])
