"""Parity at the benchmark's full size: 65,536 cells x 1,500 particles per cell per
species (196,608,000 particles), the launch configuration bench.py times.

The oracle advances the same input one step (a few seconds of CPU); both GPU forms
are compared particle by particle (matched by id), together with the initial field,
the exact fixed-point charge invariant and the particle-count bookkeeping.
"""
import numpy as np
import pytest

from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W
from tests.gpu_common import by_id, ensure_built, particle_errors, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


@pytest.fixture(scope="module")
def full_case():
    from oracle.oracle import Oracle
    phys = W.bounded_large()
    loads = W.initial_load(phys, seed=1)
    o = Oracle(phys)
    o.load_all(loads)
    m0 = o.moments()
    o.step(1)
    m1 = o.moments()
    parts = [o.particles(s) for s in range(2)]
    del o
    return phys, loads, m0, m1, parts


@pytest.mark.parametrize("precision,tol", [(capi.FP32, 1e-5), (capi.FP64, 1e-12)])
def test_full_size_one_step(full_case, precision, tol):
    ensure_built()
    phys, loads, m0, m1, ora = full_case
    sim = capi.Sim(phys, precision=precision, sort_interval=20)
    sim.load_all(loads)
    g0 = sim.moments(0)
    scale = np.abs(m0["E"]).max()
    np.testing.assert_allclose(g0["E"], m0["E"], rtol=0, atol=tol * scale)
    sim.step(1)
    g1 = sim.moments(0)
    raw, unit = sim.charge_raw(0)
    for s in range(2):
        # exact charge (the total exceeds int64 in the FP64 form: sum as Python ints)
        assert sum(map(int, raw[s])) == int(g1["live"][s]) * unit
        # every particle is either alive or counted at a wall
        assert g1["live"][s] + g1["wall_count"][s].sum() == len(loads[s])
    if precision == capi.FP64:
        np.testing.assert_array_equal(g1["live"], m1["live"])
        np.testing.assert_array_equal(g1["wall_count"], m1["wall_count"])
        np.testing.assert_array_equal(g1["collisions"], m1["collisions"])
    gp = [sim.particles(0, s) for s in range(2)]
    sim.close()
    for s, (ex, ev) in enumerate(particle_errors(phys, gp, ora)):
        assert ex < tol and ev < tol, (s, ex, ev)
    for g, o in zip(gp, ora):
        np.testing.assert_array_equal(by_id(g)["state"], o["state"])


def test_paper_case_full_size_fp64_one_cycle():
    """The paper's test case at its benchmark size (100,000 cells x 100 particles per cell
    x e, D+ and D = 30,000,000 particles; ionization depleting the D particles) over one
    whole sort cycle of 20 steps: the D particles' one move, their separate sort and
    every step's conversions of targets into ions, against the oracle (FP64: counts,
    ids and clocks exact, particles within 1e-12)."""
    from oracle.oracle import Oracle
    ensure_built()
    phys = W.ionization_case()
    loads = W.initial_load(phys, seed=phys.seed)
    steps = phys.sort_interval
    o = Oracle(phys)
    o.load_all(loads)
    o.step(steps)
    om = o.moments()
    ora = [o.particles(s) for s in range(3)]
    del o
    sim = capi.Sim(phys, precision=capi.FP64, sort_interval=phys.sort_interval)
    sim.load_all(loads)
    sim.step(steps)
    gm = sim.moments(0)
    gp = [sim.particles(0, s) for s in range(3)]
    sim.close()
    assert om["collisions"][2] > 0  # targets were converted
    np.testing.assert_array_equal(gm["live"], om["live"])
    np.testing.assert_array_equal(gm["collisions"], om["collisions"])
    for s, (ex, ev) in enumerate(particle_errors(phys, gp, ora)):
        assert ex < 1e-12 and ev < 1e-12, (s, ex, ev)
    for g, o in zip(gp, ora):
        np.testing.assert_array_equal(by_id(g)["state"], by_id(o)["state"])
