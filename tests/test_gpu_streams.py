"""Work of a time step that shares no word with the rest of it runs on a second stream:
the event kernels beside the field phase when they deposit nothing (no volume source,
no ionization, no neutral target), else the numbering of ionization products beside the
target conversions and the field phase; both joined before the next step.  With kernel
timing on, every kernel runs in order on the handle's stream without graphs, so the two
schedules are compared here bit for bit: the same particles, clocks, fields and counters
whichever branch a workload takes."""
import numpy as np
import pytest

from gpu_common import by_id, ensure_built
from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(phys, loads, steps, precision, sort_interval, serial):
    sim = capi.Sim(phys, precision=precision, sort_interval=sort_interval)
    sim.load_all(loads)
    if serial:
        sim.profile(True)
    sim.step(steps)
    parts = [by_id(sim.particles(0, s)) for s in range(len(phys.species))]
    m = sim.moments(0)
    sim.close()
    return parts, m


def _cases():
    quiet = W.bounded_small(ncells=128, ppc=40, seed=31)  # events beside the field phase
    src = W.magnetized_source(ncells=64, ppc=60, seed=32, nu=0.3, capacity_factor=3.0)
    tgt = W.ionization_case(ncells=96, ppc=40, nu_el=0.05, nu_exc=0.05, nu_iz=0.1, seed=33,
                            sort_interval=5)
    tgt.species[0].capacity_factor = 3.0
    tgt.species[1].capacity_factor = 3.0
    return [("absorbing walls, elastic + CX", quiet, 10),
            ("volume source, ionization", src, 10),
            ("neutral targets, ionization", tgt, 5)]


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
@pytest.mark.parametrize("which", [0, 1, 2])
def test_second_stream_changes_no_result(precision, which):
    ensure_built()
    name, phys, K = _cases()[which]
    loads = W.initial_load(phys, seed=30 + which)
    steps = 3 * K + 2  # several sort cycles and a partial one (graph windows of both kinds)
    a_parts, a_m = _run(phys, loads, steps, precision, K, serial=True)
    b_parts, b_m = _run(phys, loads, steps, precision, K, serial=False)
    for a, b in zip(a_parts, b_parts):
        for k in a:
            np.testing.assert_array_equal(a[k], b[k], err_msg="%s: %s" % (name, k))
    for k in ("step", "live", "collisions", "wall_count", "next_id"):
        np.testing.assert_array_equal(a_m[k], b_m[k], err_msg="%s: %s" % (name, k))
    for k in ("E", "density"):
        np.testing.assert_array_equal(a_m[k], b_m[k], err_msg="%s: %s" % (name, k))
    assert a_m["step"] == steps
