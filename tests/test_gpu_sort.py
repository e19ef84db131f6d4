"""The sort folded into the time step.  The step before a sort counts the particles per
cell at its end; the sort step then moves every particle into a slot of the other store
copy reserved by the cell it starts the step in, so the store leaves that step ordered
by start cell, with the particles the step creates after all of them.  A sort only
permutes the store, so every sort path (folded, separate, none) gives the same
particles, fields and counters."""
import numpy as np
import pytest

from gpu_common import by_id, ensure_built
from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_sort_step_orders_the_store_by_start_cell(precision):
    ensure_built()
    phys = W.magnetized_source(ncells=64, ppc=60, seed=21, nu=0.3, capacity_factor=3.0)
    loads = W.initial_load(phys, seed=21)
    K = 5
    sim = capi.Sim(phys, precision=precision, sort_interval=K)
    sim.load_all(loads)
    sim.step(2 * K - 1)  # one cycle through its graph, then single steps up to the sort step
    before = [sim.particles(0, s) for s in range(2)]
    sim.step(1)          # the sort step: (n + 1) mod K = 0
    after = [sim.particles(0, s) for s in range(2)]
    sim.close()
    moved = 0
    for b, a in zip(before, after):
        start = dict(zip(b["id"].tolist(), b["cell"].tolist()))
        old = np.array([i in start for i in a["id"].tolist()])
        # particles created in the sort step (ionization products) follow the sorted ones
        assert old.any()
        if not old.all():
            assert np.argmin(old) == old.sum() and not old[old.sum():].any()
        n = int(old.sum())
        c0 = np.array([start[i] for i in a["id"][:n].tolist()])
        assert np.all(np.diff(c0) >= 0), "store not ordered by start-of-step cell"
        moved += int(np.count_nonzero(a["cell"][:n] != c0))
    assert moved > 0  # the check would not see a sort by end-of-step cell otherwise


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_all_sort_paths_give_the_same_run(precision):
    """No sort, the separate sort every step (interval 1), the folded sort every other
    step (interval 2), and interval 5 from step 4, a sort step with no counts from a
    step before (the separate sort, then folded ones), agree bit for bit."""
    ensure_built()
    phys = W.magnetized_source(ncells=48, ppc=40, seed=22, nu=0.3, capacity_factor=3.0)
    loads = W.initial_load(phys, seed=22)
    out = []
    for sort in (0, 1, 2, 5):
        sim = capi.Sim(phys, precision=precision, sort_interval=sort)
        sim.load_all(loads)
        sim.restore_counters(4)
        sim.step(23)
        out.append(([by_id(sim.particles(0, s)) for s in range(2)], sim.moments(0)))
        sim.close()
    ref = out[0]
    assert ref[1]["step"] == 27
    for parts, m in out[1:]:
        for a, b in zip(ref[0], parts):
            for k in a:
                np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(ref[1]["E"], m["E"])
        np.testing.assert_array_equal(ref[1]["collisions"], m["collisions"])
        np.testing.assert_array_equal(ref[1]["wall_count"], m["wall_count"])
        np.testing.assert_array_equal(ref[1]["live"], m["live"])
