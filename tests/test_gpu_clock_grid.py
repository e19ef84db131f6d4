"""GPU parity across the collision clock's test grid.

Every particle's collision clock tests (draws its next candidate-free run) at the
latest on the steps whose own-step index is a multiple of 127; on those steps the
plain FP32 mover of a large batch also switches to the variant with the draw inline.
These runs cross that grid against the oracle: FP64 over 300 steps (grid steps 127
and 254), ions subcycled by 4 over 520 steps (their own grid at step 511), and the
FP32 form from a state saved at step 120 over 10 steps across step 127.  Integer state
(collision clocks, collision counts, wall counts, live counts) must be identical;
every particle within the form's tolerance (FP64 1e-12, FP32 1e-5).
"""
import numpy as np
import pytest

from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W
from tests.gpu_common import (assert_same_clocks, ensure_built, particle_errors, requires_gpu,
                              run_gpu, run_oracle)

pytestmark = [pytest.mark.gpu, requires_gpu]


def _check_integers(gm, om):
    np.testing.assert_array_equal(gm["live"], om["live"])
    np.testing.assert_array_equal(gm["wall_count"], om["wall_count"])
    np.testing.assert_array_equal(gm["collisions"], om["collisions"])


def test_bounded_small_fp64_300_steps():
    phys = W.bounded_small()
    loads = W.initial_load(phys, seed=1)
    g, gm = run_gpu(phys, loads, 300, capi.FP64, sort_interval=20)
    o, om = run_oracle(phys, loads, 300)
    _check_integers(gm, om)
    assert_same_clocks(g, o)
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < 1e-12 and ev < 1e-12, (s, ex, ev)


def test_magnetized_source_fp64_300_steps():
    phys = W.magnetized_source(ncells=64, ppc=40, seed=6, nu=0.1, capacity_factor=3.0)
    loads = W.initial_load(phys, seed=6)
    sim = capi.Sim(phys, precision=capi.FP64, sort_interval=10)
    sim.load_all(loads)
    sim.step(300)
    g = [sim.particles(0, s) for s in range(2)]
    gm = sim.moments(0)
    sim.close()
    o, om = run_oracle(phys, loads, 300)
    _check_integers(gm, om)
    assert om["collisions"][1] > 0
    assert_same_clocks(g, o)
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < 1e-12 and ev < 1e-12, (s, ex, ev)


def test_subcycled_ions_fp64_cross_their_own_grid():
    # ions advance on the steps n with (n+1) % 4 == 0; their own step index
    # (n+1)/4 - 1 reaches 127 at n = 511
    phys = W.bounded_small(ncells=128, ppc=60, seed=12, nu=0.05, ion_nstep=4)
    loads = W.initial_load(phys, seed=12)
    g, gm = run_gpu(phys, loads, 520, capi.FP64, sort_interval=20)
    o, om = run_oracle(phys, loads, 520)
    _check_integers(gm, om)
    assert om["collisions"][1] > 0
    assert_same_clocks(g, o)
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < 1e-12 and ev < 1e-12, (s, ex, ev)


@pytest.mark.parametrize("case", ["bounded", "source"])
def test_fp32_across_step_127_from_a_saved_state(case):
    """The state the oracle reaches at step 120 is loaded into both sides (clocks
    included, the step counter set to 120); ten FP32 steps cross step 127, where every
    clock without a pending candidate tests and the mover pair runs its inline
    variant."""
    from oracle.oracle import Oracle
    ensure_built()
    if case == "bounded":
        phys = W.bounded_small(ncells=200, ppc=60, seed=8, nu=0.05)
    else:
        phys = W.magnetized_source(ncells=64, ppc=60, seed=8, B=0.0, nu=0.05,
                                   capacity_factor=3.0)
    loads = W.initial_load(phys, seed=8)
    o = Oracle(phys)
    o.load_all(loads)
    o.step(120)
    snap = [o.particles(s) for s in range(len(phys.species))]
    next_id = int(max(int(p["id"].max(initial=0)) for p in snap)) + 1
    saved = [W.Load(p["cell"], p["off"], p["vx"], p["vy"], p["vz"], p["id"], p["state"])
             for p in snap]
    del o

    ref = Oracle(phys)
    ref.load_all(saved)
    ref.set_step(120, next_id)
    ref.step(10)
    want = [ref.particles(s) for s in range(len(phys.species))]
    wm = ref.moments()

    sim = capi.Sim(phys, precision=capi.FP32, sort_interval=20)
    sim.load_all(saved)
    sim.restore_counters(120, [next_id])
    sim.step(10)
    got = [sim.particles(0, s) for s in range(len(phys.species))]
    gm = sim.moments(0)
    sim.close()
    assert gm["step"] == wm["step"] == 130
    np.testing.assert_array_equal(gm["live"], wm["live"])
    if case == "bounded":  # no energy threshold: FP32 rounding decides no count
        np.testing.assert_array_equal(gm["collisions"], wm["collisions"])
    assert_same_clocks(got, want)
    for s, (ex, ev) in enumerate(particle_errors(phys, got, want)):
        assert ex < 1e-5 and ev < 1e-5, (s, ex, ev)
