"""GPU parity of per-species subcycling (Listing 7's x += nstep*vx): the ions advanced
every K steps with time step K dt, deposited every step.  Same tolerances as the other
parity tests: FP64 1e-12 relative over 100 steps with wall, collision and live counts
bit-exact; FP32 1e-5 over 10 steps."""
import numpy as np
import pytest

from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W
from tests.gpu_common import (assert_same_clocks, by_id, ensure_built, particle_errors,
                              requires_gpu, run_gpu, run_oracle)

pytestmark = [pytest.mark.gpu, requires_gpu]


@pytest.mark.parametrize("precision,steps,tol", [(capi.FP64, 100, 1e-12), (capi.FP32, 10, 1e-5)])
def test_subcycled_ions_bounded_plasma(precision, steps, tol):
    phys = W.bounded_small(ion_nstep=4)
    loads = W.initial_load(phys, seed=1)
    g, gm = run_gpu(phys, loads, steps, precision, sort_interval=20)
    o, om = run_oracle(phys, loads, steps)
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < tol and ev < tol, (s, ex, ev)
    assert_same_clocks(g, o)
    if precision == capi.FP64:
        np.testing.assert_array_equal(gm["wall_count"], om["wall_count"])
        np.testing.assert_array_equal(gm["collisions"], om["collisions"])
        np.testing.assert_array_equal(gm["live"], om["live"])
        assert om["collisions"][1] > 0  # the subcycled ions collided
        np.testing.assert_allclose(gm["kinetic"], om["kinetic"], rtol=1e-12)
        np.testing.assert_allclose(gm["wall_energy"], om["wall_energy"], rtol=1e-12)


def test_subcycled_ions_with_ionization_and_source_fp64():
    """Boris push, volume re-injection and ionization whose ion products are born in the
    subcycled species' own velocity units."""
    phys = W.magnetized_source(ncells=64, ppc=40, seed=2, nu=0.2, capacity_factor=3.0,
                               ion_nstep=3)
    loads = W.initial_load(phys, seed=2)
    steps = 100
    g, gm = run_gpu(phys, loads, steps, capi.FP64, sort_interval=10)
    o, om = run_oracle(phys, loads, steps)
    assert om["collisions"][1] > 0
    np.testing.assert_array_equal(gm["collisions"], om["collisions"])
    np.testing.assert_array_equal(gm["wall_count"], om["wall_count"])
    np.testing.assert_array_equal(gm["live"], om["live"])
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < 1e-12 and ev < 1e-12, (s, ex, ev)
    assert_same_clocks(g, o)


def test_subcycled_checkpoint_restart_off_the_cycle():
    """A checkpoint taken at a step that is not a multiple of K (cell units, clocks,
    counters) continues bit-identically."""
    ensure_built()
    phys = W.magnetized_source(ncells=48, ppc=30, seed=8, nu=0.3, capacity_factor=3.0,
                               ion_nstep=4)
    loads = W.initial_load(phys, seed=8)
    ref = capi.Sim(phys, precision=capi.FP64, sort_interval=7)
    ref.load_all(loads)
    ref.step(45)
    want = [by_id(ref.particles(0, s, cell_units=True)) for s in range(2)]
    ref.close()
    a = capi.Sim(phys, precision=capi.FP64, sort_interval=7)
    a.load_all(loads)
    a.step(25)
    snap = [a.particles(0, s, cell_units=True) for s in range(2)]
    m = a.moments(0)
    a.close()
    b = capi.Sim(phys, precision=capi.FP64, sort_interval=7)
    for s, p in enumerate(snap):
        b.load(0, s, W.Load(p["cell"], p["off"], p["vx"], p["vy"], p["vz"], p["id"], p["state"]),
               cell_units=True)
    b.restore_counters(m["step"], [m["next_id"]])
    b.step(20)
    got = [by_id(b.particles(0, s, cell_units=True)) for s in range(2)]
    b.close()
    for x, y in zip(want, got):
        for k in x:
            np.testing.assert_array_equal(x[k], y[k])


def test_subcycled_and_smoothed_instances_in_a_batch_equal_alone():
    ensure_built()
    a = W.bounded_small(ncells=64, ppc=40, seed=5, ion_nstep=3)
    b = W.magnetized_source(ncells=48, ppc=30, seed=6, nu=0.2, capacity_factor=3.0, ion_nstep=5)
    b.smooth = 1
    c = W.bounded_small(ncells=32, ppc=20, seed=7)
    phys = [a, b, c]
    loads = [W.initial_load(p, seed=p.seed) for p in phys]
    steps = 33
    sim = capi.Sim(phys, precision=capi.FP64, sort_interval=10)
    for i, ld in enumerate(loads):
        sim.load_all(ld, inst=i)
    sim.step(steps)
    batch = [[by_id(sim.particles(i, s)) for s in range(2)] for i in range(3)]
    sim.close()
    for i, p in enumerate(phys):
        s1 = capi.Sim(p, precision=capi.FP64, sort_interval=10)
        s1.load_all(loads[i])
        s1.step(steps)
        alone = [by_id(s1.particles(0, s)) for s in range(2)]
        s1.close()
        for x, y in zip(alone, batch[i]):
            for k in x:
                np.testing.assert_array_equal(x[k], y[k])
