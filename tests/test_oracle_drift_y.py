"""Pins of the oracle's y drift of 2-D species (Listing 1: yp += nstep*vy).

A species flagged sn2d carries a second coordinate yp (cell units) parallel to the
walls, advanced with its velocity in cells per own step after the push, on the steps
the species moves, and used by nothing else:

* free streaming: yp_n = yp_0 + n v_y dt/dx, also for a subcycled species (K dt per own
  step, on every K-th step);
* a uniform field along x changes x ballistically and leaves the y drift untouched;
* the flag changes nothing else: positions, velocities, clocks and counters are the
  same bits with and without it;
* a re-injected particle (volume source) starts again at yp = 0, ionization products
  start at their parent's yp.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2404_10270_gb300 import workloads as W
from tests.gpu_common import by_id


def _stream(nstep=1, field=W.FIELD_NONE, E_ext=0.0, n=64, seed=3):
    sp = [W.Species("n", 0.0 if field == W.FIELD_NONE else -1.0, 1.0, 0.01, 1.0, 0,
                    nstep=nstep, sn2d=1)]
    phys = W.Physics(ncells=32, dx=0.5, dt=0.05, species=sp, processes=[], field=field,
                     E_ext=E_ext, bc=W.BC_PERIODIC, seed=seed)
    rng = np.random.default_rng(seed)
    ld = W.Load(rng.integers(0, 32, n).astype(np.int32), rng.random(n), rng.normal(0, 1, n),
                rng.normal(0, 1, n), rng.normal(0, 1, n), np.arange(n, dtype=np.uint32),
                yp=rng.normal(0, 10, n))
    return phys, ld


@pytest.mark.parametrize("nstep", [1, 3])
def test_free_streaming_in_y(nstep):
    phys, ld = _stream(nstep=nstep)
    o = Oracle(phys)
    o.load(0, ld)
    steps = 30
    o.step(steps)
    p = by_id(o.particles(0))
    u = ld.vy * (nstep * phys.dt / phys.dx)  # cells per own step
    moves = steps // nstep                   # own steps taken: n with (n+1) % K == 0
    want = ld.yp.copy()
    for _ in range(moves):                   # the same additions, in the same order
        want = want + u
    np.testing.assert_array_equal(p["yp"], want)
    np.testing.assert_allclose(p["yp"], ld.yp + moves * u, rtol=0, atol=1e-12)
    # and the velocities are untouched (no field, no collisions; the conversion to cells
    # per step and back rounds twice)
    np.testing.assert_allclose(p["vy"], ld.vy, rtol=4e-16, atol=0)


def test_uniform_field_along_x_leaves_the_y_drift():
    phys, ld = _stream(field=W.FIELD_EXTERNAL, E_ext=0.3)
    o = Oracle(phys)
    o.load(0, ld)
    o.step(25)
    p = by_id(o.particles(0))
    u = ld.vy * (phys.dt / phys.dx)
    np.testing.assert_allclose(p["yp"], ld.yp + 25 * u, rtol=0, atol=1e-12)
    assert np.abs(p["vx"] - ld.vx).max() > 0.1  # x was accelerated


def test_the_flag_changes_nothing_else():
    base = W.magnetized_source(ncells=24, ppc=20, seed=5, nu=0.3, capacity_factor=3.0)
    loads = W.initial_load(base, seed=5)
    runs = []
    for flag in (0, 1):
        phys = W.magnetized_source(ncells=24, ppc=20, seed=5, nu=0.3, capacity_factor=3.0)
        for s in phys.species:
            s.sn2d = flag
        o = Oracle(phys)
        o.load_all(loads)
        o.step(40)
        runs.append(([by_id(o.particles(s)) for s in range(2)], o.moments()))
    (a, ma), (b, mb) = runs
    for x, y in zip(a, b):
        for k in ("cell", "off", "vx", "vy", "vz", "id", "state"):
            np.testing.assert_array_equal(x[k], y[k])
        assert (x["yp"] == 0).all() and (y["yp"] != 0).any()
    for k in ("wall_count", "collisions", "live", "E", "density"):
        np.testing.assert_array_equal(ma[k], mb[k])


def test_reinjection_restarts_and_products_inherit_yp():
    # one step of a hot volume-source plasma with ionization: every particle that left
    # through a wall and came back has yp = 0; every product sits at its parent's yp
    phys = W.magnetized_source(ncells=16, ppc=40, seed=9, nu=3.0, B=0.0, capacity_factor=3.0)
    for s in phys.species:
        s.sn2d = 1
    loads = W.initial_load(phys, seed=9)
    rng = np.random.default_rng(9)
    for ld in loads:
        ld.vx *= 40.0  # many particles reach a wall in one step
        ld.yp = rng.normal(0, 5, len(ld))
    o = Oracle(phys)
    o.load_all(loads)
    o.step(1)
    m = o.moments()
    e = by_id(o.particles(0))
    n0 = sum(len(x) for x in loads)
    assert m["wall_count"].sum() > 0 and m["collisions"][1] > 0
    old = e["id"] < len(loads[0])
    start = loads[0].yp[e["id"][old]]
    moved = start + loads[0].vy[e["id"][old]] * (phys.dt / phys.dx)
    reinjected = e["yp"][old] == 0.0
    assert reinjected.sum() > 0
    np.testing.assert_array_equal(e["yp"][old][~reinjected], moved[~reinjected])
    # products: ids from n0 on, electron 2r, ion 2r + 1; each at a parent's yp
    kids = e["id"] >= n0
    assert kids.sum() == m["collisions"][1]
    assert np.isin(e["yp"][kids], e["yp"][old]).all()
    ions = by_id(o.particles(1))
    ikids = ions["id"] >= n0
    np.testing.assert_array_equal(np.sort(ions["yp"][ikids]), np.sort(e["yp"][kids]))
