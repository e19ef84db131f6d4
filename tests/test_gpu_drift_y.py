"""GPU parity of the y drift of 2-D species (Listing 1: yp += nstep*vy).

The y coordinate (cell units) of a species flagged sn2d is compared with the oracle's,
matched by id, as |d yp| / N (the positions' |dx| / L in cell units), over the same
runs as the other parity tests: FP64 1e-12 over 100 steps, FP32 1e-5 over 10 steps.
The runs cover the sort folded into the step (both its paths), the separate sort,
re-injection by the volume source, ionization products, subcycling and the neutral
particle targets of the paper's test case.  The flag must change nothing else, and a
checkpoint through pic_get_yp / pic_load_yp continues bit-identically.
"""
import numpy as np
import pytest

from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W
from tests.gpu_common import (assert_same_clocks, by_id, ensure_built, particle_errors,
                              requires_gpu, run_oracle)

pytestmark = [pytest.mark.gpu, requires_gpu]


def _flag(phys, species=None):
    for i, s in enumerate(phys.species):
        if species is None or i in species:
            s.sn2d = 1
    return phys


def _with_yp(phys, loads, seed):
    rng = np.random.default_rng(seed)
    for s, ld in zip(phys.species, loads):
        if s.sn2d:
            ld.yp = rng.normal(0.0, 20.0, len(ld))
    return loads


def _run_gpu(phys, loads, steps, precision, sort_interval):
    ensure_built()
    sim = capi.Sim(phys, precision=precision, sort_interval=sort_interval)
    sim.load_all(loads)
    sim.step(steps)
    out = [sim.particles(0, s) for s in range(len(phys.species))]
    m = sim.moments(0)
    sim.close()
    return out, m


def _yp_errors(phys, g, o):
    res = []
    for s, (a, b) in enumerate(zip(g, o)):
        a, b = by_id(a), by_id(b)
        np.testing.assert_array_equal(a["id"], b["id"])
        if not phys.species[s].sn2d:
            assert (a["yp"] == 0).all()
            continue
        res.append(np.abs(a["yp"] - b["yp"]).max(initial=0.0) / phys.ncells)
    return res


CASES = {
    # sort folded into the step, staged path
    "bounded": lambda: (_flag(W.bounded_small(ncells=128, ppc=50, seed=3)), 20),
    # ionization products and volume re-injection, Boris push
    "source": lambda: (_flag(W.magnetized_source(ncells=64, ppc=40, seed=4, nu=0.2,
                                                 capacity_factor=3.0)), 10),
    # subcycled ions (the drift on their own steps only)
    "subcycled": lambda: (_flag(W.bounded_small(ncells=96, ppc=40, seed=5, ion_nstep=4)), 20),
    # sort every step: the separate sort
    "sort_every_step": lambda: (_flag(W.bounded_small(ncells=64, ppc=30, seed=6)), 1),
    # the paper's case: 2-D neutral targets, converted into ions by ionization
    "targets": lambda: (_flag(W.ionization_case(ncells=300, ppc=40, seed=7, nu_iz=0.05),
                              species=[2]), 20),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision,steps,tol", [(capi.FP64, 100, 1e-12), (capi.FP32, 10, 1e-5)])
def test_y_drift_matches_oracle(case, precision, steps, tol):
    phys, K = CASES[case]()
    if case == "targets":
        K = phys.sort_interval
    loads = _with_yp(phys, W.initial_load(phys, seed=phys.seed), phys.seed)
    g, gm = _run_gpu(phys, loads, steps, precision, K)
    o, om = run_oracle(phys, loads, steps)
    np.testing.assert_array_equal(gm["live"], om["live"])
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < tol and ev < tol, (s, ex, ev)
    for e in _yp_errors(phys, g, o):
        assert e < tol, e
    if precision == capi.FP64:
        np.testing.assert_array_equal(gm["collisions"], om["collisions"])
        np.testing.assert_array_equal(gm["wall_count"], om["wall_count"])
        assert_same_clocks(g, o)


def test_hot_particles_take_the_sort_fallback_with_yp():
    # particles so fast that a block's start cells spread beyond the staged span: the
    # per-warp sort path carries the y coordinates too
    sp = [W.Species("e", -1.0, 1.0, 0.5 / 400, 1.0e6, 400, sn2d=1)]  # ~100 cells per step
    phys = W.Physics(ncells=256, dx=0.5, dt=0.05, species=sp, processes=[],
                     field=W.FIELD_NONE, bc=W.BC_PERIODIC, seed=8)
    loads = _with_yp(phys, W.initial_load(phys, seed=8), 8)
    for K in (2, 3):
        g, _ = _run_gpu(phys, loads, 12, capi.FP64, K)
        o, _ = run_oracle(phys, loads, 12)
        for e in _yp_errors(phys, g, o):
            assert e < 1e-12, e


def test_the_flag_changes_nothing_else():
    ensure_built()
    runs = []
    for flag in (0, 1):
        phys = W.magnetized_source(ncells=48, ppc=30, seed=9, nu=0.3, capacity_factor=3.0)
        if flag:
            _flag(phys)
        loads = W.initial_load(phys, seed=9)
        g, m = _run_gpu(phys, loads, 45, capi.FP32, 7)
        runs.append(([by_id(x) for x in g], m))
    (a, ma), (b, mb) = runs
    for x, y in zip(a, b):
        for k in ("cell", "off", "vx", "vy", "vz", "id", "state"):
            np.testing.assert_array_equal(x[k], y[k], err_msg=k)
        assert (x["yp"] == 0).all() and (y["yp"] != 0).any()
    for k in ("live", "wall_count", "collisions", "density", "E"):
        np.testing.assert_array_equal(ma[k], mb[k], err_msg=k)


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_checkpoint_restart_carries_yp(precision):
    ensure_built()
    phys = _flag(W.magnetized_source(ncells=48, ppc=30, seed=10, nu=0.3, capacity_factor=3.0))
    loads = _with_yp(phys, W.initial_load(phys, seed=10), 10)
    ref = capi.Sim(phys, precision=precision, sort_interval=7)
    ref.load_all(loads)
    ref.step(45)
    want = [by_id(ref.particles(0, s, cell_units=True)) for s in range(2)]
    ref.close()
    a = capi.Sim(phys, precision=precision, sort_interval=7)
    a.load_all(loads)
    a.step(25)
    snap = [a.particles(0, s, cell_units=True) for s in range(2)]
    m = a.moments(0)
    a.close()
    b = capi.Sim(phys, precision=precision, sort_interval=7)
    for s, p in enumerate(snap):
        b.load(0, s, W.Load(p["cell"], p["off"], p["vx"], p["vy"], p["vz"], p["id"], p["state"],
                            p["yp"]), cell_units=True)
    b.restore_counters(m["step"], [m["next_id"]])
    b.step(20)
    got = [by_id(b.particles(0, s, cell_units=True)) for s in range(2)]
    b.close()
    for x, y in zip(want, got):
        for k in x:
            np.testing.assert_array_equal(x[k], y[k], err_msg=k)


def test_load_yp_is_checked():
    import ctypes as C
    ensure_built()
    phys = _flag(W.bounded_small(ncells=16, ppc=8, seed=11), species=[0])
    loads = W.initial_load(phys, seed=11)
    sim = capi.Sim(phys, precision=capi.FP32, sort_interval=5)
    sim.load_all(loads)
    n = len(loads[0])
    yp = np.arange(n, dtype=np.float64)
    L = capi.lib()
    assert L.pic_load_yp(sim._h, 0, 0, n - 1, yp.ctypes.data, 0) == -1  # n differs
    assert L.pic_load_yp(sim._h, 0, 1, len(loads[1]), yp.ctypes.data, 0) == -1  # no sn2d
    assert L.pic_load_yp(sim._h, 0, 0, n, yp.ctypes.data, 0) == 0
    got = np.zeros(n)
    cnt = C.c_int64()
    assert L.pic_get_yp(sim._h, 0, 0, n, got.ctypes.data, 0, C.byref(cnt)) == 0
    np.testing.assert_array_equal(np.sort(got), yp)
    sim.step(1)
    assert L.pic_load_yp(sim._h, 0, 0, n, yp.ctypes.data, 0) == -7  # after a step
    sim.step(1)  # the handle stays usable
    sim.sync()
    sim.close()
