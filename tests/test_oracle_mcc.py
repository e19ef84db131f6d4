"""Pins of the oracle's random numbers and Monte Carlo collision phase.

* Philox4x32-10 against the published known-answer vectors.
* Null-collision statistics against their closed forms: the step of the first
  collision is geometric with p = 1 - exp(-nu dt) (the discrete form of the
  exponential free-flight time); charge exchange relaxes the ion temperature as
  T_n + (T_0 - T_n)(1-p)^n; elastic scattering off neutrals of mass M removes on
  average a fraction 2 m/M of the energy per collision and isotropises a beam.
* Ionization conserves energy exactly (threshold paid once, the rest shared) and
  numbers its products by the rank of the parent id.
* Volume re-injection keeps the particle count and draws uniform positions.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

from oracle.oracle import Oracle, philox
from paper_2404_10270_gb300 import workloads as W
from tests.helpers import read_kat


def test_philox_known_answers():
    rows = read_kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        np.testing.assert_array_equal(philox(ctr, key), np.array(out, dtype=np.uint32))


def _gas(n, charge, mass, procs, T=1.0, T_n=0.05, m_n=100.0, bc=W.BC_PERIODIC, seed=9,
         ncells=32, dt=0.05):
    sp = [W.Species("s", charge, mass, 0.01, T, 0)]
    phys = W.Physics(ncells=ncells, dx=0.5, dt=dt, species=sp, processes=procs,
                     field=W.FIELD_NONE, bc=bc, T_neutral=T_n, m_neutral=m_n, seed=seed)
    rng = np.random.default_rng(seed)
    cell = rng.integers(0, ncells, n).astype(np.int32)
    off = rng.random(n)
    v = rng.normal(0, math.sqrt(T / mass), (3, n))
    ld = W.Load(cell, off, v[0].copy(), v[1].copy(), v[2].copy(), np.arange(n, dtype=np.uint32))
    return phys, ld


def _vel(p):
    return np.stack([p["vx"], p["vy"], p["vz"]])


def test_first_collision_step_is_geometric():
    nu, dt, n = 2.0, 0.05, 20000
    phys, ld = _gas(n, -1.0, 1.0, [W.Process(W.PROC_ELASTIC, 0, nu)], m_n=1e6)
    o = Oracle(phys)
    o.load(0, ld)
    p0 = _vel(o.particles(0))
    first = np.zeros(n, dtype=np.int64)
    total = 0
    prev = p0
    for k in range(1, 61):
        o.step(1)
        v = _vel(o.particles(0))
        changed = np.any(v != prev, axis=0)
        total += int(changed.sum())
        first[(first == 0) & changed] = k
        prev = v
    assert o.moments()["collisions"][0] == total
    P = -math.expm1(-nu * dt)
    ks = np.arange(1, 31)
    expect = n * (1 - P) ** (ks - 1) * P
    obs = np.array([(first == k).sum() for k in ks])
    tail_obs = n - obs.sum()
    tail_exp = n - expect.sum()
    chi = stats.chisquare(np.append(obs, tail_obs), np.append(expect, tail_exp))
    assert chi.pvalue > 1e-4, chi
    # mean number of events per particle-step
    assert abs(total / (60 * n) - P) < 5 * math.sqrt(P * (1 - P) / (60 * n))


def test_collision_gaps_stay_geometric_beyond_the_clock_range():
    """With P ~ 0.01 most runs without a candidate are longer than the 127 steps the
    collision clock can hold; the first collision step must still be geometric."""
    nu, dt, n, steps = 0.2, 0.05, 6000, 700
    phys, ld = _gas(n, -1.0, 1.0, [W.Process(W.PROC_ELASTIC, 0, nu)], m_n=1e6, seed=21)
    o = Oracle(phys)
    o.load(0, ld)
    prev = _vel(o.particles(0))
    first = np.zeros(n, dtype=np.int64)
    for k in range(1, steps + 1):
        o.step(1)
        v = _vel(o.particles(0))
        first[(first == 0) & np.any(v != prev, axis=0)] = k
        prev = v
    P = -math.expm1(-nu * dt)
    edges = np.array([1, 50, 100, 127, 128, 200, 254, 255, 300, 400, 500, 700])
    obs, exp = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        obs.append(((first >= lo) & (first < hi)).sum())
        exp.append(n * ((1 - P) ** (lo - 1) - (1 - P) ** (hi - 1)))
    obs.append((first == 0).sum() + (first >= edges[-1]).sum())
    exp.append(n - sum(exp))
    chi = stats.chisquare(obs, exp)
    assert chi.pvalue > 1e-4, (chi, obs, exp)


def test_charge_exchange_relaxes_ion_temperature():
    nu, n, m = 1.0, 40000, 100.0
    T0, Tn = 1.0, 0.05
    phys, ld = _gas(n, 1.0, m, [W.Process(W.PROC_CX, 0, nu)], T=T0, T_n=Tn, m_n=m)
    o = Oracle(phys)
    o.load(0, ld)
    P = -math.expm1(-nu * phys.dt)
    w = phys.species[0].weight
    ke0 = o.moments()["kinetic"][0] / (w * n)  # mean m v^2 / 2 of the load
    for steps in (10, 30, 60):
        o.step(steps - int(o.moments()["step"]))
        ke = o.moments()["kinetic"][0] / (w * n)
        keep = (1 - P) ** steps
        expect = keep * ke0 + (1 - keep) * 1.5 * Tn
        # per-ion energy variance of a 3D Maxwellian at T: 1.5 T^2
        se = math.sqrt((keep * 1.5 * T0 ** 2 + (1 - keep) * 1.5 * Tn ** 2) / n)
        assert abs(ke - expect) < 5 * se, (steps, ke, expect, se)


def test_elastic_energy_loss_rate():
    nu, n, M = 2.0, 40000, 10.0
    phys, ld = _gas(n, -1.0, 1.0, [W.Process(W.PROC_ELASTIC, 0, nu)], m_n=M)
    o = Oracle(phys)
    o.load(0, ld)
    w = phys.species[0].weight
    e0 = o.moments()["kinetic"][0] / (w * n)
    steps = 20
    o.step(steps)
    e = o.moments()["kinetic"][0] / (w * n)
    P = -math.expm1(-nu * phys.dt)
    expect = e0 * (1 - P * 2 * (1.0 / M)) ** steps
    assert abs(e / expect - 1) < 0.01, (e, expect)


def test_elastic_scattering_isotropises_a_beam():
    nu, n = 2.0, 30000
    phys, ld = _gas(n, -1.0, 1.0, [W.Process(W.PROC_ELASTIC, 0, nu)], m_n=1e9)
    ld.vx[:] = 1.0
    ld.vy[:] = 0.0
    ld.vz[:] = 0.0
    o = Oracle(phys)
    o.load(0, ld)
    o.step(150)
    v = _vel(o.particles(0))
    speed = np.sqrt((v ** 2).sum(0))
    # M/m = 1e9: at most 4e-9 of the energy per collision is lost
    np.testing.assert_allclose(speed, 1.0, rtol=1e-6)
    second = (v ** 2).mean(1)
    # each component^2 of an isotropic unit vector: mean 1/3, variance 4/45
    se = math.sqrt(4.0 / 45.0 / n)
    np.testing.assert_allclose(second, 1.0 / 3.0, atol=5 * se)
    assert abs(v.mean(1)).max() < 5 * math.sqrt(1.0 / 3.0 / n)


def test_ionization_energy_and_child_numbering():
    nu, n = 3.0, 4000
    Eiz = 0.68
    sp = [W.Species("e", -1.0, 1.0, 0.01, 1.0, 0), W.Species("i", 1.0, 100.0, 0.01, 1.0, 0)]
    phys = W.Physics(ncells=16, dx=0.5, dt=0.05, species=sp,
                     processes=[W.Process(W.PROC_IONIZE, 0, nu, Eiz, 1)],
                     field=W.FIELD_NONE, bc=W.BC_PERIODIC, T_neutral=0.05, m_neutral=100.0,
                     seed=4)
    rng = np.random.default_rng(4)
    cell = rng.integers(0, 16, n).astype(np.int32)
    off = rng.random(n)
    # half the electrons below threshold (E = 0.3), half above (E = 2)
    energy = np.where(np.arange(n) % 2 == 0, 0.3, 2.0)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    v = d * np.sqrt(2 * energy)
    e_ld = W.Load(cell, off, v[0].copy(), v[1].copy(), v[2].copy(), np.arange(n, dtype=np.uint32))
    i_ld = W.Load(cell.copy(), off.copy(), np.zeros(n), np.zeros(n), np.zeros(n),
                  np.arange(n, 2 * n, dtype=np.uint32))
    o = Oracle(phys)
    o.load(0, e_ld)
    o.load(1, i_ld)
    m0 = o.moments()
    before = o.particles(0)
    o.step(1)
    m1 = o.moments()
    niz = int(m1["collisions"][0])
    assert niz > 100
    assert m1["live"][0] == n + niz and m1["live"][1] == n + niz
    w = 0.01
    # electron energy drops by exactly the threshold per event (x weight)
    assert abs((m0["kinetic"][0] - m1["kinetic"][0]) - niz * w * Eiz) < 1e-9
    after = o.particles(0)
    ions = o.particles(1)
    old = after["id"] < n
    changed = np.any(_vel(after)[:, old] != _vel(before), axis=0)
    parents = after["id"][old][changed]
    assert len(parents) == niz
    assert np.all(energy[parents] > Eiz)  # nothing below threshold ionized
    # children: electron 2n + 2r, ion 2n + 2r + 1, r = rank of the parent id
    ce = after["id"][~old]
    ci = ions["id"][ions["id"] >= 2 * n]
    np.testing.assert_array_equal(ce, 2 * n + 2 * np.arange(niz))
    np.testing.assert_array_equal(ci, 2 * n + 2 * np.arange(niz) + 1)
    parents = np.sort(parents)
    pos_parent = after["cell"][old][np.searchsorted(after["id"][old], parents)]
    np.testing.assert_array_equal(after["cell"][~old], pos_parent)
    np.testing.assert_array_equal(ions["cell"][ions["id"] >= 2 * n], pos_parent)


def test_volume_source_keeps_count_and_fills_uniformly():
    n = 20000
    sp = [W.Species("e", -1.0, 1.0, 0.01, 1.0, 0)]
    phys = W.Physics(ncells=20, dx=0.5, dt=0.05, species=sp, processes=[],
                     field=W.FIELD_NONE, bc=W.BC_SOURCE, seed=6)
    rng = np.random.default_rng(6)
    cell = rng.integers(0, 20, n).astype(np.int32)
    off = rng.random(n)
    v = rng.normal(0, 200.0, (3, n))  # ~20 cells per step: most leave and re-enter
    o = Oracle(phys)
    o.load(0, W.Load(cell, off, v[0].copy(), v[1].copy(), v[2].copy(),
                     np.arange(n, dtype=np.uint32)))
    v = _vel(o.particles(0))  # as stored (cells/step and back)
    o.step(1)
    m = o.moments()
    hits = int(m["wall_count"][0].sum())
    assert m["live"][0] == n and hits > 0.5 * n
    p = o.particles(0)
    re = np.any(_vel(p) != v, axis=0)
    assert re.sum() == hits
    counts = np.bincount(p["cell"][re], minlength=20)
    assert stats.chisquare(counts).pvalue > 1e-4
    # re-injected velocities: Maxwellian at the source temperature (T = 1, m = 1)
    vre = _vel(p)[:, re]
    se = math.sqrt(2.0 / re.sum())
    np.testing.assert_allclose((vre ** 2).mean(1), 1.0, atol=5 * se)


def test_result_does_not_depend_on_load_order():
    """All 8! orderings of an 8-particle load (with collisions, walls and the
    self-consistent field) give bit-identical particles and counters."""
    sp = [W.Species("e", -1.0, 1.0, 0.5, 1.0, 0), W.Species("i", 1.0, 4.0, 0.5, 1.0, 0)]
    phys = W.Physics(ncells=6, dx=0.5, dt=0.2, species=sp,
                     processes=[W.Process(W.PROC_ELASTIC, 0, 3.0), W.Process(W.PROC_CX, 1, 3.0)],
                     T_neutral=0.1, m_neutral=4.0, seed=12)
    rng = np.random.default_rng(12)
    n = 8
    cell = rng.integers(0, 6, n).astype(np.int32)
    off = rng.random(n)
    v = rng.normal(0, 1.0, (3, n))
    spc = np.array([0, 1, 0, 1, 0, 1, 0, 1])
    ref = None
    for perm in itertools.permutations(range(n)):
        perm = np.array(perm)
        o = Oracle(phys)
        for s in (0, 1):
            idx = perm[spc[perm] == s]
            o.load(s, W.Load(cell[idx], off[idx], v[0][idx], v[1][idx], v[2][idx],
                             idx.astype(np.uint32)))
        o.step(6)
        m = o.moments()
        out = (o.particles(0), o.particles(1), m["wall_count"], m["collisions"], m["E"])
        if ref is None:
            ref = out
            assert m["collisions"].sum() > 0 and m["wall_count"].sum() >= 0
            continue
        for a, b in zip(ref[:2], out[:2]):
            for k in a:
                np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(ref[2], out[2])
        np.testing.assert_array_equal(ref[3], out[3])
        np.testing.assert_array_equal(ref[4], out[4])
