"""Pins of the oracle's gather / push / move / wall steps against closed forms.

Each test fixes a result that the mathematics determines independently of the
oracle's code: free streaming, ballistic motion in a uniform field, Boris gyration
(speed and parallel velocity conserved, rotation angle 2 atan(|q/m| B dt/2) per step),
periodic wrap, wall fluxes, and the cold-plasma oscillation frequency.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2404_10270_gb300 import workloads as W
from tests.helpers import positions


def _single_species(ncells=64, dx=0.5, dt=0.05, charge=-1.0, mass=1.0, **kw):
    sp = [W.Species("e", charge, mass, 0.01, 1.0, 0)]
    return W.Physics(ncells=ncells, dx=dx, dt=dt, species=sp, processes=[], **kw)


def _load(cell, off, vx, vy=None, vz=None, id0=0):
    n = len(cell)
    z = np.zeros(n)
    return W.Load(np.asarray(cell, np.int32), np.asarray(off, np.float64),
                  np.asarray(vx, np.float64), z.copy() if vy is None else np.asarray(vy),
                  z.copy() if vz is None else np.asarray(vz),
                  np.arange(id0, id0 + n, dtype=np.uint32))


def test_free_streaming_matches_straight_lines():
    """Field off: x_n = x_0 + n v dt (Section 2 mover with E = 0)."""
    phys = _single_species(ncells=400, field=W.FIELD_NONE)
    rng = np.random.default_rng(3)
    n = 500
    cell = rng.integers(150, 250, n)
    off = rng.random(n)
    v = rng.normal(0.0, 1.0, n)
    o = Oracle(phys)
    o.load(0, _load(cell, off, v))
    steps = 300
    o.step(steps)
    p = o.particles(0)
    x0 = (cell + off) * phys.dx
    expect = x0 + steps * v * phys.dt
    got = positions(p, phys.dx)
    # one rounding of the offset per step, relative to a cell of dx
    assert np.max(np.abs(got - expect)) < 1e-12 * steps
    np.testing.assert_allclose(p["vx"], v, rtol=0, atol=1e-14)


def test_uniform_field_ballistic_closed_form():
    """Uniform external E, velocity updated first (leapfrog):
    v_n = v_0 + n a dt, x_n = x_0 + n dt v_0 + a dt^2 n(n+1)/2."""
    E0 = 0.37
    phys = _single_species(ncells=4000, field=W.FIELD_EXTERNAL, E_ext=E0, charge=-1.0, mass=1.0)
    rng = np.random.default_rng(5)
    n = 200
    cell = rng.integers(1800, 2200, n)
    off = rng.random(n)
    v = rng.normal(0.0, 1.0, n)
    o = Oracle(phys)
    o.load(0, _load(cell, off, v))
    steps = 100
    o.step(steps)
    p = o.particles(0)
    a = -1.0 * E0  # q E / m
    dt = phys.dt
    x0 = (cell + off) * phys.dx
    x_expect = x0 + steps * dt * v + a * dt * dt * steps * (steps + 1) / 2
    v_expect = v + steps * a * dt
    np.testing.assert_allclose(positions(p, phys.dx), x_expect, rtol=0, atol=1e-10)
    np.testing.assert_allclose(p["vx"], v_expect, rtol=0, atol=1e-12)


def test_boris_gyration_conserves_speed_and_rotates_by_known_angle():
    """E = 0, uniform B: the Boris rotation keeps |v| and v_parallel, and turns v_perp
    by exactly 2 atan(|q/m| |B| dt / 2) per step (Boris 1970)."""
    Bmag, th = 2.0, math.radians(80.0)
    B = (Bmag * math.cos(th), Bmag * math.sin(th), 0.0)
    phys = _single_species(ncells=64, field=W.FIELD_NONE, bc=W.BC_PERIODIC, B=B)
    rng = np.random.default_rng(7)
    n = 64
    cell = rng.integers(0, 64, n)
    off = rng.random(n)
    v = rng.normal(0, 1.0, (3, n))
    o = Oracle(phys)
    o.load(0, _load(cell, off, v[0], v[1], v[2]))
    bhat = np.array(B) / Bmag
    speed0 = np.sqrt((v ** 2).sum(0))
    vpar0 = bhat @ v
    expect_angle = 2.0 * math.atan(Bmag * phys.dt / 2.0)
    prev = None
    for _ in range(50):
        o.step(1)
        p = o.particles(0)
        vv = np.stack([p["vx"], p["vy"], p["vz"]])
        np.testing.assert_allclose(np.sqrt((vv ** 2).sum(0)), speed0, rtol=1e-13)
        np.testing.assert_allclose(bhat @ vv, vpar0, rtol=0, atol=1e-13)
        perp = vv - np.outer(bhat, bhat @ vv)
        if prev is not None:
            c = (perp * prev).sum(0) / (np.linalg.norm(perp, axis=0) * np.linalg.norm(prev, axis=0))
            ang = np.arccos(np.clip(c, -1, 1))
            np.testing.assert_allclose(ang, expect_angle, rtol=0, atol=1e-7)
            # electrons (q < 0) gyrate right-handed about B
            cross = np.cross(prev.T, perp.T) @ bhat
            assert np.all(cross > 0)
        prev = perp


def test_periodic_wrap():
    phys = _single_species(ncells=10, field=W.FIELD_NONE, bc=W.BC_PERIODIC)
    dx, dt = phys.dx, phys.dt
    o = Oracle(phys)
    o.load(0, _load([9, 0], [0.5, 0.5], [0.3 * dx / dt, -0.7 * dx / dt]))
    o.step(1)
    p = o.particles(0)
    np.testing.assert_array_equal(p["cell"], [9, 9])
    np.testing.assert_allclose(p["off"], [0.8, 0.8], atol=1e-15)
    o.step(1)
    p = o.particles(0)
    np.testing.assert_array_equal(p["cell"], [0, 9])
    np.testing.assert_allclose(p["off"], [0.1, 0.1], atol=1e-15)


def test_absorbing_walls_count_and_energy():
    """Ballistic particles: exactly those whose straight line leaves [0, L] within n
    steps are absorbed, at the wall they head for, carrying w m v^2 / 2 each."""
    phys = _single_species(ncells=50, field=W.FIELD_NONE)
    rng = np.random.default_rng(11)
    n = 2000
    cell = rng.integers(0, 50, n)
    off = rng.random(n)
    v = rng.normal(0.0, 1.0, (3, n))
    o = Oracle(phys)
    o.load(0, _load(cell, off, v[0], v[1], v[2]))
    steps = 40
    o.step(steps)
    x0 = (cell + off) * phys.dx
    xend = x0 + steps * phys.dt * v[0]
    L = phys.length
    # keep clear of the boundary by a margin that rounding cannot cross
    margin = 1e-9
    assert np.all((np.abs(xend) > margin) & (np.abs(xend - L) > margin))
    left, right = xend < 0, xend >= L
    m = o.moments()
    assert m["wall_count"][0, 0] == left.sum()
    assert m["wall_count"][0, 1] == right.sum()
    ke = 0.5 * 1.0 * 0.01 * (v ** 2).sum(0)
    np.testing.assert_allclose(m["wall_energy"][0], [ke[left].sum(), ke[right].sum()], rtol=1e-12)
    assert m["live"][0] == n - left.sum() - right.sum()
    ids = o.particles(0)["id"]
    np.testing.assert_array_equal(np.sort(ids), np.nonzero(~(left | right))[0])


def test_cold_plasma_oscillation_frequency():
    """Cold electrons displaced by a standing wave over fixed ions oscillate at the
    plasma frequency; leapfrog gives sin(w dt/2) = w_pe dt/2 (w_pe = 1), up to the
    O((k dx)^2) grid correction."""
    phys, loads = W.cold_wave(ncells=256, ppc=16, amplitude=1e-3, mode=2)
    o = Oracle(phys)
    o.load_all(loads)
    L = phys.length
    k = 2 * math.pi / L
    n = len(loads[0])
    x_lattice = (np.arange(n) + 0.5) * (L / n)  # undisplaced electron positions
    proj_w = np.sin(k * x_lattice)
    series = []
    nsteps = 700
    for _ in range(nsteps):
        o.step(1)
        p = o.particles(0)
        disp = positions(p, phys.dx) - x_lattice[p["id"]]
        series.append(float((disp * proj_w[p["id"]]).sum()))
    s = np.array(series)
    # zero crossings by linear interpolation
    idx = np.nonzero(np.sign(s[:-1]) != np.sign(s[1:]))[0]
    t = idx + s[idx] / (s[idx] - s[idx + 1])
    half_periods = np.diff(t)
    period_steps = 2 * half_periods.mean()
    w_meas = 2 * math.pi / (period_steps * phys.dt)
    w_theory = 2.0 / phys.dt * math.asin(phys.dt / 2.0)
    assert len(idx) >= 8
    assert abs(w_meas / w_theory - 1.0) < 2e-3, (w_meas, w_theory)
