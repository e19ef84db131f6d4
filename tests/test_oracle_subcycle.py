"""Pins of the oracle's per-species subcycling (Listing 7's x += nstep*vx) against
closed forms.

A species with subcycling factor K is advanced on the steps n = K-1, 2K-1, ... (so that
every species is at the same time at the multiples of K dt) with the time step K dt and
deposited every step, so after n steps it has made floor(n/K) moves of K dt each: free
streaming gives x = x_0 + floor(n/K) K v dt; in a uniform field
the leapfrog with step K dt gives, after m moves, v_m = v_0 + m a K dt and
x_m = x_0 + m K dt v_0 + a (K dt)^2 m (m+1)/2; and the candidate steps of its collision
clock are a Bernoulli sequence on its own steps with P = 1 - exp(-nu K dt).  K = 1 is
the plain step (the same numbers as without subcycling).
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2404_10270_gb300 import workloads as W
from tests.helpers import positions


def _species(K, charge=-1.0, mass=1.0):
    return [W.Species("e", charge, mass, 0.01, 1.0, 0, nstep=K)]


def _load(cell, off, vx):
    n = len(cell)
    z = np.zeros(n)
    return W.Load(np.asarray(cell, np.int32), np.asarray(off, np.float64),
                  np.asarray(vx, np.float64), z.copy(), z.copy(), np.arange(n, dtype=np.uint32))


@pytest.mark.parametrize("K,steps", [(1, 40), (3, 40), (4, 40), (7, 20)])
def test_subcycled_free_streaming(K, steps):
    phys = W.Physics(ncells=400, dx=0.5, dt=0.05, species=_species(K), processes=[],
                     field=W.FIELD_NONE)
    rng = np.random.default_rng(K)
    n = 300
    cell, off, v = rng.integers(150, 250, n), rng.random(n), rng.normal(0.0, 1.0, n)
    o = Oracle(phys)
    o.load(0, _load(cell, off, v))
    o.step(steps)
    p = o.particles(0)
    moves = steps // K
    expect = (cell + off) * phys.dx + moves * K * v * phys.dt
    assert np.max(np.abs(positions(p, phys.dx) - expect)) < 1e-12 * steps
    # velocities are returned in physical units whatever K is
    np.testing.assert_allclose(p["vx"], v, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("K", [2, 5])
def test_subcycled_uniform_field_ballistic(K):
    E0 = 0.37
    phys = W.Physics(ncells=4000, dx=0.5, dt=0.05, species=_species(K), processes=[],
                     field=W.FIELD_EXTERNAL, E_ext=E0)
    rng = np.random.default_rng(11)
    n = 200
    cell, off, v = rng.integers(1800, 2200, n), rng.random(n), rng.normal(0.0, 1.0, n)
    o = Oracle(phys)
    o.load(0, _load(cell, off, v))
    m = 20
    o.step(m * K)
    p = o.particles(0)
    a, h = -E0, K * phys.dt
    x_expect = (cell + off) * phys.dx + m * h * v + a * h * h * m * (m + 1) / 2
    np.testing.assert_allclose(positions(p, phys.dx), x_expect, rtol=0, atol=1e-10)
    np.testing.assert_allclose(p["vx"], v + m * a * h, rtol=0, atol=1e-12)
    # the next K - 1 steps change nothing; the K-th moves again
    o.step(K - 1)
    q1 = o.particles(0)
    for k in ("cell", "off", "vx"):
        np.testing.assert_array_equal(q1[k], p[k])
    o.step(1)
    q2 = o.particles(0)
    assert np.any(q2["off"] != p["off"])


def test_subcycled_collision_rate_uses_the_species_step():
    """Elastic collisions at frequency nu: a species with K = 4 collides on its own
    steps with P = 1 - exp(-4 nu dt) per move, so over n steps the expected count is
    floor(n/4) N P (an elastic event changes the direction only, never the count)."""
    K, nu, dt = 4, 0.02, 0.05
    ppc, ncells = 400, 64
    sp = [W.Species("e", -1.0, 1.0, 0.5 / ppc, 1.0, ppc, nstep=K)]
    phys = W.Physics(ncells=ncells, dx=0.5, dt=dt, species=sp,
                     processes=[W.Process(W.PROC_ELASTIC, 0, nu)], bc=W.BC_PERIODIC,
                     field=W.FIELD_NONE, m_neutral=1000.0, seed=9)
    loads = W.initial_load(phys, seed=9)
    o = Oracle(phys)
    o.load_all(loads)
    steps = 400
    o.step(steps)
    got = o.moments()["collisions"][0]
    npart = ppc * ncells
    P = -math.expm1(-nu * K * dt)
    expect = (steps // K) * npart * P
    sd = math.sqrt(expect * (1 - P))
    assert abs(got - expect) < 4 * sd, (got, expect, sd)
    # the same physics without subcycling collides about K times as often per move
    # but the same number of times per unit time: the rates agree within the noise
    sp1 = [W.Species("e", -1.0, 1.0, 0.5 / ppc, 1.0, ppc, nstep=1)]
    phys1 = W.Physics(ncells=ncells, dx=0.5, dt=dt, species=sp1,
                      processes=[W.Process(W.PROC_ELASTIC, 0, nu)], bc=W.BC_PERIODIC,
                      field=W.FIELD_NONE, m_neutral=1000.0, seed=9)
    o1 = Oracle(phys1)
    o1.load_all(W.initial_load(phys1, seed=9))
    o1.step(steps)
    got1 = o1.moments()["collisions"][0]
    assert abs(got1 - got) < 4 * math.sqrt(got + got1)
