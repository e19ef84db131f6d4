"""Pins of the oracle's neutral-particle target (the paper's test case, Section 3 and
Table 1: electrons, D+ ions and D neutrals as particles; ionization depletes the
neutrals, the paper's dn/dt = -n n_e R with the sign read as a decrease).

The model: a collision candidate of an electron in cell j is kept with probability
min(1, n_j / nref) (n_j the live neutrals of cell j at the start of the step), then the
usual process selection; an ionization turns the smallest-id live neutral of cell j
(as of the start of the step) into an ion with the same id, position and velocity, and
creates one electron.

* Logistic law: ionization only, threshold 0, equal initial densities n0 of e, D+, D and
  nref = n0: n + n_e = 2 n0 and dn/dt = -(nu / n0) n n_e give n(t) = 2 n0 / (1 + e^{2 nu t}).
  The oracle's neutral count after T steps must agree within 3 standard errors of the
  event count (the discrete-time and cell-fluctuation corrections are far smaller).
* Exact bookkeeping: every ionization removes one neutral and adds one ion and one
  electron (n_n + n_i and n_e - n_i are conserved); the new ions are exactly the
  smallest-id neutrals of the cells where electrons ionized, with the neutrals'
  positions and velocities; ids stay unique.
* Excitation only: the electrons' kinetic energy drops by exactly E_exc per event.
* The density acceptance halves the collision rate when nref = 2 n0.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2404_10270_gb300 import workloads as W


def _case(ncells=64, ppc=200, nu_el=0.0, nu_exc=0.0, nu_iz=0.0, thr_iz=0.0, thr_exc=0.5,
          nref=None, seed=3, K=20):
    w = 0.5 / ppc
    sp = [W.Species("e", -1.0, 1.0, w, 1.0, ppc, 3.0), W.Species("D+", 1.0, 3670.0, w, 1.0, ppc, 3.0),
          W.Species("D", 0.0, 3670.0, w, 0.05, ppc, 1.0, nstep=K)]
    pr = []
    if nu_el:
        pr.append(W.Process(W.PROC_ELASTIC, 0, nu_el))
    if nu_exc:
        pr.append(W.Process(W.PROC_EXCITE, 0, nu_exc, thr_exc))
    if nu_iz:
        pr.append(W.Process(W.PROC_IONIZE, 0, nu_iz, thr_iz, 1))
    return W.Physics(ncells=ncells, dx=0.5, dt=0.05, species=sp, processes=pr, bc=W.BC_PERIODIC,
                     field=W.FIELD_NONE, T_neutral=0.05, m_neutral=3670.0, seed=seed,
                     sort_interval=K, target=3, nref=nref or ppc)


def test_logistic_depletion():
    nu, steps = 0.05, 400
    phys = _case(ncells=64, ppc=200, nu_iz=nu)
    o = Oracle(phys)
    o.load_all(W.initial_load(phys, seed=3))
    n0 = 64 * 200
    o.step(steps)
    m = o.moments()
    t = steps * phys.dt
    expect = 2 * n0 / (1 + math.exp(2 * nu * t))
    events = n0 - m["live"][2]
    assert m["collisions"][0] == events
    se = math.sqrt(events)
    assert abs(m["live"][2] - expect) < 3 * se, (m["live"][2], expect, se)


def test_ionization_bookkeeping_is_exact():
    phys = _case(ncells=16, ppc=40, nu_iz=0.3, nu_el=0.1, seed=5, K=7)
    o = Oracle(phys)
    o.load_all(W.initial_load(phys, seed=5))
    n0 = 16 * 40
    ids_seen = set()
    for step in range(30):
        before_n = o.particles(2)
        before_i = set(o.particles(1)["id"].tolist())
        o.step(1)
        m = o.moments()
        e, i, n = (int(x) for x in m["live"][:3])
        assert n + i == 2 * n0 and e - i == 0
        after_n = o.particles(2)
        after_i = o.particles(1)
        new_ions = set(after_i["id"].tolist()) - before_i
        gone = set(before_n["id"].tolist()) - set(after_n["id"].tolist())
        assert new_ions == gone
        # the converted neutrals are the smallest ids of their start-of-step cells
        cells = before_n["cell"]
        for cid in gone:
            c = cells[before_n["id"] == cid][0]
            in_cell = np.sort(before_n["id"][cells == c])
            taken = sorted(x for x in gone if cells[before_n["id"] == x][0] == c)
            assert in_cell[:len(taken)].tolist() == taken
        # an ion that was a neutral keeps its (physical) velocity; positions too unless
        # the neutral moved this step (K = 7: moves on steps 6, 13, ...)
        for cid in new_ions:
            a = after_i["id"] == cid
            b = before_n["id"] == cid
            np.testing.assert_allclose(after_i["vx"][a], before_n["vx"][b], rtol=1e-15)
            if (step + 1) % 7 != 0:
                assert after_i["cell"][a][0] == before_n["cell"][b][0]
                assert after_i["off"][a][0] == before_n["off"][b][0]
        allids = np.concatenate([o.particles(s)["id"] for s in range(3)])
        assert len(np.unique(allids)) == len(allids)
        ids_seen |= new_ions
    assert len(ids_seen) > 20


def test_excitation_loses_exactly_the_threshold():
    thr = 0.5
    phys = _case(ncells=8, ppc=100, nu_exc=0.5, thr_exc=thr, seed=7)
    o = Oracle(phys)
    o.load_all(W.initial_load(phys, seed=7))
    k0 = o.moments()["kinetic"][0]
    o.step(20)
    m = o.moments()
    # energy thr (units of T_e) per event, times the weight, per macro-particle
    w = phys.species[0].weight
    assert m["collisions"][0] > 50
    np.testing.assert_allclose(k0 - m["kinetic"][0], m["collisions"][0] * thr * w, rtol=1e-10)


def test_density_acceptance_scales_the_rate():
    nu, steps, ppc = 0.05, 60, 200
    counts = []
    for nref in (ppc, 2 * ppc):
        phys = _case(ncells=64, ppc=ppc, nu_el=nu, nref=nref, seed=11)
        o = Oracle(phys)
        o.load_all(W.initial_load(phys, seed=11))
        o.step(steps)
        counts.append(o.moments()["collisions"][0])
    P = -math.expm1(-nu * 0.05)
    expect = steps * 64 * ppc * P
    for c, f in zip(counts, (1.0, 0.5)):
        assert abs(c - f * expect) < 4 * math.sqrt(f * expect), (c, f * expect)
