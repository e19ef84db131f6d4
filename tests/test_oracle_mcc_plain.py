"""The oracle's collision clock against the plain null-collision definition.

The null-collision method (Skullerud 1968; Vahedi & Surendra 1995) makes every
particle-step a collision candidate with probability P = 1 - exp(-nu_max dt),
independently of every other step, and gives a candidate to process k with
probability nu_k / nu_max.  Its plain form draws one COLLIDE word per particle and step
and compares it with floor(P 2^32).  The oracle instead samples the same sequence
through its geometric runs (the per-particle collision clock, cut at multiples of 127
steps).  These tests check, over runs that span three multiples of 127, that what the
oracle produces is distributed like the plain form:

* candidates per step: Binomial(n, P), also on the grid steps themselves;
* consecutive gaps between candidates: independent geometric(P) pairs, the joint
  table of (gap_i, gap_i+1) against the product of geometric laws, and the same
  statistic on a plain per-step sampler written here (its calibration);
* gaps that straddle a multiple of 127: what remains after the grid step is again
  geometric (memorylessness), and straddles happen as often as (1-P)^D predicts;
* the oracle's and the plain sampler's gap histograms, as two samples of one law;
* the split of events over three processes of unequal nu with zero thresholds: the
  multinomial nu_k / nu_max.

The plain sampler below restates Philox4x32-10 (Salmon et al., SC'11) with numpy
arrays; it is checked against the published known-answer vectors first.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle.oracle import Oracle
from paper_2404_10270_gb300 import workloads as W
from tests.helpers import read_kat

NU = (0.05, 0.10, 0.25)     # three processes, unequal frequencies, zero thresholds
DT = 0.05
NMAX = sum(NU)
P = -math.expm1(-NMAX * DT)  # candidate probability per particle-step (~0.0198)
N_PART = 16000
STEPS = 500                  # grid steps 127, 254, 381 inside the run
CAP = 100                    # gaps binned 1..CAP-1, and >= CAP


def philox_np(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 on arrays of counters (uint32 words), one key."""
    M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
    W0, W1 = 0x9E3779B9, 0xBB67AE85
    c = [np.asarray(x, np.uint64) & np.uint64(0xFFFFFFFF) for x in (c0, c1, c2, c3)]
    k0, k1 = int(k0), int(k1)
    mask = np.uint64(0xFFFFFFFF)
    for r in range(10):
        if r:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        c = [((p1 >> np.uint64(32)) ^ c[1] ^ np.uint64(k0)) & mask, p1 & mask,
             ((p0 >> np.uint64(32)) ^ c[3] ^ np.uint64(k1)) & mask, p0 & mask]
    return [x.astype(np.uint32) for x in c]


def test_numpy_philox_known_answers():
    for ctr, key, out in read_kat():
        got = philox_np(*[np.array([w]) for w in ctr], key[0], key[1])
        assert [int(g[0]) for g in got] == out


def plain_candidates(n, steps, seed):
    """Plain per-step null collision: candidate iff COLLIDE(id, step) word 0 <
    floor(P 2^32).  Returns a boolean array (steps, n)."""
    T = np.uint32(math.floor(P * 2.0 ** 32))
    ids = np.arange(n, dtype=np.uint64)
    out = np.zeros((steps, n), bool)
    for t in range(steps):
        w = philox_np(ids, np.zeros(n), np.full(n, t), np.zeros(n), seed & 0xFFFFFFFF,
                      seed >> 32)
        out[t] = w[0] < T
    return out


@pytest.fixture(scope="module")
def oracle_run():
    """Candidate steps of every particle (boolean array (steps, n)) and the per-process
    event totals of an oracle run with three zero-threshold processes.  Every candidate
    is a real event that changes the velocity (elastic off a very heavy neutral,
    excitation with zero loss, charge exchange), and nothing else changes it (no field,
    periodic walls)."""
    sp = [W.Species("e", -1.0, 1.0, 0.01, 1.0, 0)]
    procs = [W.Process(W.PROC_ELASTIC, 0, NU[0]), W.Process(W.PROC_EXCITE, 0, NU[1], 0.0),
             W.Process(W.PROC_CX, 0, NU[2])]
    phys = W.Physics(ncells=32, dx=0.5, dt=DT, species=sp, processes=procs,
                     field=W.FIELD_NONE, bc=W.BC_PERIODIC, T_neutral=1.0, m_neutral=1e6,
                     seed=77)
    rng = np.random.default_rng(77)
    n = N_PART
    v = rng.normal(0, 1.0, (3, n))
    o = Oracle(phys)
    o.load(0, W.Load(rng.integers(0, 32, n).astype(np.int32), rng.random(n), v[0].copy(),
                     v[1].copy(), v[2].copy(), np.arange(n, dtype=np.uint32)))
    p = o.particles(0)
    prev = np.stack([p["vx"], p["vy"], p["vz"]])
    cand = np.zeros((STEPS, n), bool)
    for t in range(STEPS):
        o.step(1)
        p = o.particles(0)
        cur = np.stack([p["vx"], p["vy"], p["vz"]])
        cand[t] = np.any(cur != prev, axis=0)
        prev = cur
    counts = o.moments()["collisions"]
    assert counts.sum() == cand.sum()
    return cand, counts


SENT = 10 ** 6  # "no later candidate inside the run": longer than any bin


def _gaps(cand):
    """For every candidate of every particle: its step t_i, the gap to the particle's
    next candidate and the gap after that (SENT where the run ends first; callers only
    use gaps whose window lies inside the run, so SENT always lands in a tail bin)."""
    starts, gaps, nexts = [], [], []
    for i in range(cand.shape[1]):
        t = np.nonzero(cand[:, i])[0]
        if len(t) == 0:
            continue
        d = np.append(np.diff(t), SENT)
        starts.append(t)
        gaps.append(d)
        nexts.append(np.append(d[1:], SENT))
    return np.concatenate(starts), np.concatenate(gaps), np.concatenate(nexts)


def _geom_bins(cap):
    """P(gap = g) for g = 1..cap-1 and P(gap >= cap)."""
    g = np.arange(1, cap)
    p = (1 - P) ** (g - 1) * P
    return np.append(p, (1 - P) ** (cap - 1))


def _binned(g, cap):
    return np.bincount(np.minimum(g, cap), minlength=cap + 1)[1:]


def test_candidates_per_step_are_binomial(oracle_run):
    cand, _ = oracle_run
    c = cand.sum(axis=1)
    n = cand.shape[1]
    mean, var = n * P, n * P * (1 - P)
    # the law of the per-step counts: binned chi-square against Binomial(n, P)
    edges = np.unique(np.round(stats.binom.ppf(np.linspace(0, 1, 13)[1:-1], n, P)))
    obs = np.bincount(np.searchsorted(edges, c, side="right"), minlength=len(edges) + 1)
    cdf = np.append(stats.binom.cdf(edges - 1, n, P), 1.0)
    exp = np.diff(np.insert(cdf, 0, 0.0)) * len(c)
    assert stats.chisquare(obs, exp).pvalue > 1e-4, (obs, exp)
    # dispersion: no correlation between the particles of a step
    assert abs(c.var(ddof=1) / var - 1) < 5 * math.sqrt(2.0 / (len(c) - 1))
    # the grid steps (own index a multiple of 127) and the steps after them
    for t in (127, 128, 254, 255, 381, 382):
        assert abs(c[t] - mean) < 5 * math.sqrt(var), (t, c[t], mean)


def test_consecutive_gaps_are_independent_geometric(oracle_run):
    cand, _ = oracle_run
    plain = plain_candidates(cand.shape[1], STEPS, 1077)
    B = 20  # pairs binned: gap 1..B-1, >= B
    for name, c in (("oracle", cand), ("plain", plain)):
        starts, gaps, nexts = _gaps(c)
        # pairs (g_i, g_i+1) with g_i < B whose window [t_i, t_i + 2B] lies inside the
        # run (so a second gap cut off by the end of the run is >= B, the tail bin)
        sel = (starts + 2 * B < STEPS) & (gaps < B)
        a, b = gaps[sel], np.minimum(nexts[sel], B)
        table = np.zeros((B - 1, B))
        np.add.at(table, (a - 1, b - 1), 1)
        pg = _geom_bins(B)
        exp = np.outer(pg[:-1] / pg[:-1].sum(), pg) * table.sum()
        res = stats.chisquare(table.ravel(), exp.ravel())
        assert res.pvalue > 1e-4, (name, res)
        assert exp.min() > 5


def test_gaps_straddling_the_grid_stay_geometric(oracle_run):
    cand, _ = oracle_run
    starts, gaps, _ = _gaps(cand)
    # steps from the gap's start to the next multiple of 127 (the clock's cut)
    D = 127 - (starts % 127)
    ok = starts + D + CAP < STEPS
    s, g, d = starts[ok], gaps[ok], D[ok]
    straddle = g > d
    # how many straddle: sum of (1-P)^D over the gaps, with its binomial spread
    p_st = (1 - P) ** d
    exp_n = p_st.sum()
    assert abs(straddle.sum() - exp_n) < 5 * math.sqrt((p_st * (1 - p_st)).sum())
    # what remains after the grid step is geometric again
    rem = (g - d)[straddle]
    obs = _binned(rem, CAP)
    exp = _geom_bins(CAP) * len(rem)
    assert stats.chisquare(obs, exp).pvalue > 1e-4


def test_oracle_and_plain_sampler_give_one_gap_law(oracle_run):
    cand, _ = oracle_run
    plain = plain_candidates(cand.shape[1], STEPS, 1077)
    hist = []
    for c in (cand, plain):
        starts, gaps, _ = _gaps(c)
        g = gaps[starts + CAP < STEPS]
        hist.append(_binned(g, CAP))
    table = np.array(hist)
    table = table[:, table.min(axis=0) > 0]
    chi2, p, dof, _ = stats.chi2_contingency(table)
    assert p > 1e-4, (chi2, dof)
    # and both have the same per-step event rate, P
    for c in (cand, plain):
        rate = c.mean()
        assert abs(rate - P) < 5 * math.sqrt(P * (1 - P) / c.size)


def test_process_split_follows_the_frequencies(oracle_run):
    _, counts = oracle_run
    total = counts.sum()
    exp = np.array(NU) / NMAX * total
    res = stats.chisquare(counts, exp)
    assert res.pvalue > 1e-4, (counts, exp)
    # unequal frequencies: a slot order mix-up (e.g. reversed bounds) moves counts by
    # far more than the noise
    assert counts[2] > 2 * counts[1] > 2 * counts[0]
