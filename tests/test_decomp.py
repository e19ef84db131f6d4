"""The domain decomposition of one instance by cells (the paper's Section 2), on CPU:
its host logic alone, then two and three gloo ranks (with three, the middle one
exchanges with both neighbours), each stepping its part of an instance with the
oracle's particle step, the field solved jointly, against the oracle's undivided run;
with elastic + charge exchange, and with electron-impact ionization as well (the
children renumbered by their parents' ranks over all subdomains); a periodic instance
(no field solve), whose ranks form a ring; and the paper's own test case (periodic,
neutral particle targets that ionization converts) with the target halo and the
hand-over of ionizations recorded in a neighbour's cell.

Velocities cross the oracle's interface in physical units; with dt/dx a power of two
(here 1/8) that conversion is exact, so a particle that changes rank keeps its state
bit for bit."""
import os
import socket
from fractions import Fraction

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle.oracle import Oracle, poisson as oracle_poisson
from paper_2404_10270_gb300 import workloads as W
from paper_2404_10270_gb300.decomp import Subdomain, fixed_deposit, partition
from tests.gpu_common import by_id

STEPS = 40


def _physics(ionize=False, periodic=False):
    phys = W.bounded_small(ncells=64, ppc=40, seed=21, nu=0.2, dt=0.0625)
    if ionize:  # electron-impact ionization (threshold 13.6 eV / T_e 20 eV) into the ions
        phys.processes.append(W.Process(W.PROC_IONIZE, 0, 0.2, 13.6 / 20.0, 1))
    if periodic:  # the ends joined; no grounded-wall field solve
        phys.bc = W.BC_PERIODIC
        phys.field = W.FIELD_NONE
    return phys


def test_partition_covers_the_cells_and_balances():
    rng = np.random.default_rng(0)
    counts = rng.integers(0, 100, 500)
    for world in (1, 2, 3, 7):
        cuts = partition(counts, world)
        assert cuts[0] == 0 and cuts[-1] == 500 and len(cuts) == world + 1
        assert all(b > a for a, b in zip(cuts, cuts[1:]))
        loads = [counts[a:b].sum() for a, b in zip(cuts, cuts[1:])]
        assert max(loads) - min(loads) <= 2 * counts.max()
    assert partition([0, 0, 5, 0], 4) == [0, 1, 2, 3, 4]  # one cell each at least
    with pytest.raises(ValueError):
        partition([1, 1], 3)


def test_split_deposit_adds_up_to_the_whole_one():
    rng = np.random.default_rng(1)
    N, n = 50, 4000
    cell = rng.integers(0, N, n)
    off = rng.random(n)
    whole = fixed_deposit(cell, off, 0, N)
    cuts = [0, 17, 31, N]
    total = np.zeros(N + 1, np.int64)
    for a, b in zip(cuts, cuts[1:]):
        m = (cell >= a) & (cell < b)
        total[a:b + 1] += fixed_deposit(cell[m], off[m], a, b)
    np.testing.assert_array_equal(total, whole)
    assert whole.sum() == n * (1 << 48)  # every particle adds one unit


def test_one_periodic_rank_joins_node_n_to_node_0():
    rng = np.random.default_rng(3)
    N = 20
    cell = rng.integers(0, N, 500)
    off = rng.random(500)
    dep = fixed_deposit(cell, off, 0, N)[None, :]
    got = Subdomain(N, [0, N], 0, 0.5, periodic=True).exchange_shared(dep)
    assert got[0, 0] == got[0, N] == dep[0, 0] + dep[0, N]
    np.testing.assert_array_equal(got[0, 1:N], dep[0, 1:N])
    with pytest.raises(ValueError):
        Subdomain(N, [0, N], 0, 0.5, periodic=True).field([Fraction(0)] * (N + 1))


def test_whole_instance_field_is_the_dirichlet_solution():
    # uniform charge: phi_i = (dx^2 rho / eps0) i (N - i) / 2, E linear, exactly
    N, dx = 16, 0.5
    sub = Subdomain(N, [0, N], 0, dx)
    rho = [Fraction(3, 4)] * (N + 1)
    E = sub.field(rho)
    for i in range(1, N):
        # E_i = (phi_{i-1} - phi_{i+1}) / (2 dx) = (dx rho / eps0) (i - N/2)
        assert E[i] == float(Fraction(dx) * Fraction(3, 4) * (i - Fraction(N, 2)))
    # a random charge against the oracle's binary128 Thomas solve (both round once)
    rng = np.random.default_rng(2)
    rho = rng.normal(0, 1, N + 1)
    E = sub.field([Fraction(float(r)) for r in rho])
    _, E_o = oracle_poisson(rho, dx)
    np.testing.assert_array_equal(E, E_o)


def test_births_are_renumbered_by_the_parents_rank_over_all_subdomains(monkeypatch):
    # two subdomains' parents of one step: rank 0 had 3 and 11, rank 1 had 7; children
    # of the r-th parent overall are base + 2r (electron) and base + 2r + 1 (ion)
    base = 100
    sub = Subdomain(16, [0, 8, 16], 0, 0.5)
    monkeypatch.setattr(sub, "_gather", lambda obj: [np.array([3, 11]), np.array([7])])
    e = dict(id=np.array([3, 11, 100, 102], np.uint32), cell=np.arange(4))
    i = dict(id=np.array([5, 101, 103], np.uint32), cell=np.arange(3))
    (e2, i2), nxt = sub.renumber_births([e, i], np.array([3, 11]), base, 2)
    np.testing.assert_array_equal(e2["id"], [3, 11, 100, 104])  # parent 11 is 3rd overall
    np.testing.assert_array_equal(i2["id"], [5, 101, 105])
    np.testing.assert_array_equal(e2["cell"], e["cell"])
    assert e2["id"].dtype == np.uint32 and nxt == base + 2 * 3
    # with a neutral particle target one id a parent (the ion is a converted target)
    (e3,), nxt = sub.renumber_births([dict(id=np.array([100, 101], np.uint32))],
                                     np.array([3, 11]), base, 1)
    np.testing.assert_array_equal(e3["id"], [100, 102])
    assert nxt == base + 3
    # a parent on two ranks, or a child without a parent, is refused
    monkeypatch.setattr(sub, "_gather", lambda obj: [np.array([3, 11]), np.array([11])])
    with pytest.raises(ValueError):
        sub.renumber_births([e, i], np.array([3, 11]), base, 2)
    monkeypatch.setattr(sub, "_gather", lambda obj: [np.array([3])])
    with pytest.raises(ValueError):
        sub.renumber_births([e, i], np.array([3]), base, 2)


def test_oracle_follows_a_supplied_field():
    # the oracle handed its own field every step takes the same steps bit for bit
    phys = _physics()
    loads = W.initial_load(phys, seed=21)
    a, b = Oracle(phys), Oracle(phys)
    a.load_all(loads)
    b.load_all(loads)
    for _ in range(10):
        b.set_field(a.moments()["E"])
        a.step(1)
        b.step(1)
    for s in range(2):
        pa, pb = by_id(a.particles(s)), by_id(b.particles(s))
        for k in pa:
            np.testing.assert_array_equal(pa[k], pb[k])
    # and a supplied zero field is no field
    c = Oracle(phys)
    c.load_all(loads)
    c.set_field(np.zeros(phys.ncells + 1))
    c.step(1)
    assert not np.array_equal(by_id(c.particles(0))["vx"], by_id(a.particles(0))["vx"])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _joint_field(sub, parts, qw):
    """This rank's E on all N+1 nodes (its own nodes set, zero elsewhere)."""
    dep = np.stack([fixed_deposit(p["cell"], p["off"], sub.lo, sub.hi) for p in parts])
    dep = sub.exchange_shared(dep)
    E = np.zeros(sub.N + 1)
    E[sub.lo:sub.hi + 1] = sub.field(sub.rho(dep, qw))
    return E, dep


def _rank(rank, world, port, q, ionize, periodic):
    try:
        _rank_body(rank, world, port, q, ionize, periodic)
    except BaseException as e:  # reported, so that the test fails at once
        q.put((rank, "error", repr(e)))
        raise


def _rank_body(rank, world, port, q, ionize, periodic):
    import datetime
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    # a rank that fails leaves the others in a collective: they give up after a minute
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    try:
        phys = _physics(ionize, periodic)
        N = phys.ncells
        loads = W.initial_load(phys, seed=21)
        cuts = partition(np.bincount(np.concatenate([ld.cell for ld in loads]), minlength=N),
                         world)
        sub = Subdomain(N, cuts, rank, phys.dx, phys.eps0, periodic=periodic)
        qw = [s.charge * s.weight for s in phys.species]
        orc = Oracle(phys)  # the whole grid; only this rank's particles in it
        for s, ld in enumerate(loads):
            m = (ld.cell >= sub.lo) & (ld.cell < sub.hi)
            orc.load(s, ld.take(m))
        # the instance's next free id (every rank's created ids count from it)
        base = int(max(ld.id.max() for ld in loads)) + 1
        orc.set_step(0, base)
        first = None
        for n in range(STEPS):
            parts = [orc.particles(s) for s in range(len(loads))]
            if periodic:  # the shared nodes' deposit only: no field solve
                E = None
                dep = sub.exchange_shared(np.stack(
                    [fixed_deposit(p["cell"], p["off"], sub.lo, sub.hi) for p in parts]))
            else:
                E, dep = _joint_field(sub, parts, qw)
            if n == 0:
                first = (None if E is None else E[sub.lo:sub.hi + 1].copy(), dep)
            if E is not None:
                orc.set_field(E)
            orc.step(1)
            # children numbered over all ranks' parents, then the particles that crossed
            # an edge change rank; the rest are loaded back
            parts, base = sub.renumber_births([orc.particles(s) for s in range(len(loads))],
                                              orc.last_parents(), base, 2)
            for s in range(len(loads)):
                p = sub.migrate(parts[s])
                orc.load(s, W.Load(p["cell"], p["off"], p["vx"], p["vy"], p["vz"],
                                   p["id"].astype(np.uint32), p["state"].astype(np.uint8)))
            orc.set_step(n + 1, base)
        m = orc.moments()
        q.put((rank, cuts, first, [orc.particles(s) for s in range(len(loads))],
               m["wall_count"], m["collisions"], m["live"]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ionize,periodic", [(False, False), (True, False), (True, True)])
@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reproduce_the_undivided_oracle_run(world, ionize, periodic):
    phys = _physics(ionize, periodic)
    loads = W.initial_load(phys, seed=21)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q, ionize, periodic), daemon=True)
             for r in range(world)]
    for p in procs:
        p.start()
    try:
        got = [q.get(timeout=300) for _ in procs]
        errors = [g for g in got if g[1] == "error"]
        assert not errors, errors
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    out = sorted(got, key=lambda t: t[0])
    for p in procs:
        assert p.exitcode == 0
    cuts = out[0][1]
    assert len(cuts) == world + 1 and all(0 < c < phys.ncells for c in cuts[1:-1])

    # the joint deposit and field of the first step equal the undivided ones bit for bit
    whole = Subdomain(phys.ncells, [0, phys.ncells], 0, phys.dx, phys.eps0, periodic=periodic)
    parts = [dict(cell=ld.cell, off=ld.off) for ld in loads]
    if periodic:
        E1 = None
        dep1 = whole.exchange_shared(np.stack(
            [fixed_deposit(p["cell"], p["off"], 0, phys.ncells) for p in parts]))
    else:
        E1, dep1 = _joint_field(whole, parts, [s.charge * s.weight for s in phys.species])
    for rank, c, (E_r, dep_r), *_ in out:
        lo, hi = c[rank], c[rank + 1]
        if E1 is not None:
            np.testing.assert_array_equal(E_r, E1[lo:hi + 1])
        np.testing.assert_array_equal(dep_r, dep1[:, lo:hi + 1])

    # against the oracle's own undivided run (its field in binary128 from the exact
    # weights, the joint one from the fixed-point deposit): counters bit for bit,
    # particles within the FP64 form's tolerance
    o = Oracle(phys)
    o.load_all(loads)
    o.step(STEPS)
    om = o.moments()
    np.testing.assert_array_equal(sum(o_[4] for o_ in out), om["wall_count"])
    np.testing.assert_array_equal(sum(o_[5] for o_ in out), om["collisions"])
    np.testing.assert_array_equal(sum(o_[6] for o_ in out), om["live"])
    assert om["collisions"].sum() > 0 and (periodic or om["wall_count"].sum() > 0)
    if ionize:
        assert om["collisions"][2] > 100  # children numbered over all subdomains
    L = phys.ncells
    moved = wrapped = 0
    for s in range(len(phys.species)):
        want = by_id(o.particles(s))
        got = {k: np.concatenate([o_[3][s][k] for o_ in out]) for k in want}
        got = by_id(got)
        np.testing.assert_array_equal(got["id"], want["id"])
        np.testing.assert_array_equal(got["state"], want["state"])
        if periodic:  # no field: every particle's arithmetic is the undivided run's
            for k in ("cell", "off", "vx", "vy", "vz"):
                np.testing.assert_array_equal(got[k], want[k])
        x_got = got["cell"] + got["off"]
        x_want = want["cell"] + want["off"]
        assert np.abs(x_got - x_want).max() / L < 1e-12
        vscale = max(np.abs(want["vx"]).max(), 1.0)
        for k in ("vx", "vy", "vz"):
            assert np.abs(got[k] - want[k]).max() / vscale < 1e-12
        # some particles did change rank
        ld = loads[s]
        start = dict(zip(ld.id.tolist(), ld.cell.tolist()))
        owner = lambda c: int(np.searchsorted(cuts, c, side="right")) - 1  # noqa: E731
        moved += sum(owner(start[i]) != owner(c)
                     for i, c in zip(want["id"].tolist(), want["cell"].tolist()) if i in start)
        # (periodic: some went around the ring's join, between the last rank and the first)
        wrapped += sum(abs(c - start[i]) > L // 2
                       for i, c in zip(want["id"].tolist(), want["cell"].tolist()) if i in start)
    assert moved > 0
    assert (wrapped > 0) == periodic


def _paper_physics():
    # the paper's test case on 64 cells; dt/dx = 1/8 and a target subcycling factor of 4
    # keep the conversions of velocities at the oracle's interface exact
    return W.ionization_case(ncells=64, ppc=40, nu_el=0.05, nu_exc=0.05, nu_iz=0.1, seed=27,
                             sort_interval=4, dt=0.0625)


def _paper_rank(rank, world, port, q):
    try:
        _paper_rank_body(rank, world, port, q)
    except BaseException as e:  # reported, so that the test fails at once
        q.put((rank, "error", repr(e)))
        raise


def _paper_rank_body(rank, world, port, q):
    import datetime
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    try:
        phys = _paper_physics()
        N, S, t = phys.ncells, len(phys.species), phys.target - 1
        loads = W.initial_load(phys, seed=27)
        cuts = partition(np.bincount(np.concatenate([ld.cell for ld in loads]), minlength=N),
                         world)
        sub = Subdomain(N, cuts, rank, phys.dx, phys.eps0, periodic=True)
        orc = Oracle(phys)
        for s, ld in enumerate(loads):
            m = (ld.cell >= sub.lo) & (ld.cell < sub.hi)
            orc.load(s, ld.take(m))
        base = int(max(ld.id.max() for ld in loads)) + 1
        orc.set_step(0, base)
        handed = 0
        keys = ("cell", "off", "vx", "vy", "vz", "id", "state")
        for n in range(STEPS):
            own = orc.particles(t)
            halo = sub.halo(own)
            both = {k: np.concatenate([own[k], halo[k]]) for k in keys}
            orc.load(t, W.Load(*[both[k] for k in keys]))
            orc.step_loop()
            away = orc.births_take(sub.lo, sub.hi)
            handed += len(away)
            orc.births_add(sub.hand_over_births(away))
            orc.step_finish()
            parts = [orc.particles(s) for s in range(S)]
            keep = ~np.isin(parts[t]["id"], halo["id"])  # the halo copies go
            parts[t] = {k: v[keep] for k, v in parts[t].items()}
            parts, base = sub.renumber_births(parts, orc.last_parents(), base, 1)
            for s in range(S):
                p = sub.migrate(parts[s])
                orc.load(s, W.Load(*[np.asarray(p[k]).astype(
                    {"cell": np.int32, "id": np.uint32, "state": np.uint8}.get(k, np.float64))
                    for k in keys]))
            orc.set_step(n + 1, base)
        m = orc.moments()
        q.put((rank, cuts, handed, [orc.particles(s) for s in range(S)], m["collisions"],
               m["live"]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_reproduce_the_papers_test_case(world):
    phys = _paper_physics()
    loads = W.initial_load(phys, seed=27)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_paper_rank, args=(r, world, port, q), daemon=True)
             for r in range(world)]
    for p in procs:
        p.start()
    try:
        got = [q.get(timeout=300) for _ in procs]
        errors = [g for g in got if g[1] == "error"]
        assert not errors, errors
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    out = sorted(got, key=lambda t: t[0])
    o = Oracle(phys)
    o.load_all(loads)
    o.step(STEPS)
    om = o.moments()
    np.testing.assert_array_equal(sum(r[4] for r in out), om["collisions"])
    np.testing.assert_array_equal(sum(r[5] for r in out), om["live"])
    assert om["collisions"][2] > 50  # ionizations converted neutrals into ions
    assert om["live"][2] < len(loads[2])
    assert sum(r[2] for r in out) > 0  # some were recorded in a neighbour's cell
    for s in range(len(phys.species)):  # no field: every particle as undivided, bit for bit
        want = by_id(o.particles(s))
        got_s = by_id({k: np.concatenate([r[3][s][k] for r in out]) for k in want})
        for k in ("id", "state", "cell", "off", "vx", "vy", "vz"):
            np.testing.assert_array_equal(got_s[k], want[k], err_msg="species %d %s" % (s, k))
