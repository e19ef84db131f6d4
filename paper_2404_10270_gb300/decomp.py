"""Host side of one instance split over several ranks by cells: the one-dimensional
domain decomposition of the paper's Section 2, as designed for one process per GPU.

Rank r of R owns the cells [c_r, c_{r+1}) and the nodes [c_r, c_{r+1}]; node c_r is
shared with rank r-1.  Per step the ranks exchange, with torch.distributed (NCCL
between GPUs; gloo on CPU in the tests):

1. the fixed-point deposit of each shared node (a particle adds S - Q to node j and Q to
   node j+1, Q = rint(f S)), int64, point to point with the neighbour and added:
   integer addition, so the split deposit equals the whole one bit for bit;
2. the field.  The Dirichlet solution of -phi_{i-1} + 2 phi_i - phi_{i+1} =
   dx^2 rho_i / eps0, phi_0 = phi_N = 0, is
       phi_i = (dx^2 / eps0) [((N - i) / N) L_i + (i / N) R_i],
       L_i = sum_{1 <= k <= i} k rho_k,   R_i = sum_{i < k <= N-1} (N - k) rho_k,
   a two-level scan: every rank sums its own interior nodes, one all-gather of the R
   pairs of totals gives each rank the sums before and after it, and the potentials
   next to its edges come from the neighbours in a second exchange.  E = -dphi/dx
   (centred inside, Gauss's law over the half cell at a wall) is the exact value
   rounded once;
3. the particles that crossed an edge (cell, offset, velocities, id, collision
   clock), point to point to the neighbour;
4. with neutral particle targets (the paper's test case), two more: before the step each
   rank receives a copy of the neighbours' targets in the cell next to each of its edges
   (a one-cell halo), so that an electron that crosses an edge during the step meets the
   start-of-step target count of the cell it collides in; and between the particle loop
   and the creation of products, an ionization recorded in a neighbour's cell goes to
   that neighbour, which converts its targets for it together with its own (a cell's
   first r_j targets by id, the requests in the order of their parents' ids); the halo
   copies are dropped after the step;
5. the ids of the step's ionization products: the children of a step's ionizations are
   numbered by the rank of their parent's id among all the step's ionizing parents of
   the instance, so the ranks all-gather their parents' ids and each renumbers its own
   children (a child's state comes from its parent's draws and its first collision-clock
   test is drawn with its id only on the next step, so the renumbering between steps
   leaves the undivided run's arithmetic as it is).

The sums are exact (integers and rationals), so the field and the particles do not
depend on the number of ranks.  The particle step itself is the library's mover; the
tests drive this protocol with a CPU stepper per rank.
"""
from __future__ import annotations

from fractions import Fraction
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

S48 = 1 << 48  # fixed-point unit of one particle's charge (the FP64 form's)


def partition(cell_counts: Sequence[int], world: int) -> List[int]:
    """Cuts 0 = c_0 < c_1 < ... < c_R = N of N cells into `world` contiguous ranges
    with about equal particle counts (each range at least one cell)."""
    counts = np.asarray(cell_counts, dtype=np.int64)
    N = len(counts)
    if world < 1 or world > N:
        raise ValueError("need 1 <= world <= ncells")
    cum = np.concatenate([[0], np.cumsum(counts)])
    total = int(cum[-1])
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        c = int(np.searchsorted(cum, target, side="left"))
        c = max(c, cuts[-1] + 1)          # at least one cell per range
        c = min(c, N - (world - r))       # and room for the ranges after it
        cuts.append(c)
    cuts.append(N)
    return cuts


def fixed_deposit(cell: np.ndarray, off: np.ndarray, lo: int, hi: int,
                  S: int = S48) -> np.ndarray:
    """Fixed-point cloud-in-cell deposit of particles in cells [lo, hi) on the nodes
    lo..hi (int64): S - Q on node j, Q = rint(f S) (ties to even) on node j+1."""
    dep = np.zeros(hi - lo + 1, dtype=np.int64)
    if len(cell) == 0:
        return dep
    j = np.asarray(cell, dtype=np.int64) - lo
    if j.min() < 0 or j.max() >= hi - lo:
        raise ValueError("particle outside the subdomain")
    Q = np.rint(np.asarray(off, dtype=np.float64) * float(S)).astype(np.int64)
    np.add.at(dep, j, S - Q)
    np.add.at(dep, j + 1, Q)
    return dep


class Subdomain:
    """Rank `rank`'s part of an N-cell instance cut at `cuts` (from partition), with
    the exchanges of one step.  `world` 1 (no torch.distributed needed) is the whole
    instance, solved by the same arithmetic.  periodic: the instance's ends are joined
    (node N is node 0), so the ranks form a ring: the last and the first share that
    node, and a particle that wraps around goes to the rank at the other end (a periodic
    instance has no Poisson solve with grounded walls, so no field is exchanged)."""

    def __init__(self, N: int, cuts: Sequence[int], rank: int, dx: float, eps0: float = 1.0,
                 periodic: bool = False):
        self.periodic = bool(periodic)
        self.N = int(N)
        self.cuts = [int(c) for c in cuts]
        self.world = len(self.cuts) - 1
        self.rank = int(rank)
        self.lo, self.hi = self.cuts[rank], self.cuts[rank + 1]
        self.dx = Fraction(dx)
        self.eps0 = Fraction(eps0)
        if not (0 <= rank < self.world) or self.cuts[0] != 0 or self.cuts[-1] != N:
            raise ValueError("bad cuts or rank")

    # -- 1. the shared nodes' deposit -----------------------------------------------
    def _ring(self):
        """The distinct neighbours of a periodic rank: (left, right), left == right for two
        ranks, none for one."""
        R, r = self.world, self.rank
        return [] if R == 1 else sorted({(r - 1) % R, (r + 1) % R})

    def exchange_shared(self, dep: np.ndarray) -> np.ndarray:
        """dep: int64 [species, hi - lo + 1], this rank's deposit on its nodes.  Returns
        it with each shared node holding the sum of both neighbours' deposits."""
        dep = np.array(dep, dtype=np.int64, copy=True)
        if self.periodic:
            return self._exchange_ring(dep)
        if self.world == 1:
            return dep
        import torch
        import torch.distributed as dist
        ops, inbox = [], {}
        for nb, col in ((self.rank - 1, 0), (self.rank + 1, -1)):
            if 0 <= nb < self.world:
                send = torch.from_numpy(np.ascontiguousarray(dep[:, col]))
                recv = torch.zeros_like(send)
                ops.append(dist.isend(send, nb))
                ops.append(dist.irecv(recv, nb))
                inbox[col] = recv
        for op in ops:
            op.wait()
        for col, recv in inbox.items():
            dep[:, col] += recv.numpy()
        return dep

    def _exchange_ring(self, dep: np.ndarray) -> np.ndarray:
        # the first column (node lo) is shared with the left neighbour's last column, the
        # last (node hi) with the right neighbour's first; the tag says which edge a
        # column is, so two ranks, each the other's left and right neighbour, match up
        R, r = self.world, self.rank
        if R == 1:  # node N is node 0 of the same rank
            tot = dep[:, 0] + dep[:, -1]
            dep[:, 0] = tot
            dep[:, -1] = tot
            return dep
        import torch
        import torch.distributed as dist
        left, right = (r - 1) % R, (r + 1) % R
        send_l = torch.from_numpy(np.ascontiguousarray(dep[:, 0]))
        send_r = torch.from_numpy(np.ascontiguousarray(dep[:, -1]))
        recv_l, recv_r = torch.zeros_like(send_l), torch.zeros_like(send_r)
        ops = [dist.isend(send_l, left, tag=0), dist.isend(send_r, right, tag=1),
               dist.irecv(recv_l, left, tag=1), dist.irecv(recv_r, right, tag=0)]
        for op in ops:
            op.wait()
        dep[:, 0] += recv_l.numpy()
        dep[:, -1] += recv_r.numpy()
        return dep

    # -- 2. the field ---------------------------------------------------------------
    def rho(self, dep: np.ndarray, qw: Sequence[float], S: int = S48) -> List[Fraction]:
        """Exact charge density on the rank's nodes from the (exchanged) deposit: the
        node charge sum_s q_s w_s dep_s / S over the cell (half the cell at a wall)."""
        out = []
        for n, j in enumerate(range(self.lo, self.hi + 1)):
            q = sum((Fraction(c) * int(dep[s, n]) for s, c in enumerate(qw)), Fraction(0)) / S
            vol = self.dx / 2 if j in (0, self.N) else self.dx
            out.append(q / vol)
        return out

    def _gather(self, obj):
        if self.world == 1:
            return [obj]
        import torch.distributed as dist
        out = [None] * self.world
        dist.all_gather_object(out, obj)
        return out

    def field(self, rho: List[Fraction]) -> np.ndarray:
        """E on the nodes lo..hi (Dirichlet walls), the exact solution rounded once."""
        if self.periodic:
            raise ValueError("a periodic instance has no grounded-wall Poisson solve")
        N, lo, hi = self.N, self.lo, self.hi
        r_at = lambda k: rho[k - lo]  # noqa: E731
        own_lo = lo + 1 if self.rank > 0 else 1   # interior nodes this rank sums
        own_hi = min(hi, N - 1)
        T = sum((k * r_at(k) for k in range(own_lo, own_hi + 1)), Fraction(0))
        U = sum(((N - k) * r_at(k) for k in range(own_lo, own_hi + 1)), Fraction(0))
        tot = self._gather((T, U))
        L = sum((t for t, _ in tot[:self.rank]), Fraction(0))      # L_{own_lo - 1}
        R_after = sum((u for _, u in tot[self.rank + 1:]), Fraction(0))  # R_{own_hi}
        # L_i and R_i on the rank's nodes
        Ls, Rs = {}, {}
        acc = L
        for i in range(lo, hi + 1):
            if own_lo <= i <= own_hi:
                acc += i * r_at(i)
            Ls[i] = acc
        acc = R_after
        for i in range(hi, lo - 1, -1):
            Rs[i] = acc
            if own_lo <= i <= own_hi:
                acc += (N - i) * r_at(i)
        h2 = self.dx * self.dx / self.eps0
        phi = {i: h2 * (Fraction(N - i, N) * Ls[i] + Fraction(i, N) * Rs[i])
               for i in range(lo, hi + 1)}
        # the potentials one node outside the edges, from the neighbours
        edges = self._gather((phi.get(lo + 1), phi.get(hi - 1)))
        if self.rank > 0:
            phi[lo - 1] = edges[self.rank - 1][1]
        if self.rank < self.world - 1:
            phi[hi + 1] = edges[self.rank + 1][0]
        E = np.zeros(hi - lo + 1)
        half = self.dx / (2 * self.eps0)
        for i in range(lo, hi + 1):
            if i == 0:
                e = -(phi[1] - phi[0]) / self.dx - r_at(0) * half
            elif i == N:
                e = -(phi[N] - phi[N - 1]) / self.dx + r_at(N) * half
            else:
                e = (phi[i - 1] - phi[i + 1]) / (2 * self.dx)
            E[i - lo] = float(e)  # rounded once
        return E

    # -- 3. the particles that crossed an edge ---------------------------------------
    _FLOATS = ("off", "vx", "vy", "vz")
    _INTS = ("cell", "id", "state")

    def migrate(self, parts: Dict[str, np.ndarray]) -> Dict[str, np.ndarray]:
        """parts: one species' particles of this rank after the step (cell, off, vx,
        vy, vz, id, state).  Those now outside [lo, hi) go to the neighbour (at most one
        subdomain away); returns the kept ones followed by the ones received."""
        cell = np.asarray(parts["cell"])
        if self.periodic:
            # (the particle step wraps cells into [0, N)): each goes to its owner, which
            # must be this rank or a neighbour on the ring
            owner = np.searchsorted(self.cuts, cell, side="right") - 1
            away = owner != self.rank
            if away.any() and not np.isin(owner[away], self._ring()).all():
                raise ValueError("particle crossed more than one subdomain")
            keep = ~away
            sends = [(nb, owner == nb) for nb in self._ring()]
        else:
            left, right = cell < self.lo, cell >= self.hi
            if (self.rank == 0 and left.any()) or (self.rank == self.world - 1 and right.any()):
                raise ValueError("particle outside the instance")
            if left.any() and self.rank > 0 and cell[left].min() < self.cuts[self.rank - 1]:
                raise ValueError("particle crossed more than one subdomain")
            if right.any() and self.rank < self.world - 1 and cell[right].max() >= self.cuts[self.rank + 2]:
                raise ValueError("particle crossed more than one subdomain")
            keep = ~(left | right)
            sends = [(nb, m) for nb, m in ((self.rank - 1, left), (self.rank + 1, right))
                     if 0 <= nb < self.world]
        out = {k: np.asarray(parts[k])[keep] for k in self._FLOATS + self._INTS}
        if self.world == 1:
            return out
        import torch
        import torch.distributed as dist

        def pack(mask):
            f = np.stack([np.asarray(parts[k], dtype=np.float64)[mask] for k in self._FLOATS], 1)
            i = np.stack([np.asarray(parts[k]).astype(np.int64)[mask] for k in self._INTS], 1)
            return torch.from_numpy(np.ascontiguousarray(f.reshape(-1, 4))), \
                torch.from_numpy(np.ascontiguousarray(i.reshape(-1, 3)))

        nbs = sends
        # counts first, then the particles
        ops, counts = [], {}
        for nb, m in nbs:
            counts[nb] = torch.zeros(1, dtype=torch.int64)
            ops.append(dist.isend(torch.tensor([int(m.sum())], dtype=torch.int64), nb))
            ops.append(dist.irecv(counts[nb], nb))
        for op in ops:
            op.wait()
        ops, got = [], []
        for nb, m in nbs:  # (nothing is sent or received for an empty list)
            if m.any():
                f, i = pack(m)
                ops += [dist.isend(f, nb), dist.isend(i, nb)]
            n = int(counts[nb][0])
            if n > 0:
                rf = torch.zeros((n, 4), dtype=torch.float64)
                ri = torch.zeros((n, 3), dtype=torch.int64)
                ops += [dist.irecv(rf, nb), dist.irecv(ri, nb)]
                got.append((rf, ri))
        for op in ops:
            op.wait()
        for rf, ri in got:
            for c, k in enumerate(self._FLOATS):
                out[k] = np.concatenate([out[k], rf[:, c].numpy()])
            for c, k in enumerate(self._INTS):
                out[k] = np.concatenate([out[k], ri[:, c].numpy().astype(out[k].dtype)])
        return out

    # -- 4. the ids of this step's ionization products -------------------------------
    def renumber_births(self, parts: List[Dict[str, np.ndarray]], parents: np.ndarray,
                        base: int, per: int) -> Tuple[List[Dict[str, np.ndarray]], int]:
        """parts: this rank's species after the step (every array kept as it is but the
        ids); parents: the ids of this rank's ionizing parents of the step, ascending,
        whose r-th one's children carry the ids base + per r + c (c = 0 the electron,
        1 the ion; per = 1 with a neutral particle target, whose ion is a converted
        target); base: the instance's first new id of the step, the same on every rank.
        Returns the species with every child renumbered by its parent's rank among all
        ranks' parents, and the instance's next free id."""
        parents = np.asarray(parents, dtype=np.int64)
        allp = np.sort(np.concatenate([np.asarray(p, dtype=np.int64)
                                       for p in self._gather(parents)]))
        if len(allp) and np.any(allp[1:] == allp[:-1]):
            raise ValueError("an ionizing parent on two ranks")
        rank_of = np.searchsorted(allp, parents)  # each local parent's rank among all
        out = []
        for p in parts:
            q = dict(p)
            ids = np.asarray(p["id"]).astype(np.int64)
            new = ids >= base
            if new.any():
                k = ids[new] - base
                r = k // per
                if r.max() >= len(parents):
                    raise ValueError("a new id without its parent")
                ids[new] = base + per * rank_of[r] + k % per
                q["id"] = ids.astype(np.asarray(p["id"]).dtype)
            out.append(q)
        return out, base + per * len(allp)

    # -- 4. neutral particle targets: the halo and the ionizations handed over --------
    def _neighbours(self) -> List[int]:
        if self.periodic:
            return self._ring()
        return [nb for nb in (self.rank - 1, self.rank + 1) if 0 <= nb < self.world]

    def _owner(self, cell: np.ndarray) -> np.ndarray:
        return np.searchsorted(self.cuts, np.asarray(cell), side="right") - 1

    def _swap(self, outgoing: Dict[int, np.ndarray], dtype) -> np.ndarray:
        """Send each neighbour its structured array (counts first, then the bytes) and
        return what the neighbours sent, concatenated."""
        if self.world == 1:
            return np.zeros(0, dtype)
        import torch
        import torch.distributed as dist
        nbs = self._neighbours()
        ops, counts = [], {}
        for nb in nbs:
            counts[nb] = torch.zeros(1, dtype=torch.int64)
            ops.append(dist.isend(torch.tensor([len(outgoing.get(nb, ()))], dtype=torch.int64), nb))
            ops.append(dist.irecv(counts[nb], nb))
        for op in ops:
            op.wait()
        ops, got = [], []
        for nb in nbs:
            a = outgoing.get(nb)
            if a is not None and len(a):
                ops.append(dist.isend(torch.from_numpy(np.ascontiguousarray(a).view(np.uint8)), nb))
            n = int(counts[nb][0])
            if n > 0:
                buf = torch.zeros(n * np.dtype(dtype).itemsize, dtype=torch.uint8)
                ops.append(dist.irecv(buf, nb))
                got.append(buf)
        for op in ops:
            op.wait()
        if not got:
            return np.zeros(0, dtype)
        return np.concatenate([b.numpy().view(dtype) for b in got])

    _PARTICLE = np.dtype([("cell", np.int64), ("off", np.float64), ("vx", np.float64),
                          ("vy", np.float64), ("vz", np.float64), ("id", np.int64),
                          ("state", np.int64)])

    def halo(self, targets: Dict[str, np.ndarray]) -> Dict[str, np.ndarray]:
        """targets: this rank's target particles at the start of the step.  Returns
        copies of the neighbours' targets in the cells next to this rank's edges (for the
        step only: they are neither moved for good nor converted here)."""
        cell = np.asarray(targets["cell"])
        N, lo, hi = self.N, self.lo, self.hi
        out = {}
        for nb in self._neighbours():
            # the neighbour's halo cells on this rank's side: this rank's edge cells
            nlo, nhi = self.cuts[nb], self.cuts[nb + 1]
            edge = []
            if lo == nhi % N if self.periodic else lo == nhi:
                edge.append(lo)
            if hi % N == nlo if self.periodic else hi == nlo:
                edge.append(hi - 1)
            m = np.isin(cell, edge)
            a = np.zeros(int(m.sum()), self._PARTICLE)
            for k in self._PARTICLE.names:
                a[k] = np.asarray(targets[k])[m]
            out[nb] = a
        got = self._swap(out, self._PARTICLE)
        res = {k: got[k] for k in self._PARTICLE.names}
        res["cell"] = res["cell"].astype(np.int32)
        res["id"] = res["id"].astype(np.uint32)
        res["state"] = res["state"].astype(np.uint8)
        return res

    def hand_over_births(self, recs: np.ndarray) -> np.ndarray:
        """recs: the ionizations this rank's particle loop recorded in cells outside its
        own (a structured array with a `cell` field).  Sends each to the rank that owns
        its cell (a neighbour) and returns those recorded elsewhere in this rank's
        cells."""
        owner = self._owner(recs["cell"]) if len(recs) else np.zeros(0, np.int64)
        nbs = self._neighbours()
        if len(recs) and not np.isin(owner, nbs).all():
            raise ValueError("an ionization recorded beyond the neighbouring subdomains")
        return self._swap({nb: recs[owner == nb] for nb in nbs}, recs.dtype)
