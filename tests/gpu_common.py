"""Shared pieces of the GPU tests: running both sides on the same seeded input and
comparing particles matched by id (the relative errors of the accuracy contract:
|dx|/L for positions and |dv| / max(|v_ref|, v_th,s) for velocities)."""
import math

import numpy as np
import pytest

from paper_2404_10270_gb300 import capi


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


requires_gpu = pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")


def ensure_built():
    from paper_2404_10270_gb300 import build
    build.build()


def run_gpu(phys, loads, steps, precision, sort_interval=0, block=0):
    ensure_built()
    sim = capi.Sim(phys, precision=precision, sort_interval=sort_interval, block=block)
    sim.load_all(loads)
    sim.step(steps)
    out = [sim.particles(0, s) for s in range(len(phys.species))]
    m = sim.moments(0)
    sim.close()
    return out, m


def run_oracle(phys, loads, steps):
    from oracle.oracle import Oracle
    o = Oracle(phys)
    o.load_all(loads)
    o.step(steps)
    return [o.particles(s) for s in range(len(phys.species))], o.moments()


def by_id(p):
    order = np.argsort(p["id"], kind="stable")
    return {k: v[order] for k, v in p.items()}


def assert_same_clocks(gpu_parts, ora_parts):
    """The collision clocks are integer state driven by id-keyed draws: identical."""
    for g, o in zip(gpu_parts, ora_parts):
        g, o = by_id(g), by_id(o)
        np.testing.assert_array_equal(g["id"], o["id"])
        np.testing.assert_array_equal(g["state"], o["state"])


def particle_errors(phys, gpu_parts, ora_parts):
    """Max relative position and velocity error per species (ids must match)."""
    L = phys.length
    res = []
    for s, (g, o) in enumerate(zip(gpu_parts, ora_parts)):
        g, o = by_id(g), by_id(o)
        np.testing.assert_array_equal(g["id"], o["id"])
        if len(g["id"]) == 0:
            res.append((0.0, 0.0))
            continue
        xg = (g["cell"] + g["off"]) * phys.dx
        xo = (o["cell"] + o["off"]) * phys.dx
        ex = np.abs(xg - xo).max() / L
        vth = math.sqrt(max(phys.species[s].temperature, 1e-30) / phys.species[s].mass)
        dv = np.sqrt((g["vx"] - o["vx"]) ** 2 + (g["vy"] - o["vy"]) ** 2 + (g["vz"] - o["vz"]) ** 2)
        vref = np.sqrt(o["vx"] ** 2 + o["vy"] ** 2 + o["vz"] ** 2)
        ev = (dv / np.maximum(vref, vth)).max()
        res.append((ex, ev))
    return res


def oracle_with_ionization_record(phys, loads, steps):
    """Oracle run that also returns the ids of every ionization participant: products
    (ids beyond the load) and electrons that lost more than the threshold energy in one
    step (the parents)."""
    from oracle.oracle import Oracle
    o = Oracle(phys)
    o.load_all(loads)
    n0 = sum(len(x) for x in loads)
    eiz = max([q.threshold for q in phys.processes if q.kind == 2] + [0.0])
    m_e = phys.species[0].mass
    prev = by_id(o.particles(0))
    parents = set()
    for _ in range(steps):
        o.step(1)
        cur = by_id(o.particles(0))
        old = cur["id"] < n0
        idx = np.searchsorted(prev["id"], cur["id"][old])
        e0 = 0.5 * m_e * (prev["vx"][idx] ** 2 + prev["vy"][idx] ** 2 + prev["vz"][idx] ** 2)
        e1 = 0.5 * m_e * (cur["vx"][old] ** 2 + cur["vy"][old] ** 2 + cur["vz"][old] ** 2)
        parents.update(cur["id"][old][e0 - e1 > eiz * (1 - 1e-6)].tolist())
        prev = cur
    return [o.particles(s) for s in range(len(phys.species))], o.moments(), n0, parents


def participant_mask(o, n0, parents):
    """Particles of an oracle species dict (by id) that took part in an ionization."""
    ids = by_id(o)["id"]
    return (ids >= n0) | np.isin(ids, np.fromiter(parents, np.int64, len(parents)))


def velocity_errors(phys, g, o, s):
    """Per-particle relative velocity errors |dv| / max(|v_ref|, v_th) (matched by id)."""
    g, o = by_id(g), by_id(o)
    np.testing.assert_array_equal(g["id"], o["id"])
    vth = math.sqrt(max(phys.species[s].temperature, 1e-30) / phys.species[s].mass)
    dv = np.sqrt((g["vx"] - o["vx"]) ** 2 + (g["vy"] - o["vy"]) ** 2 + (g["vz"] - o["vz"]) ** 2)
    vref = np.sqrt(o["vx"] ** 2 + o["vy"] ** 2 + o["vz"] ** 2)
    return dv / np.maximum(vref, vth)
