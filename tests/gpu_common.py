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
