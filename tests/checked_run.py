"""Runs a set of small workloads through the library that $BITPIC_LIB selects (the
bounds-checked build, or the normal one) and saves every particle (by id) and the
moments to an .npz file; used by test_gpu_checked.py in a subprocess per library.

Usage: python -m tests.checked_run OUT.npz
"""
import sys

import numpy as np

from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W


def by_id(p):
    order = np.argsort(p["id"], kind="stable")
    return {k: v[order] for k, v in p.items()}


def cases():
    mag = W.magnetized_source(ncells=64, ppc=40, seed=2, nu=0.2, capacity_factor=3.0)
    sub = W.bounded_small(ncells=96, ppc=40, seed=5, ion_nstep=4)
    y2 = W.bounded_small(ncells=128, ppc=30, seed=3)
    for s in y2.species:
        s.sn2d = 1
    tgt = W.ionization_case(ncells=300, ppc=40, seed=4, nu_iz=0.05)
    return [("bounded_small", W.bounded_small(), capi.FP64, 20, 130),
            ("bounded_small_f32", W.bounded_small(), capi.FP32, 20, 130),
            ("magnetized", mag, capi.FP64, 10, 60),
            ("subcycled", sub, capi.FP32, 20, 60),
            ("drift_y", y2, capi.FP32, 5, 30),
            ("separate_sort", W.bounded_small(ncells=64, ppc=30, seed=6), capi.FP64, 1, 20),
            ("targets", tgt, capi.FP32, tgt.sort_interval, 60)]


def main(out):
    res = {"probe": capi.lib().pic_bounds_probe(None)}
    for name, phys, prec, K, steps in cases():
        sim = capi.Sim(phys, precision=prec, sort_interval=K)
        loads = W.initial_load(phys, seed=phys.seed)
        sim.load_all(loads)
        sim.step(steps)
        sim.sync()  # a latched refusal raises here
        for s in range(len(phys.species)):
            p = by_id(sim.particles(0, s))
            for k, v in p.items():
                res["%s/%d/%s" % (name, s, k)] = v
        m = sim.moments(0)
        for k in ("live", "wall_count", "collisions", "density", "E"):
            res["%s/%s" % (name, k)] = m[k]
        sim.close()
    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1])
