"""Long-run statistics of the FP32 form against the FP64 oracle: over 1000 steps of the
small bounded plasma (about 20 plasma periods, walls absorbing, collisions on), the
time-averaged density and potential profiles and the wall particle fluxes of the two
agree within 1 % or 3 ensemble standard errors (ensemble over seeds)."""
import numpy as np
import pytest

from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W
from tests.gpu_common import ensure_built, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]

STEPS, SAMPLE_FROM, EVERY, BINS = 1000, 500, 50, 16


def _observe(step_fn, moments_fn, ncells):
    dens, phi = [], []
    done = 0
    while done < STEPS:
        n = EVERY if done >= SAMPLE_FROM else SAMPLE_FROM
        step_fn(n)
        done += n
        if done > SAMPLE_FROM - 1:
            m = moments_fn()
            # coarse-grain interior nodes into bins
            w = (ncells - 1) // BINS * BINS
            d = m["density"][:, 1:1 + w].reshape(2, BINS, -1).mean(axis=2)
            p = m["phi"][1:1 + w].reshape(BINS, -1).mean(axis=1)
            dens.append(d)
            phi.append(p)
    m = moments_fn()
    return np.mean(dens, axis=0), np.mean(phi, axis=0), m["wall_count"].astype(float)


def _runs(seed):
    from oracle.oracle import Oracle
    phys = W.bounded_small(ncells=256, ppc=100, seed=seed)
    loads = W.initial_load(phys, seed=seed)
    sim = capi.Sim(phys, precision=capi.FP32, sort_interval=20)
    sim.load_all(loads)
    g = _observe(sim.step, lambda: sim.moments(0), phys.ncells)
    sim.close()
    o = Oracle(phys)
    o.load_all(loads)
    r = _observe(o.step, o.moments, phys.ncells)
    return g, r


def test_long_run_profiles_and_fluxes_agree():
    ensure_built()
    seeds = range(1, 7)
    res = [_runs(s) for s in seeds]
    for q in range(3):  # density, potential, wall counts
        g = np.array([r[0][q] for r in res])
        o = np.array([r[1][q] for r in res])
        mg, mo = g.mean(0), o.mean(0)
        se = np.sqrt(g.var(0, ddof=1) / len(g) + o.var(0, ddof=1) / len(o))
        ok = (np.abs(mg - mo) <= 0.01 * np.abs(mo)) | (np.abs(mg - mo) <= 3 * se)
        assert ok.all(), (q, mg, mo, se)
