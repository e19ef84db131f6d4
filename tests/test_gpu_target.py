"""GPU parity of the neutral-particle target (the paper's test case, Section 3 and Table
1): electrons, D+ and D neutrals as particles, periodic, no field solve; electron-neutral
elastic, excitation and ionization against the neutrals, each ionization turning the
smallest-id live neutral of the electron's cell (as of the start of the step) into an
ion.  FP64: particles by id within 1e-12 over 100 steps, live / collision counts and
collision clocks exact, the converted ions with the neutrals' ids; FP32: 1e-5 over 10
steps."""
import numpy as np
import pytest

from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W
from tests.gpu_common import (assert_same_clocks, by_id, particle_errors, requires_gpu,
                              run_gpu, run_oracle)

pytestmark = [pytest.mark.gpu, requires_gpu]


@pytest.mark.parametrize("precision,steps,tol", [(capi.FP64, 100, 1e-12), (capi.FP32, 10, 1e-5)])
def test_paper_case_parity(precision, steps, tol):
    phys = W.ionization_case(ncells=256, ppc=64, nu_el=0.05, nu_exc=0.05, nu_iz=0.05, seed=2)
    loads = W.initial_load(phys, seed=2)
    g, gm = run_gpu(phys, loads, steps, precision, sort_interval=phys.sort_interval)
    o, om = run_oracle(phys, loads, steps)
    np.testing.assert_array_equal(gm["live"], om["live"])
    if precision == capi.FP64:
        np.testing.assert_array_equal(gm["collisions"], om["collisions"])
        assert om["collisions"][2] > 20  # ionizations happened
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < tol and ev < tol, (s, ex, ev)
    assert_same_clocks(g, o)
    for s in range(3):  # the same particles (ids) in every species
        np.testing.assert_array_equal(np.sort(g[s]["id"]), np.sort(o[s]["id"]))


def test_depletion_to_exhaustion_fp64():
    """Strong ionization in a small system: several ionizations per cell and step, cells
    running out of neutrals; ids, counts and every particle as the oracle."""
    phys = W.ionization_case(ncells=16, ppc=40, nu_el=0.0, nu_exc=0.0, nu_iz=1.0, seed=6,
                             sort_interval=5)
    phys.processes[2].threshold = 0.0
    # a cell with fewer neutrals than ionizations still gains the electrons
    phys.species[0].capacity_factor = 4.0
    phys.species[1].capacity_factor = 3.0
    loads = W.initial_load(phys, seed=6)
    g, gm = run_gpu(phys, loads, 60, capi.FP64, sort_interval=5)
    o, om = run_oracle(phys, loads, 60)
    np.testing.assert_array_equal(gm["live"], om["live"])
    np.testing.assert_array_equal(gm["collisions"], om["collisions"])
    assert om["live"][2] < 0.5 * 16 * 40  # most neutrals are gone
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < 1e-12 and ev < 1e-12, (s, ex, ev)
    for s in range(3):
        np.testing.assert_array_equal(np.sort(g[s]["id"]), np.sort(o[s]["id"]))


def test_target_instances_in_a_batch_equal_alone():
    """Two Table-1 instances of different sizes and seeds, plus a plain bounded plasma,
    in one handle: each target instance gives exactly what it gives alone (every count,
    every particle bit for bit)."""
    from tests.gpu_common import ensure_built
    ensure_built()
    a = W.ionization_case(ncells=128, ppc=48, nu_iz=0.1, nu_exc=0.05, nu_el=0.05, seed=3)
    b = W.ionization_case(ncells=96, ppc=64, nu_iz=0.2, nu_exc=0.0, nu_el=0.1, seed=4)
    phys = [a, b]
    loads = [W.initial_load(p, seed=p.seed) for p in phys]
    steps = 45
    sim = capi.Sim(phys, precision=capi.FP64, sort_interval=20)
    for i, ld in enumerate(loads):
        sim.load_all(ld, inst=i)
    sim.step(steps)
    batch = [([by_id(sim.particles(i, s)) for s in range(3)], sim.moments(i)) for i in range(2)]
    sim.close()
    for i, p in enumerate(phys):
        s1 = capi.Sim(p, precision=capi.FP64, sort_interval=20)
        s1.load_all(loads[i])
        s1.step(steps)
        alone = [by_id(s1.particles(0, s)) for s in range(3)]
        m = s1.moments(0)
        s1.close()
        np.testing.assert_array_equal(batch[i][1]["live"], m["live"])
        np.testing.assert_array_equal(batch[i][1]["collisions"], m["collisions"])
        for x, y in zip(alone, batch[i][0]):
            for k in x:
                np.testing.assert_array_equal(x[k], y[k])
