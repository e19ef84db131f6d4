"""Pins of the oracle's density smoother (Section 2's "Density Smoother" phase; the
paper names a filter against spurious high frequencies and gives no formula: the
reading is the 1-2-1 binomial filter of the interior node densities, wall nodes kept).

* A sine mode that vanishes at the walls, rho_j = sin(pi k j / N), is an eigenvector:
  the filter multiplies it by cos^2(pi k / (2N)) exactly (the transfer function
  (1 + cos theta) / 2 of the stencil).
* A uniform density (walls included) is unchanged; the wall entries never change.
* Through the field: the potential of the filtered sine mode is the unfiltered one times
  the same factor (the Dirichlet Poisson operator has the same eigenvectors), and an
  oracle run with the smoother on gives exactly Poisson(filter(rho)) of its deposit.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, poisson, smooth
from paper_2404_10270_gb300 import workloads as W


@pytest.mark.parametrize("N,k", [(16, 1), (64, 5), (257, 100), (1000, 999)])
def test_sine_mode_is_attenuated_by_cos_squared(N, k):
    j = np.arange(N + 1)
    # the argument reduced to [0, 2 pi) before the sine, so that the input is the sine
    # mode to within one rounding per entry
    rho = np.sin(math.pi * ((k * j) % (2 * N)) / N)
    rho[0] = rho[N] = 0.0
    got = smooth(rho)
    fac = math.cos(math.pi * k / (2 * N)) ** 2
    np.testing.assert_allclose(got, fac * rho, rtol=0, atol=1.5e-15)


def test_uniform_density_and_walls_unchanged():
    rho = np.full(33, 2.5)
    np.testing.assert_array_equal(smooth(rho), rho)
    r = np.random.default_rng(1).normal(size=41)
    s = smooth(r)
    assert s[0] == r[0] and s[-1] == r[-1]
    # the interior is a local average: never outside the range of its three inputs
    lo = np.minimum(np.minimum(r[:-2], r[1:-1]), r[2:])
    hi = np.maximum(np.maximum(r[:-2], r[1:-1]), r[2:])
    assert np.all(s[1:-1] >= lo - 1e-15) and np.all(s[1:-1] <= hi + 1e-15)


def test_filtered_potential_of_a_sine_mode():
    N, k, dx = 128, 7, 0.5
    j = np.arange(N + 1)
    rho = np.sin(math.pi * ((k * j) % (2 * N)) / N)
    rho[0] = rho[N] = 0.0
    phi0, _ = poisson(rho, dx)
    phi1, _ = poisson(smooth(rho), dx)
    fac = math.cos(math.pi * k / (2 * N)) ** 2
    np.testing.assert_allclose(phi1, fac * phi0, rtol=0, atol=1e-13 * np.abs(phi0).max())


def test_oracle_run_uses_the_filtered_density():
    phys = W.bounded_small(ncells=64, ppc=20, seed=4)
    phys.smooth = 1
    loads = W.initial_load(phys, seed=4)
    o = Oracle(phys)
    o.load_all(loads)
    o.step(3)
    m = o.moments()
    N, S = phys.ncells, len(phys.species)
    dens = m["density"].reshape(S, N + 1)  # number density per node (walls: half cells)
    rho = sum(sp.charge * dens[i] for i, sp in enumerate(phys.species))
    phi, E = poisson(smooth(rho), phys.dx, phys.eps0)
    np.testing.assert_allclose(m["phi"], phi, rtol=0, atol=1e-13 * np.abs(phi).max())
    np.testing.assert_allclose(m["E"], E, rtol=0, atol=1e-13 * np.abs(E).max())
