"""Pins of the oracle's density (cloud-in-cell) and field (Poisson) phases.

* Poisson: against a dense LAPACK solve of the same tridiagonal system, against the
  exact rational solution (the discrete Green's function of the three-point Dirichlet
  Laplacian, G(j, k) = min(j, k) (N - max(j, k)) / N, summed in Python integers) up
  to 65,536 cells, against the closed form phi = rho x (L - x) / (2 eps0) for uniform
  charge (exact for the three-point Laplacian), and against Gauss's law over the
  whole gap, E_N - E_0 = (integral of rho) / eps0.
* Deposit: linear weighting preserves total charge and the first moment (centre of
  charge) of every particle exactly; a uniform lattice deposits a uniform density.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, poisson
from paper_2404_10270_gb300 import workloads as W


@pytest.mark.parametrize("N", [1, 2, 3, 7, 64, 257])
def test_poisson_matches_dense_solve(N):
    rng = np.random.default_rng(N)
    dx, eps0 = 0.37, 1.3
    rho = rng.normal(size=N + 1)
    phi, E = poisson(rho, dx, eps0)
    assert phi[0] == 0.0 and phi[N] == 0.0
    if N >= 2:
        M = N - 1
        A = 2 * np.eye(M) - np.eye(M, k=1) - np.eye(M, k=-1)
        ref = np.linalg.solve(A, dx * dx * rho[1:N] / eps0)
        np.testing.assert_allclose(phi[1:N], ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())


def _exact_solution(rho, dx, eps0):
    """phi and E of the grounded three-point problem as exact rationals, rounded to
    FP64 once.  phi_j = (dx^2/eps0) sum_k G(j, k) rho_k with the discrete Green's
    function G(j, k) = min(j, k) (N - max(j, k)) / N, i.e.
    phi_j = h2 [(N - j) sum_{k<=j} k rho_k + j sum_{k>j} (N - k) rho_k] / N,
    with every rho_k an exact dyadic rational (scaled to integers by a common 2^K)."""
    from fractions import Fraction
    N = len(rho) - 1
    fr = [Fraction(float(r)) for r in rho]
    D = max(f.denominator for f in fr)
    R = [f.numerator * (D // f.denominator) for f in fr]  # rho_k = R_k / D
    S1 = [0] * (N + 1)   # sum_{1<=k<=j} k R_k
    for j in range(1, N):
        S1[j] = S1[j - 1] + j * R[j]
    S2 = [0] * (N + 1)   # sum_{j<k<=N-1} (N - k) R_k
    for j in range(N - 2, -1, -1):
        S2[j] = S2[j + 1] + (N - (j + 1)) * R[j + 1]
    h2 = Fraction(dx) ** 2 / Fraction(eps0)
    scale = h2 / (N * D)
    q = [scale * ((N - j) * S1[j] + j * S2[j]) for j in range(N + 1)]
    q[0] = q[N] = Fraction(0)
    fdx = Fraction(dx)
    half = fdx / (2 * Fraction(eps0))
    E = [Fraction(0)] * (N + 1)
    for j in range(1, N):
        E[j] = (q[j - 1] - q[j + 1]) / (2 * fdx)
    E[0] = -(q[1] - q[0]) / fdx - fr[0] * half
    E[N] = -(q[N] - q[N - 1]) / fdx + fr[N] * half
    return np.array([float(v) for v in q]), np.array([float(v) for v in E])


@pytest.mark.parametrize("N", [2, 257, 8192, 65536])
def test_poisson_is_the_rounded_exact_solution(N):
    """The oracle's Thomas solve (binary128, one final rounding) against the exact
    rational solution: every phi and E within one unit in the last place (the exact
    value rounded to FP64 is within half a unit; the binary128 recurrences add ~1e-25
    relative).  An FP64 Thomas solve misses this by ~1e-11 at N = 8192."""
    rng = np.random.default_rng(N + 11)
    dx, eps0 = 0.5, 1.0
    # a plasma-like charge: two nearly cancelling species densities
    rho = rng.normal(1.0, 0.1, N + 1) - rng.normal(1.0, 0.1, N + 1)
    phi, E = poisson(rho, dx, eps0)
    ephi, eE = _exact_solution(rho, dx, eps0)
    for got, want in ((phi, ephi), (E, eE)):
        floor = 1e-22 * np.abs(want).max()
        bad = np.abs(got - want) > np.spacing(np.abs(want)) + floor
        assert not bad.any(), (np.nonzero(bad)[0][:5], got[bad][:3], want[bad][:3])


def test_poisson_against_lapack_banded_at_8192():
    """LAPACK's banded LU (gbsv) on the same system: its own forward error is bounded
    by cond(A) eps ~ (4 N^2 / pi^2) eps of the solution's scale, which bounds the gap."""
    from scipy.linalg import solve_banded
    N = 8192
    rng = np.random.default_rng(8192)
    dx, eps0 = 0.5, 1.0
    rho = rng.normal(size=N + 1)
    phi, _ = poisson(rho, dx, eps0)
    M = N - 1
    ab = np.zeros((3, M))
    ab[0, 1:] = -1.0
    ab[1, :] = 2.0
    ab[2, :-1] = -1.0
    ref = solve_banded((1, 1), ab, dx * dx * rho[1:N] / eps0)
    cond = 4.0 * N * N / np.pi ** 2
    tol = 8 * cond * np.finfo(float).eps * np.abs(ref).max()
    assert np.abs(phi[1:N] - ref).max() < tol


@pytest.mark.parametrize("N", [4, 100, 1000, 65536])
def test_poisson_uniform_charge_closed_form(N):
    dx, eps0, rho0 = 0.5, 1.0, 0.7
    L = N * dx
    rho = np.full(N + 1, rho0)  # wall entries: half-cell densities, also rho0
    phi, E = poisson(rho, dx, eps0)
    x = np.arange(N + 1) * dx
    exact = rho0 * x * (L - x) / (2 * eps0)
    # the oracle's solution is the exact one rounded once; the closed form evaluated
    # in FP64 adds a few roundings of its own
    tol = 4 * np.finfo(float).eps
    np.testing.assert_allclose(phi, exact, rtol=0, atol=tol * np.abs(exact).max())
    # E = -dphi/dx = rho0 (x - L/2) / eps0, also at both walls
    np.testing.assert_allclose(E, rho0 * (x - L / 2) / eps0, rtol=0,
                               atol=tol * rho0 * L / eps0)


def test_poisson_gauss_law_over_the_gap():
    rng = np.random.default_rng(2)
    N, dx, eps0 = 300, 0.25, 2.0
    rho = rng.normal(size=N + 1)
    phi, E = poisson(rho, dx, eps0)
    total = rho[1:N].sum() * dx + (rho[0] + rho[N]) * dx / 2
    assert abs((E[N] - E[0]) - total / eps0) < 1e-10


def _one_species_field_off(ncells, ppc=0):
    sp = [W.Species("e", -1.0, 1.0, 0.25, 1.0, ppc)]
    return W.Physics(ncells=ncells, dx=0.5, dt=0.05, species=sp, processes=[],
                     field=W.FIELD_NONE)


@pytest.mark.parametrize("npart", [1, 2, 5, 8])
def test_deposit_conserves_charge_and_centre_of_charge(npart):
    """Up to eight particles at arbitrary positions: the CIC node weights sum to one
    per particle and place the centre of charge exactly at the particle."""
    rng = np.random.default_rng(npart)
    phys = _one_species_field_off(12)
    cell = rng.integers(0, 12, npart).astype(np.int32)
    off = rng.random(npart)
    z = np.zeros(npart)
    ld = W.Load(cell, off, z.copy(), z.copy(), z.copy(), np.arange(npart, dtype=np.uint32))
    o = Oracle(phys)
    o.load(0, ld)
    d = o.moments()["density"][0]
    N, dx, w = 12, phys.dx, 0.25
    vol = np.full(N + 1, dx)
    vol[0] = vol[N] = dx / 2  # wall nodes report half-cell densities
    count = d * vol / w  # CIC weight sum per node
    assert abs(count.sum() - npart) < 1e-13
    nodes = np.arange(N + 1) * dx
    x = (cell + off) * dx
    assert abs((count * nodes).sum() - x.sum()) < 1e-12
    # each particle touches only the two nodes of its cell
    touched = np.nonzero(count > 0)[0]
    allowed = set(cell.tolist()) | set((cell + 1).tolist())
    assert set(touched.tolist()) <= allowed


def test_uniform_lattice_deposits_uniform_density():
    ppc, N = 8, 16
    phys = _one_species_field_off(N, ppc)
    n = N * ppc
    xc = (np.arange(n) + 0.5) / ppc  # positions in cell units
    cell = np.floor(xc).astype(np.int32)
    off = xc - cell
    z = np.zeros(n)
    o = Oracle(phys)
    o.load(0, W.Load(cell, off, z.copy(), z.copy(), z.copy(), np.arange(n, dtype=np.uint32)))
    d = o.moments()["density"][0]
    expect = ppc * 0.25 / phys.dx
    np.testing.assert_allclose(d[1:N], expect, rtol=1e-14)
    # the half cells next to the walls hold half as many particles per volume
    # dx/2 ... which makes the wall-node density the same uniform value
    np.testing.assert_allclose(d[[0, N]], expect, rtol=1e-14)


def test_field_of_a_charge_sheet():
    """A single sheet of charge Q at x_s between grounded plates: the exact
    (continuum) potential is piecewise linear with phi(x_s) = Q x_s (L - x_s) / (eps0 L);
    with the charge on a node the discrete solution is exact."""
    N, dx = 40, 0.5
    L = N * dx
    sp = [W.Species("i", 1.0, 1e12, 0.3, 0.0, 0)]
    phys = W.Physics(ncells=N, dx=dx, dt=0.05, species=sp, processes=[], m_neutral=1e12)
    o = Oracle(phys)
    o.load(0, W.Load(np.array([13], np.int32), np.array([0.0]), np.zeros(1), np.zeros(1),
                     np.zeros(1), np.zeros(1, np.uint32)))
    m = o.moments()
    x = np.arange(N + 1) * dx
    xs, Q = 13 * dx, 0.3
    phi = np.where(x <= xs, Q * x * (L - xs) / L, Q * xs * (L - x) / L)
    np.testing.assert_allclose(m["phi"], phi, rtol=1e-12, atol=1e-13)
    # field: -Q (L - xs)/L on the left of the sheet, Q xs / L on the right (also at walls)
    left = x < xs
    right = x > xs
    np.testing.assert_allclose(m["E"][left], -Q * (L - xs) / L, rtol=1e-12)
    np.testing.assert_allclose(m["E"][right], Q * xs / L, rtol=1e-12)
