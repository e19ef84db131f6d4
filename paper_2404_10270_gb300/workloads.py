"""Seeded synthetic workloads: physics parameters and initial particle loads.

This module holds the workload definitions shared by the tests, the benchmark and
the smoke check.  It draws the initial particles (exactly ``ppc`` particles per
cell per species, uniform in-cell offsets, Maxwellian velocities) from numpy's own
seeded generator and contains none of the time step's arithmetic, so the GPU
library and the CPU oracle can both be fed the same inputs.

All quantities are in normalised units: eps0 = e = m_e = n0 = lambda_D =
omega_pe = 1 (electron thermal speed and temperature 1).  The macro-particle weight
is w = n0 * dx / ppc, so that each species starts at density n0.

Named workloads (bounded 1D plasma between grounded absorbing walls unless noted):
  * ``bounded_small``   256 cells, dx 0.5, dt 0.05, e + i (m_i/m_e 100), 100 ppc each,
                        B = 0, e-neutral elastic and i-neutral charge exchange at
                        0.01 omega_pe, seed 1.
  * ``magnetized_source`` 4096 cells, 200 ppc, m_i/m_e 1836, |B| = 2 at 80 degrees to the
                        wall normal, volume source replacing wall losses, elastic +
                        ionization (threshold 0.68 T_e) + charge exchange at 0.01.
  * ``bounded_large``   65,536 cells, 1,500 ppc per species (196,608,000 particles),
                        physics of ``bounded_small``, sort every 20 steps.
  * ``ensemble``        512 independent ``magnetized_source`` instances: cells
                        log-uniform in [256, 8192], ppc uniform in [50, 400],
                        m_i/m_e in {100, 1836}, B angle uniform in [0, 89] degrees,
                        Philox seeds 1..512; instance parameters drawn with key 0.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

# enums, identical in meaning on both sides of the library boundary
BC_ABSORB, BC_PERIODIC, BC_SOURCE = 0, 1, 2
FIELD_POISSON, FIELD_NONE, FIELD_EXTERNAL = 0, 1, 2
PROC_ELASTIC, PROC_CX, PROC_IONIZE, PROC_EXCITE = 0, 1, 2, 3


@dataclasses.dataclass
class Species:
    name: str
    charge: float
    mass: float
    weight: float
    temperature: float
    ppc: int = 0                 # particles per cell at load time
    capacity_factor: float = 1.0  # slots reserved per loaded particle (creation slack)
    nstep: int = 1                # subcycling: advanced with nstep*dt on steps n, (n+1) % nstep == 0
    sn2d: int = 0                 # 1: also drifts in y (yp += nstep*vy, yp in cell units)


@dataclasses.dataclass
class Process:
    kind: int
    species: int
    nu: float
    threshold: float = 0.0
    product: int = -1


@dataclasses.dataclass
class Physics:
    ncells: int
    dx: float
    dt: float
    species: List[Species]
    processes: List[Process]
    eps0: float = 1.0
    bc: int = BC_ABSORB
    field: int = FIELD_POISSON
    E_ext: float = 0.0
    B: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    T_neutral: float = 0.05
    m_neutral: float = 100.0
    seed: int = 1
    sort_interval: int = 20
    smooth: int = 0           # 1: density smoother (1-2-1 filter) before the field solve
    target: int = 0           # k+1: species k (neutral particles) is the collision target
    nref: int = 0             # target particles per cell at which the processes' nu apply

    @property
    def length(self) -> float:
        return self.ncells * self.dx

    def n_particles(self) -> int:
        return sum(s.ppc for s in self.species) * self.ncells


def bounded_small(ncells: int = 256, ppc: int = 100, seed: int = 1,
                  m_i: float = 100.0, nu: float = 0.01, dx: float = 0.5,
                  dt: float = 0.05, ion_nstep: int = 1) -> Physics:
    """Grounded absorbing walls, electrons + ions, elastic e-n and i-n charge exchange.
    ion_nstep > 1 subcycles the ions (advanced every ion_nstep steps)."""
    w = dx / ppc
    sp = [Species("e", -1.0, 1.0, w, 1.0, ppc),
          Species("i", 1.0, m_i, w, 1.0, ppc, nstep=ion_nstep)]
    pr = [Process(PROC_ELASTIC, 0, nu), Process(PROC_CX, 1, nu)]
    return Physics(ncells=ncells, dx=dx, dt=dt, species=sp, processes=pr,
                   T_neutral=1.0 / 20.0, m_neutral=m_i, seed=seed)


def magnetized_source(ncells: int = 4096, ppc: int = 200, seed: int = 1,
                      m_i: float = 1836.0, angle_deg: float = 80.0, B: float = 2.0,
                      nu: float = 0.01, capacity_factor: float = 1.5,
                      ion_nstep: int = 1) -> Physics:
    """Oblique magnetic field, volume source, elastic + ionization + charge exchange."""
    dx, dt = 0.5, 0.05
    w = dx / ppc
    th = math.radians(angle_deg)
    sp = [Species("e", -1.0, 1.0, w, 1.0, ppc, capacity_factor),
          Species("i", 1.0, m_i, w, 1.0, ppc, capacity_factor, nstep=ion_nstep)]
    pr = [Process(PROC_ELASTIC, 0, nu), Process(PROC_IONIZE, 0, nu, 13.6 / 20.0, 1),
          Process(PROC_CX, 1, nu)]
    return Physics(ncells=ncells, dx=dx, dt=dt, species=sp, processes=pr, bc=BC_SOURCE,
                   B=(B * math.cos(th), B * math.sin(th), 0.0), T_neutral=1.0 / 20.0,
                   m_neutral=m_i, seed=seed)


def ionization_case(ncells: int = 100000, ppc: int = 100, seed: int = 1,
                    nu_el: float = 0.01, nu_exc: float = 0.002, nu_iz: float = 0.002,
                    m_d: float = 3670.0, sort_interval: int = 20,
                    dx: float = 0.5, dt: float = 0.05) -> Physics:
    """The paper's test case (Section 3, Table 1) in normalized units: a periodic
    unbounded plasma of electrons, D+ ions and D neutrals, all particles, uniform at
    equal densities (ppc each); T_e = T_i = 1 (20 eV), T_n = 0.05 (1 eV); no field solve
    and no smoother; electron-neutral elastic, excitation (10.2 eV) and ionization
    (13.6 eV) against the neutral particles, which the ionizations deplete.  The
    neutrals move once per sort cycle (nstep = sort_interval)."""
    w = dx / ppc
    sp = [Species("e", -1.0, 1.0, w, 1.0, ppc, 2.0),
          Species("D+", 1.0, m_d, w, 1.0, ppc, 2.0),
          Species("D", 0.0, m_d, w, 0.05, ppc, 1.0, nstep=sort_interval)]
    pr = [Process(PROC_ELASTIC, 0, nu_el), Process(PROC_EXCITE, 0, nu_exc, 10.2 / 20.0),
          Process(PROC_IONIZE, 0, nu_iz, 13.6 / 20.0, 1)]
    return Physics(ncells=ncells, dx=dx, dt=dt, species=sp, processes=pr, bc=BC_PERIODIC,
                   field=FIELD_NONE, T_neutral=0.05, m_neutral=m_d, seed=seed,
                   sort_interval=sort_interval, target=3, nref=ppc)


def bounded_large(ncells: int = 65536, ppc: int = 1500, seed: int = 1) -> Physics:
    """The small bounded plasma's physics on 65,536 cells at 1,500 particles/cell."""
    return bounded_small(ncells=ncells, ppc=ppc, seed=seed)


def ensemble(n_instances: int = 512, key: int = 0, capacity_factor: float = 1.5,
             scale: float = 1.0) -> List[Physics]:
    """Batched ensemble of uneven bounded plasmas (magnetized, volume source,
    elastic + ionization + charge exchange).  ``scale`` multiplies every instance's
    particles per cell (scale < 1 gives a smaller ensemble of the same shape)."""
    rng = np.random.Generator(np.random.Philox(key=key))
    u = rng.random((n_instances, 4))
    out = []
    for i in range(n_instances):
        cells = int(np.rint(256.0 * 32.0 ** u[i, 0]))
        ppc = max(1, int(round((50 + int(np.floor(351.0 * u[i, 1]))) * scale)))
        m_i = 100.0 if u[i, 2] < 0.5 else 1836.0
        angle = 89.0 * u[i, 3]
        out.append(magnetized_source(ncells=cells, ppc=ppc, seed=i + 1, m_i=m_i,
                                     angle_deg=angle, capacity_factor=capacity_factor))
    return out


@dataclasses.dataclass
class Load:
    cell: np.ndarray  # int32
    off: np.ndarray   # float64 in [0, 1)
    vx: np.ndarray    # float64, physical units
    vy: np.ndarray
    vz: np.ndarray
    id: np.ndarray    # uint32
    # collision clock per particle (bits 0-6 steps to skip, bit 7 candidate pending);
    # None = all zero, which is how a fresh load starts
    state: Optional[np.ndarray] = None
    # y coordinate (cell units) of a species that drifts in y; None = 0
    yp: Optional[np.ndarray] = None

    def __len__(self) -> int:
        return len(self.cell)

    def take(self, idx) -> "Load":
        return Load(self.cell[idx], self.off[idx], self.vx[idx], self.vy[idx],
                    self.vz[idx], self.id[idx],
                    None if self.state is None else self.state[idx],
                    None if self.yp is None else self.yp[idx])


def initial_load(phys: Physics, seed: int = 1, cells=None) -> List[Load]:
    """Exactly ppc particles per cell per species, offsets uniform in [0, 1),
    velocities Maxwellian at the species temperature; ids species-major from 0.

    ``cells`` (optional, an index array) restricts the load to those cells, which
    gives a bounded sample of a large workload with the same per-cell statistics.
    """
    rng = np.random.Generator(np.random.Philox(key=seed))
    loads = []
    next_id = 0
    cell_list = np.arange(phys.ncells, dtype=np.int32) if cells is None else \
        np.asarray(cells, dtype=np.int32)
    for s in phys.species:
        n = s.ppc * len(cell_list)
        cell = np.repeat(cell_list, s.ppc).astype(np.int32)
        off = rng.random(n)
        vth = math.sqrt(s.temperature / s.mass)
        v = rng.standard_normal((3, n)) * vth
        ids = np.arange(next_id, next_id + n, dtype=np.uint64)
        if next_id + n >= 2 ** 32:
            raise ValueError("more than 2^32 particles in one instance")
        loads.append(Load(cell, off, v[0].copy(), v[1].copy(), v[2].copy(),
                          ids.astype(np.uint32)))
        next_id += n
    return loads


def cold_wave(ncells: int = 256, ppc: int = 16, amplitude: float = 1e-3, mode: int = 2,
              dx: float = 0.5, dt: float = 0.05) -> Tuple[Physics, List[Load]]:
    """Cold electrons on an evenly spaced lattice displaced by amplitude*sin(k x0),
    k = mode*pi/L, over ions on the same lattice that are heavy enough to stay put.
    An even mode keeps the walls neutral and the mean displacement zero."""
    w = dx / ppc
    sp = [Species("e", -1.0, 1.0, w, 0.0, ppc), Species("i", 1.0, 1e12, w, 0.0, ppc)]
    phys = Physics(ncells=ncells, dx=dx, dt=dt, species=sp, processes=[], m_neutral=1e12)
    L = ncells * dx
    n = ncells * ppc
    x0 = (np.arange(n, dtype=np.float64) + 0.5) * (L / n)
    k = mode * math.pi / L
    loads = []
    for si in range(2):
        x = x0 + (amplitude * np.sin(k * x0) if si == 0 else 0.0)
        xc = x / dx
        cell = np.floor(xc).astype(np.int32)
        off = xc - cell
        z = np.zeros(n)
        loads.append(Load(cell, off, z.copy(), z.copy(), z.copy(),
                          np.arange(si * n, (si + 1) * n, dtype=np.uint32)))
    return phys, loads
