"""ctypes front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline
leg use it to produce expected values.  Nothing in the GPU library imports it.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List

import numpy as np

from . import build as _build

MAX_SPECIES = 4
MAX_PROC = 8


class _Species(C.Structure):
    _fields_ = [("charge", C.c_double), ("mass", C.c_double), ("weight", C.c_double),
                ("temperature", C.c_double), ("nstep", C.c_int32), ("sn2d", C.c_int32)]


class _Process(C.Structure):
    _fields_ = [("kind", C.c_int32), ("species", C.c_int32), ("product", C.c_int32),
                ("pad", C.c_int32), ("nu", C.c_double), ("threshold", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("ncells", C.c_int32), ("bc", C.c_int32), ("field", C.c_int32),
                ("nspecies", C.c_int32), ("dx", C.c_double), ("dt", C.c_double),
                ("eps0", C.c_double), ("E_ext", C.c_double), ("B", C.c_double * 3),
                ("T_neutral", C.c_double), ("m_neutral", C.c_double),
                ("sp", _Species * MAX_SPECIES), ("nproc", C.c_int32), ("smooth", C.c_int32),
                ("proc", _Process * MAX_PROC), ("seed", C.c_uint64), ("target", C.c_int32),
                ("nref", C.c_int32)]


class _Moments(C.Structure):
    _fields_ = [("step", C.c_int64), ("live", C.c_int64 * MAX_SPECIES),
                ("wall_count", (C.c_int64 * 2) * MAX_SPECIES),
                ("wall_energy", (C.c_double * 2) * MAX_SPECIES),
                ("collisions", C.c_int64 * MAX_PROC),
                ("kinetic", C.c_double * MAX_SPECIES)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Params)]
        L.orc_destroy.argtypes = [C.c_void_p]
        P = C.c_void_p
        L.orc_load.argtypes = [C.c_void_p, C.c_int32, C.c_int64, P, P, P, P, P, P, P, P]
        L.orc_step.argtypes = [C.c_void_p, C.c_int64]
        L.orc_set_field.argtypes = [C.c_void_p, P]
        L.orc_set_step.argtypes = [C.c_void_p, C.c_int64, C.c_uint32]
        L.orc_step_loop.argtypes = [C.c_void_p]
        L.orc_step_finish.argtypes = [C.c_void_p]
        L.orc_births_take.restype = C.c_int64
        L.orc_births_take.argtypes = [C.c_void_p, C.c_int32, C.c_int32, P, C.c_int64]
        L.orc_births_add.argtypes = [C.c_void_p, P, C.c_int64]
        L.orc_last_parents.restype = C.c_int64
        L.orc_last_parents.argtypes = [C.c_void_p, P, C.c_int64]
        L.orc_count.restype = C.c_int64
        L.orc_count.argtypes = [C.c_void_p, C.c_int32]
        L.orc_get.argtypes = [C.c_void_p, C.c_int32, P, P, P, P, P, P, P, P]
        L.orc_moments_get.argtypes = [C.c_void_p, C.POINTER(_Moments), P, P, P]
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_poisson.argtypes = [C.c_int32, C.c_double, C.c_double, P, P, P]
        L.orc_smooth.argtypes = [C.c_int32, P]
        L.orc_smooth.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# one recorded ionization (orc_birth_rec), C layout
BIRTH = np.dtype([("parent", np.uint32), ("esp", np.int32), ("isp", np.int32),
                  ("psp", np.int32), ("cell", np.int32), ("pad", np.int32),
                  ("off", np.float64), ("yp", np.float64), ("e", np.float64, (3,)),
                  ("i", np.float64, (3,))], align=True)


def params_struct(phys) -> _Params:
    p = _Params()
    p.ncells = phys.ncells
    p.bc = phys.bc
    p.field = phys.field
    p.nspecies = len(phys.species)
    p.dx, p.dt, p.eps0, p.E_ext = phys.dx, phys.dt, phys.eps0, phys.E_ext
    for k in range(3):
        p.B[k] = phys.B[k]
    p.T_neutral, p.m_neutral = phys.T_neutral, phys.m_neutral
    for i, s in enumerate(phys.species):
        p.sp[i] = _Species(s.charge, s.mass, s.weight, s.temperature, s.nstep, s.sn2d)
    p.nproc = len(phys.processes)
    p.smooth = phys.smooth
    for k, q in enumerate(phys.processes):
        p.proc[k] = _Process(q.kind, q.species, q.product, 0, q.nu, q.threshold)
    p.seed = phys.seed
    p.target, p.nref = phys.target, phys.nref
    return p


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 4-word counter under one 2-word key."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def poisson(rho, dx: float, eps0: float = 1.0):
    """Thomas solve of the grounded Dirichlet problem; returns (phi, E)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    N = len(rho) - 1
    phi = np.zeros(N + 1)
    E = np.zeros(N + 1)
    rc = lib().orc_poisson(N, dx, eps0, _ptr(rho), _ptr(phi), _ptr(E))
    if rc:
        raise RuntimeError("orc_poisson failed: %d" % rc)
    return phi, E


def smooth(rho):
    """The density smoother (1-2-1 filter of the interior entries); returns a copy."""
    out = np.array(rho, dtype=np.float64, copy=True)
    lib().orc_smooth(len(out) - 1, _ptr(out))
    return out


class Oracle:
    """One bounded-plasma instance advanced by the FP64 CPU oracle."""

    def __init__(self, phys):
        self.phys = phys
        self._p = params_struct(phys)
        self._h = lib().orc_create(C.byref(self._p))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def load(self, species: int, ld) -> None:
        arrs = [np.ascontiguousarray(ld.cell, dtype=np.int32),
                np.ascontiguousarray(ld.off, dtype=np.float64),
                np.ascontiguousarray(ld.vx, dtype=np.float64),
                np.ascontiguousarray(ld.vy, dtype=np.float64),
                np.ascontiguousarray(ld.vz, dtype=np.float64),
                None if ld.id is None else np.ascontiguousarray(ld.id, dtype=np.uint32),
                None if getattr(ld, "state", None) is None else
                np.ascontiguousarray(ld.state, dtype=np.uint8),
                None if getattr(ld, "yp", None) is None else
                np.ascontiguousarray(ld.yp, dtype=np.float64)]
        rc = lib().orc_load(self._h, species, len(arrs[0]), *[_ptr(a) for a in arrs])
        if rc:
            raise ValueError("orc_load failed: %d" % rc)

    def load_all(self, loads: List) -> None:
        for i, ld in enumerate(loads):
            self.load(i, ld)

    def step(self, n: int = 1) -> None:
        rc = lib().orc_step(self._h, n)
        if rc:
            raise RuntimeError("orc_step failed: %d" % rc)

    def set_field(self, E) -> None:
        """Use E (N+1 node values) as the next step's field instead of the one formed
        from this instance's own particles."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        if E.shape != (self.phys.ncells + 1,):
            raise ValueError("E must have ncells + 1 entries")
        rc = lib().orc_set_field(self._h, _ptr(E))
        if rc:
            raise RuntimeError("orc_set_field failed: %d" % rc)

    def set_step(self, step: int, next_id: int = 0) -> None:
        """Continue a saved run at `step` with created ids from at least next_id."""
        rc = lib().orc_set_step(self._h, step, next_id)
        if rc:
            raise RuntimeError("orc_set_step failed: %d" % rc)

    def step_loop(self) -> None:
        """The first half of a step: every particle moved, the ionizations recorded."""
        rc = lib().orc_step_loop(self._h)
        if rc:
            raise RuntimeError("orc_step_loop failed: %d" % rc)

    def step_finish(self) -> None:
        """The second half: products, target conversions, deposit, field."""
        rc = lib().orc_step_finish(self._h)
        if rc:
            raise RuntimeError("orc_step_finish failed: %d" % rc)

    def births_take(self, lo: int, hi: int) -> np.ndarray:
        """Between the halves: remove and return the ionizations recorded in cells
        outside [lo, hi) (a structured array of BIRTH records)."""
        cap = 1 << 20
        out = np.zeros(cap, BIRTH)
        n = lib().orc_births_take(self._h, lo, hi, _ptr(out), cap)
        if n < 0:
            raise RuntimeError("orc_births_take failed: %d" % n)
        return out[:n].copy()

    def births_add(self, recs: np.ndarray) -> None:
        """Between the halves: ionizations recorded by another subdomain in this one's
        cells, whose products are made here."""
        recs = np.ascontiguousarray(recs, dtype=BIRTH)
        rc = lib().orc_births_add(self._h, _ptr(recs) if len(recs) else None, len(recs))
        if rc:
            raise RuntimeError("orc_births_add failed: %d" % rc)

    def last_parents(self) -> np.ndarray:
        """Parent ids of the last step's ionizations, ascending (the order in which their
        children were numbered)."""
        n = lib().orc_last_parents(self._h, None, 0)
        out = np.zeros(max(n, 0), np.uint32)
        if n > 0:
            lib().orc_last_parents(self._h, _ptr(out), n)
        return out

    def particles(self, species: int) -> dict:
        n = lib().orc_count(self._h, species)
        out = dict(cell=np.zeros(n, np.int32), off=np.zeros(n), vx=np.zeros(n),
                   vy=np.zeros(n), vz=np.zeros(n), id=np.zeros(n, np.uint32),
                   state=np.zeros(n, np.uint8), yp=np.zeros(n))
        rc = lib().orc_get(self._h, species, *[_ptr(out[k]) for k in
                                                ("cell", "off", "vx", "vy", "vz", "id", "state",
                                                 "yp")])
        if rc:
            raise RuntimeError("orc_get failed: %d" % rc)
        return out

    def moments(self) -> dict:
        m = _Moments()
        N = self.phys.ncells
        S = len(self.phys.species)
        dens = np.zeros(S * (N + 1))
        phi = np.zeros(N + 1)
        E = np.zeros(N + 1)
        rc = lib().orc_moments_get(self._h, C.byref(m), _ptr(dens), _ptr(phi), _ptr(E))
        if rc:
            raise RuntimeError("orc_moments_get failed: %d" % rc)
        nproc = len(self.phys.processes)
        return dict(step=m.step,
                    live=np.array(m.live[:S], dtype=np.int64),
                    wall_count=np.array([list(m.wall_count[i]) for i in range(S)], np.int64),
                    wall_energy=np.array([list(m.wall_energy[i]) for i in range(S)]),
                    collisions=np.array(m.collisions[:nproc], dtype=np.int64),
                    kinetic=np.array(m.kinetic[:S]),
                    density=dens.reshape(S, N + 1), phi=phi, E=E)
