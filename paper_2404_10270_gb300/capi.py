"""ctypes binding of the C-ABI library ``libbitpic.so`` (include/pic.h).

Argument marshalling only: every step of the time step runs in the library's CUDA
kernels.  There is no CPU fallback: :func:`lib` raises when the compiled library is
missing, and every call that fails raises :class:`PicError` with the library's
message.  PyTorch is used only for device memory and the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
# $BITPIC_LIB selects another build of the library (the bounds-checked one, for tests)
LIB_PATH = os.environ.get("BITPIC_LIB") or os.path.join(HERE, "_native", "libbitpic.so")

MAX_SPECIES = 4
MAX_PROC = 8
FP32, FP64 = 0, 1
DEVICE, CELL_UNITS = 1, 2  # flags of load / get

STATUS = {0: "PIC_OK", -1: "PIC_EINVAL", -2: "PIC_ENOMEM", -3: "PIC_ECUDA",
          -4: "PIC_ECAPACITY", -5: "PIC_ENONFINITE", -6: "PIC_ETIMEOUT", -7: "PIC_ESTATE"}

EXPORTS = ("pic_create", "pic_load_particles", "pic_load_particles_f32", "pic_step", "pic_sync",
           "pic_moments", "pic_count", "pic_get_particles", "pic_get_particles_f32",
           "pic_restore_counters", "pic_charge_raw", "pic_profile", "pic_kernel_time",
           "pic_destroy", "pic_last_error", "pic_philox", "pic_field_solve_noalloc",
           "pic_load_yp", "pic_get_yp", "pic_bounds_probe")


class PicError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class pic_species(C.Structure):
    _fields_ = [("charge", C.c_double), ("mass", C.c_double), ("weight", C.c_double),
                ("temperature", C.c_double), ("capacity", C.c_int64), ("nstep", C.c_int32),
                ("sn2d", C.c_int32)]


class pic_process(C.Structure):
    _fields_ = [("kind", C.c_int32), ("species", C.c_int32), ("product", C.c_int32),
                ("pad", C.c_int32), ("nu", C.c_double), ("threshold", C.c_double)]


class pic_instance(C.Structure):
    _fields_ = [("ncells", C.c_int32), ("bc", C.c_int32), ("field", C.c_int32),
                ("nspecies", C.c_int32), ("dx", C.c_double), ("dt", C.c_double),
                ("eps0", C.c_double), ("E_ext", C.c_double), ("B", C.c_double * 3),
                ("T_neutral", C.c_double), ("m_neutral", C.c_double),
                ("sp", pic_species * MAX_SPECIES), ("nproc", C.c_int32), ("smooth", C.c_int32),
                ("proc", pic_process * MAX_PROC), ("seed", C.c_uint64), ("target", C.c_int32),
                ("nref", C.c_int32)]


class pic_config(C.Structure):
    _fields_ = [("n_instances", C.c_int32), ("precision", C.c_int32),
                ("sort_interval", C.c_int32), ("block", C.c_int32),
                ("inst", C.POINTER(pic_instance)), ("cuda_stream", C.c_void_p)]


class pic_moments_out(C.Structure):
    _fields_ = [("step", C.c_int64), ("live", C.c_int64 * MAX_SPECIES),
                ("wall_count", (C.c_int64 * 2) * MAX_SPECIES),
                ("wall_energy", (C.c_double * 2) * MAX_SPECIES),
                ("collisions", C.c_int64 * MAX_PROC),
                ("kinetic", C.c_double * MAX_SPECIES), ("next_id", C.c_int64)]


_lib = None


def lib():
    """The loaded library.  Raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libbitpic.so is not built (%s); run "
                               "paper_2404_10270_gb300.build.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
        L.pic_create.argtypes = [C.POINTER(pic_config), C.POINTER(C.c_void_p)]
        L.pic_load_particles.argtypes = [P, I32, I32, I64, P, P, P, P, P, P, P, I32]
        L.pic_load_particles_f32.argtypes = [P, I32, I32, I64, P, P, P, P, P, P, P, I32]
        L.pic_step.argtypes = [P, I64]
        L.pic_sync.argtypes = [P]
        L.pic_moments.argtypes = [P, I32, C.POINTER(pic_moments_out), P, P, P]
        L.pic_count.argtypes = [P, I32, I32, C.POINTER(C.c_int64)]
        L.pic_get_particles.argtypes = [P, I32, I32, I64, P, P, P, P, P, P, P, I32,
                                        C.POINTER(C.c_int64)]
        L.pic_get_particles_f32.argtypes = [P, I32, I32, I64, P, P, P, P, P, P, P, I32,
                                            C.POINTER(C.c_int64)]
        L.pic_restore_counters.argtypes = [P, I64, P]
        L.pic_charge_raw.argtypes = [P, I32, P, C.POINTER(C.c_int64)]
        L.pic_profile.argtypes = [P, I32]
        L.pic_kernel_time.argtypes = [P, I32, C.POINTER(C.c_int64), C.POINTER(C.c_double)]
        L.pic_destroy.argtypes = [P]
        L.pic_last_error.argtypes = [P]
        L.pic_last_error.restype = C.c_char_p
        L.pic_philox.argtypes = [C.c_uint64, P, P, I64, I32, P]
        L.pic_field_solve_noalloc.argtypes = [I32, I32, P, P, C.c_double, I64, C.c_double, P, P]
        L.pic_load_yp.argtypes = [P, I32, I32, I64, P, I32]
        L.pic_get_yp.argtypes = [P, I32, I32, I64, P, I32, C.POINTER(C.c_int64)]
        L.pic_bounds_probe.argtypes = [P]
        _lib = L
    return _lib


def _check(rc: int, handle=None):
    if rc != 0:
        msg = lib().pic_last_error(handle)
        raise PicError(rc, (msg or b"").decode(errors="replace"))


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _on_device(a) -> bool:
    return not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def _current_stream() -> Optional[int]:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover - torch without CUDA
        pass
    return None


def instance_struct(phys: W.Physics, capacity: Optional[Sequence[int]] = None) -> pic_instance:
    """pic_instance of a workload; capacity per species defaults to
    ppc * ncells * capacity_factor."""
    I = pic_instance()
    I.ncells = phys.ncells
    I.bc, I.field = phys.bc, phys.field
    I.nspecies = len(phys.species)
    I.dx, I.dt, I.eps0, I.E_ext = phys.dx, phys.dt, phys.eps0, phys.E_ext
    for k in range(3):
        I.B[k] = phys.B[k]
    I.T_neutral, I.m_neutral = phys.T_neutral, phys.m_neutral
    for i, s in enumerate(phys.species):
        cap = capacity[i] if capacity is not None else int(s.ppc * phys.ncells * s.capacity_factor)
        I.sp[i] = pic_species(s.charge, s.mass, s.weight, s.temperature, max(int(cap), 4),
                              s.nstep, getattr(s, "sn2d", 0))
    I.nproc = len(phys.processes)
    I.smooth = phys.smooth
    for k, q in enumerate(phys.processes):
        I.proc[k] = pic_process(q.kind, q.species, q.product, 0, q.nu, q.threshold)
    I.seed = phys.seed
    I.target, I.nref = phys.target, phys.nref
    return I


def philox(ctr: np.ndarray, key: int) -> np.ndarray:
    """The library's GPU Philox4x32-10 on n counters (array of shape (n, 4))."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(c)
    _check(lib().pic_philox(key, c.ctypes.data, out.ctypes.data, len(c), 0, _current_stream()))
    return out


class Sim:
    """A batch of bounded-plasma instances advanced on the GPU."""

    def __init__(self, phys: Sequence[W.Physics] | W.Physics, precision: int = FP32,
                 sort_interval: int = 0, block: int = 0, stream: Optional[int] = None,
                 capacity: Optional[List[Sequence[int]]] = None):
        if isinstance(phys, W.Physics):
            phys = [phys]
        self.phys = list(phys)
        self.precision = precision
        n = len(self.phys)
        self._inst = (pic_instance * n)()
        for i, p in enumerate(self.phys):
            self._inst[i] = instance_struct(p, None if capacity is None else capacity[i])
        cfg = pic_config()
        cfg.n_instances = n
        cfg.precision = precision
        cfg.sort_interval = sort_interval
        cfg.block = block
        cfg.inst = self._inst
        cfg.cuda_stream = stream if stream is not None else _current_stream()
        h = C.c_void_p()
        _check(lib().pic_create(C.byref(cfg), C.byref(h)), None)
        self._h = h

    # -- lifetime -------------------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().pic_destroy(h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls ----------------------------------------------------------------------
    def load(self, inst: int, species: int, ld, cell_units: bool = False) -> None:
        """Load particles from a workloads.Load (numpy, host) or an object with the
        same fields as CUDA tensors (cell int32, off/vx/vy/vz float64 or float32, id
        uint32/int32).  Float32 offsets and velocities (all four) go through
        pic_load_particles_f32, the rest through pic_load_particles.  cell_units:
        velocities are in cells per step (as particles(..., cell_units=True) returns
        them), for exact checkpoints."""
        arrs = [ld.cell, ld.off, ld.vx, ld.vy, ld.vz]
        f32 = all(str(getattr(a, "dtype", "")).endswith("float32") for a in arrs[1:])
        if isinstance(ld.cell, np.ndarray):
            ft = np.float32 if f32 else np.float64
            arrs = [np.ascontiguousarray(ld.cell, np.int32)] + \
                   [np.ascontiguousarray(a, ft) for a in arrs[1:]]
            ids = None if ld.id is None else np.ascontiguousarray(ld.id, np.uint32)
            st = getattr(ld, "state", None)
            st = None if st is None else np.ascontiguousarray(st, np.uint8)
            dev = 0
        else:
            ids = ld.id
            st = getattr(ld, "state", None)
            dev = 1 if _on_device(ld.cell) else 0
        n = len(arrs[0])
        flags = (DEVICE if dev else 0) | (CELL_UNITS if cell_units else 0)
        fn = lib().pic_load_particles_f32 if f32 else lib().pic_load_particles
        _check(fn(self._h, inst, species, n, *[_ptr(a) for a in arrs], _ptr(ids), _ptr(st),
                  flags), self._h)
        yp = getattr(ld, "yp", None)
        if yp is not None and getattr(self.phys[inst].species[species], "sn2d", 0):
            if isinstance(yp, np.ndarray):
                yp = np.ascontiguousarray(yp, np.float64)
            _check(lib().pic_load_yp(self._h, inst, species, n, _ptr(yp),
                                     DEVICE if _on_device(yp) else 0), self._h)

    def load_all(self, loads: List, inst: int = 0) -> None:
        for s, ld in enumerate(loads):
            self.load(inst, s, ld)

    def step(self, n: int = 1) -> None:
        _check(lib().pic_step(self._h, n), self._h)

    def sync(self) -> None:
        _check(lib().pic_sync(self._h), self._h)

    def count(self, inst: int, species: int) -> int:
        n = C.c_int64()
        _check(lib().pic_count(self._h, inst, species, C.byref(n)), self._h)
        return n.value

    def particles(self, inst: int, species: int, cell_units: bool = False,
                  dtype=np.float64) -> Dict[str, np.ndarray]:
        """Live particles of (inst, species) in storage order (host numpy); velocities
        physical, or in cells per step with cell_units=True.  dtype=np.float32 reads
        offsets and velocities through pic_get_particles_f32."""
        n = self.count(inst, species)
        ft = np.dtype(dtype)
        out = dict(cell=np.zeros(n, np.int32), off=np.zeros(n, ft), vx=np.zeros(n, ft),
                   vy=np.zeros(n, ft), vz=np.zeros(n, ft), id=np.zeros(n, np.uint32),
                   state=np.zeros(n, np.uint8))
        got = C.c_int64()
        fn = lib().pic_get_particles_f32 if ft == np.float32 else lib().pic_get_particles
        _check(fn(self._h, inst, species, n,
                  *[_ptr(out[k]) for k in ("cell", "off", "vx", "vy", "vz", "id", "state")],
                  CELL_UNITS if cell_units else 0, C.byref(got)), self._h)
        assert got.value == n
        # the y coordinates of a 2-D species (zeros for the others), same order
        out["yp"] = np.zeros(n)
        if getattr(self.phys[inst].species[species], "sn2d", 0):
            _check(lib().pic_get_yp(self._h, inst, species, n, out["yp"].ctypes.data, 0,
                                    C.byref(got)), self._h)
            assert got.value == n
        return out

    def moments(self, inst: int = 0) -> dict:
        p = self.phys[inst]
        N, S = p.ncells, len(p.species)
        m = pic_moments_out()
        dens = np.zeros(S * (N + 1))
        phi = np.zeros(N + 1)
        E = np.zeros(N + 1)
        _check(lib().pic_moments(self._h, inst, C.byref(m), _ptr(dens), _ptr(phi), _ptr(E)), self._h)
        return dict(step=m.step, live=np.array(m.live[:S], np.int64),
                    wall_count=np.array([list(m.wall_count[i]) for i in range(S)], np.int64),
                    wall_energy=np.array([list(m.wall_energy[i]) for i in range(S)]),
                    collisions=np.array(m.collisions[:len(p.processes)], np.int64),
                    kinetic=np.array(m.kinetic[:S]), next_id=m.next_id,
                    density=dens.reshape(S, N + 1), phi=phi, E=E)

    def restore_counters(self, step: int, next_id=None) -> None:
        """Set the step count and (optionally) each instance's next particle id."""
        arr = None if next_id is None else np.ascontiguousarray(next_id, np.uint64)
        _check(lib().pic_restore_counters(self._h, step, _ptr(arr)), self._h)

    def charge_raw(self, inst: int = 0):
        p = self.phys[inst]
        N, S = p.ncells, len(p.species)
        out = np.zeros(S * (N + 1), np.int64)
        unit = C.c_int64()
        _check(lib().pic_charge_raw(self._h, inst, out.ctypes.data, C.byref(unit)), self._h)
        return out.reshape(S, N + 1), unit.value

    def profile(self, enable: bool = True) -> None:
        _check(lib().pic_profile(self._h, 1 if enable else 0), self._h)

    def kernel_time(self, which: int):
        """(launches, total_ms) of kernel class 0 mover, 1 field, 2 sort, 3 other,
        5 the mover of a sort step; class 4 gives (kernels launched, 0)."""
        n = C.c_int64()
        ms = C.c_double()
        _check(lib().pic_kernel_time(self._h, which, C.byref(n), C.byref(ms)), self._h)
        return n.value, ms.value
