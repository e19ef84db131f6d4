"""The allocation-free field solve, checked against the handle's own field phase.

pic_field_solve_noalloc serves callers that cannot allocate device memory (code
running under CUDA graph capture, latency-critical loops, frameworks that own all
device memory through their own pools).  It must give the same E as the handle
computes from the same fixed-point deposit, on consecutive calls that reuse its
static scratch.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W
from tests.gpu_common import ensure_built, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _unit_and_z(phys):
    qw = [s.charge * s.weight for s in phys.species]
    delta = min(abs(x) for x in qw if x != 0)
    return delta, [int(round(x / delta)) for x in qw]


def _rho_from_raw(phys, raw, unit):
    """Charge density on the nodes from the fixed-point deposits (wall nodes: half
    cells), as the oracle's field phase takes it."""
    q = sum(s.charge * s.weight * raw[k].astype(np.float64) / unit
            for k, s in enumerate(phys.species))
    vol = np.full(phys.ncells + 1, phys.dx)
    vol[0] = vol[-1] = 0.5 * phys.dx
    return q / vol


def _solve(phys, dcharge, z, delta, unit, stream):
    import torch
    N = phys.ncells
    zc = (C.c_int32 * len(z))(*z)
    dE = torch.full((N + 1,), float("nan"), dtype=torch.float64, device="cuda")
    rc = capi.lib().pic_field_solve_noalloc(N, len(z), dcharge.data_ptr(), zc, delta, unit,
                                            phys.eps0, dE.data_ptr(), stream)
    assert rc == 0, capi.lib().pic_last_error(None)
    torch.cuda.synchronize()
    return dE.cpu().numpy()


@pytest.mark.parametrize("ncells,ppc", [(1, 8), (300, 40), (2047, 6), (65536, 2)])
@pytest.mark.parametrize("precision", [capi.FP32, capi.FP64])
def test_noalloc_field_matches_handle_field(precision, ncells, ppc):
    """From one node per thread of its scan block (300) to several (2047) and the
    maximum its static scratch holds (65,536 cells: the total U sits in the last slot),
    and the single cell; two calls in a row on fresh deposits each time.  Compared with
    the handle's field of the same deposits and with the oracle's solve of the charge
    density they stand for."""
    import torch
    from oracle.oracle import poisson
    ensure_built()
    phys = W.bounded_small(ncells=ncells, ppc=ppc, seed=6)
    loads = W.initial_load(phys, seed=6)
    sim = capi.Sim(phys, precision=precision, sort_interval=10)
    sim.load_all(loads)
    delta, z = _unit_and_z(phys)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):  # two calls in a row share the static scratch
        sim.step(7)
        raw, unit = sim.charge_raw(0)
        expect = sim.moments(0)["E"]
        dcharge = torch.from_numpy(raw.reshape(-1).copy()).cuda()
        got = _solve(phys, dcharge, z, delta, unit, stream)
        scale = max(np.abs(expect).max(), 1e-300)
        np.testing.assert_allclose(got, expect, rtol=0, atol=1e-12 * scale)
        _, Eo = poisson(_rho_from_raw(phys, raw, unit), phys.dx, phys.eps0)
        np.testing.assert_allclose(got, Eo, rtol=0, atol=1e-12 * scale)
    sim.close()


def test_noalloc_field_takes_the_deposits_unsmoothed():
    """For an instance with the density smoother, the call still solves for the charge it
    is given (no filter): the oracle's solve of the unfiltered density."""
    import torch
    from oracle.oracle import poisson
    ensure_built()
    phys = W.bounded_small(ncells=200, ppc=30, seed=9)
    phys.smooth = 1
    loads = W.initial_load(phys, seed=9)
    sim = capi.Sim(phys, precision=capi.FP64, sort_interval=10)
    sim.load_all(loads)
    sim.step(5)
    raw, unit = sim.charge_raw(0)
    sim.close()
    delta, z = _unit_and_z(phys)
    dcharge = torch.from_numpy(raw.reshape(-1).copy()).cuda()
    got = _solve(phys, dcharge, z, delta, unit, torch.cuda.current_stream().cuda_stream)
    _, Eo = poisson(_rho_from_raw(phys, raw, unit), phys.dx, phys.eps0)
    np.testing.assert_allclose(got, Eo, rtol=0, atol=1e-12 * np.abs(Eo).max())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    ensure_built()
    z = (C.c_int32 * 2)(-1, 1)
    dummy = torch.zeros(4, dtype=torch.int64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = capi.lib().pic_field_solve_noalloc(65537, 2, dummy.data_ptr(), z, 1.0, 1 << 24, 1.0,
                                            out.data_ptr(), None)
    assert rc == -1
    assert b"ncells" in capi.lib().pic_last_error(None)
