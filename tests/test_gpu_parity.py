"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances are the accuracy contract of the method's two forms:
  * FP64 form: particles matched by id within 1e-12 relative over 100 steps, wall
    absorption counts and collision event counts bit-exact;
  * FP32 form (FP32 state, fixed-point deposit, FP64 field): 1e-5 relative over 10 steps.
"""
import math

import numpy as np
import pytest

from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W
from tests.gpu_common import (assert_same_clocks, by_id, ensure_built, particle_errors,
                              requires_gpu, run_gpu, run_oracle)
from tests.helpers import read_kat

pytestmark = [pytest.mark.gpu, requires_gpu]


def test_philox_known_answers_and_oracle():
    from oracle.oracle import philox as ophilox
    ensure_built()
    for ctr, key, out in read_kat():
        k = key[0] | (key[1] << 32)
        np.testing.assert_array_equal(capi.philox(np.array([ctr]), k)[0], np.array(out, np.uint32))
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(3000, 4), dtype=np.uint64).astype(np.uint32)
    key = 0x1234_5678_9ABC_DEF0
    got = capi.philox(ctr, key)
    kw = np.array([key & 0xFFFFFFFF, key >> 32], np.uint32)
    for i in range(0, 3000, 97):
        np.testing.assert_array_equal(got[i], ophilox(ctr[i], kw))


_CURAND_PHILOX = r"""
#include <cstdint>
#include <curand_kernel.h>
__global__ void k_ref(const uint4* c, const uint2* k, uint4* o, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = curand_Philox4x32_10(c[i], k[i]);
}
extern "C" int curand_philox(const uint32_t* c, const uint32_t* k, uint32_t* o, int n)
{
    uint4 *dc = nullptr, *dout = nullptr;
    uint2* dk = nullptr;
    cudaError_t e = cudaMalloc(&dc, 16 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dk, 8 * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&dout, 16 * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(dc, c, 16 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, k, 8 * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_ref<<<(n + 127) / 128, 128>>>(dc, dk, dout, n);
        e = cudaMemcpy(o, dout, 16 * (size_t)n, cudaMemcpyDeviceToHost);
    }
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return (int)e;
}
"""


def test_oracle_philox_matches_curand(tmp_path):
    """The oracle's Philox4x32-10 against the CUDA toolkit's own (cuRAND's device
    function, called on random counters and keys): an independent implementation of
    the published generator.  The GPU path is checked against the oracle above."""
    import ctypes as C
    import shutil
    import subprocess
    from oracle.oracle import philox as ophilox
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = tmp_path / "curand_philox.cu"
    src.write_text(_CURAND_PHILOX)
    so = tmp_path / "libcurand_philox.so"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler",
                    "-fPIC", "-o", str(so), str(src)], check=True, capture_output=True)
    lib = C.CDLL(str(so))
    rng = np.random.default_rng(7)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0], key[0] = 0, 0
    ctr[1], key[1] = 0xFFFFFFFF, 0xFFFFFFFF
    out = np.zeros((n, 4), np.uint32)
    P = C.POINTER(C.c_uint32)
    rc = lib.curand_philox(ctr.ctypes.data_as(P), key.ctypes.data_as(P), out.ctypes.data_as(P), n)
    assert rc == 0
    for i in list(range(0, n, 37)) + [0, 1]:
        np.testing.assert_array_equal(ophilox(ctr[i], key[i]), out[i])


@pytest.mark.parametrize("precision,steps,tol", [(capi.FP64, 100, 1e-12), (capi.FP32, 10, 1e-5)])
def test_bounded_small_parity(precision, steps, tol):
    phys = W.bounded_small()
    loads = W.initial_load(phys, seed=1)
    g, gm = run_gpu(phys, loads, steps, precision, sort_interval=20)
    o, om = run_oracle(phys, loads, steps)
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < tol and ev < tol, (s, ex, ev)
    assert_same_clocks(g, o)
    assert gm["step"] == om["step"] == steps
    if precision == capi.FP64:
        np.testing.assert_array_equal(gm["wall_count"], om["wall_count"])
        np.testing.assert_array_equal(gm["collisions"], om["collisions"])
        np.testing.assert_array_equal(gm["live"], om["live"])
        assert om["collisions"].sum() > 0 and om["wall_count"].sum() > 0
        np.testing.assert_allclose(gm["wall_energy"], om["wall_energy"], rtol=1e-12)
        np.testing.assert_allclose(gm["kinetic"], om["kinetic"], rtol=1e-12)
        scale = np.abs(om["E"]).max()
        np.testing.assert_allclose(gm["E"], om["E"], rtol=0, atol=1e-11 * scale)
        np.testing.assert_allclose(gm["phi"], om["phi"], rtol=0, atol=1e-11 * np.abs(om["phi"]).max())
        np.testing.assert_allclose(gm["density"], om["density"], rtol=1e-13, atol=1e-13)
    else:
        # counts can differ only by particles within rounding of a wall
        assert np.abs(gm["wall_count"] - om["wall_count"]).sum() <= 2
        np.testing.assert_allclose(gm["kinetic"], om["kinetic"], rtol=1e-5)
        scale = np.abs(om["E"]).max()
        np.testing.assert_allclose(gm["E"], om["E"], rtol=0, atol=1e-5 * scale)
        np.testing.assert_allclose(gm["density"], om["density"], rtol=0, atol=1e-5)


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_initial_field_matches_oracle(precision):
    phys = W.bounded_small(ncells=300, ppc=37, seed=3)  # ragged tiles
    loads = W.initial_load(phys, seed=3)
    g, gm = run_gpu(phys, loads, 0, precision)
    o, om = run_oracle(phys, loads, 0)
    tol = 1e-12 if precision == capi.FP64 else 1e-6
    np.testing.assert_allclose(gm["E"], om["E"], rtol=0, atol=tol * np.abs(om["E"]).max())
    np.testing.assert_allclose(gm["density"], om["density"], rtol=0, atol=tol)
    np.testing.assert_allclose(gm["phi"], om["phi"], rtol=0, atol=tol * np.abs(om["phi"]).max())


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_deposit_is_exact_fixed_point(precision):
    """Every live particle adds exactly one unit S split over its two nodes."""
    ensure_built()
    phys = W.bounded_small(ncells=64, ppc=33, seed=5)
    loads = W.initial_load(phys, seed=5)
    runs = []
    for rep in range(2):
        sim = capi.Sim(phys, precision=precision, sort_interval=7)
        sim.load_all(loads)
        sim.step(15)
        raw, unit = sim.charge_raw(0)
        m = sim.moments(0)
        for s in range(2):
            assert sum(map(int, raw[s])) == int(m["live"][s]) * unit
        runs.append(raw.copy())
        sim.close()
    np.testing.assert_array_equal(runs[0], runs[1])  # run-to-run deterministic


def test_batch_instance_equals_instance_alone():
    ensure_built()
    physs = [W.bounded_small(ncells=n, ppc=p, seed=sd) for n, p, sd in
             ((64, 20, 11), (100, 13, 12), (37, 50, 13))]
    loads = [W.initial_load(p, seed=i + 20) for i, p in enumerate(physs)]
    sim = capi.Sim(physs, precision=capi.FP64, sort_interval=5)
    for i, ld in enumerate(loads):
        sim.load_all(ld, inst=i)
    sim.step(30)
    batch = [[by_id(sim.particles(i, s)) for s in range(2)] for i in range(3)]
    bm = [sim.moments(i) for i in range(3)]
    sim.close()
    for i, (p, ld) in enumerate(zip(physs, loads)):
        g, m = run_gpu(p, ld, 30, capi.FP64, sort_interval=5)
        for s in range(2):
            a = by_id(g[s])
            for k in a:
                np.testing.assert_array_equal(a[k], batch[i][s][k])
        np.testing.assert_array_equal(m["collisions"], bm[i]["collisions"])
        np.testing.assert_array_equal(m["E"], bm[i]["E"])


def test_results_do_not_depend_on_launch_shape_or_sort_interval():
    phys = W.bounded_small(ncells=96, ppc=40, seed=7)
    loads = W.initial_load(phys, seed=7)
    ref = None
    for block, sort in ((256, 0), (128, 5), (512, 20), (256, 1)):
        g, m = run_gpu(phys, loads, 25, capi.FP64, sort_interval=sort, block=block)
        cur = ([by_id(x) for x in g], m)
        if ref is None:
            ref = cur
            continue
        for a, b in zip(ref[0], cur[0]):
            for k in a:
                np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(ref[1]["E"], cur[1]["E"])
        np.testing.assert_array_equal(ref[1]["collisions"], cur[1]["collisions"])


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_graph_replay_equals_direct_launches(precision):
    """pic_step replays one captured CUDA graph per window of steps inside a sort cycle
    (cached by store copy, place in the cycle, length and whether the step before counted
    cells for the sort); with kernel timing on it launches kernels one by one.  Calls of
    3 + 17 steps, of one step at a time, and of mixed lengths that start mid-cycle all
    give the direct launches' results."""
    ensure_built()
    phys = W.magnetized_source(ncells=40, ppc=30, seed=14, nu=0.3, capacity_factor=3.0,
                               B=2.0 if precision == capi.FP64 else 0.0)
    loads = W.initial_load(phys, seed=14)
    out = []
    for calls in ("profile", (3, 17), (1,) * 20, (2, 5, 1, 6, 3, 3)):
        sim = capi.Sim(phys, precision=precision, sort_interval=4)
        sim.load_all(loads)
        if calls == "profile":
            sim.profile(True)
            calls = (3, 17)
        for n in calls:
            sim.step(n)
        out.append(([by_id(sim.particles(0, s)) for s in range(2)], sim.moments(0)))
        sim.close()
    a, am = out[0]
    for b, bm in out[1:]:
        for x, y in zip(a, b):
            for k in x:
                np.testing.assert_array_equal(x[k], y[k])
        np.testing.assert_array_equal(am["E"], bm["E"])
        np.testing.assert_array_equal(am["collisions"], bm["collisions"])
        assert am["step"] == bm["step"] == 20


def test_autotuner_changes_nothing_but_speed(tmp_path, monkeypatch):
    """block = 0 and sort_interval = -1 make the library time its candidates on the first
    steps of the run; the particles must come out exactly as with a fixed choice, and
    the choice lands in the cache file."""
    import json
    ensure_built()
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("BITPIC_TUNE_CACHE", str(cache))
    phys = W.bounded_small(ncells=128, ppc=50, seed=15)
    loads = W.initial_load(phys, seed=15)
    runs = []
    for block, sort in ((0, -1), (256, 20)):
        sim = capi.Sim(phys, precision=capi.FP64, sort_interval=sort, block=block)
        sim.load_all(loads)
        sim.step(400)
        runs.append([by_id(sim.particles(0, s)) for s in range(2)])
        sim.close()
    for x, y in zip(*runs):
        for k in x:
            np.testing.assert_array_equal(x[k], y[k])
    entries = json.loads(cache.read_text())
    assert len(entries) == 1
    (block, sort), = entries.values()
    assert block in (128, 256, 512) and sort in (10, 20, 40, 80)


def test_load_order_does_not_matter():
    phys = W.bounded_small(ncells=32, ppc=25, seed=9)
    loads = W.initial_load(phys, seed=9)
    rng = np.random.default_rng(9)
    perm = [ld.take(rng.permutation(len(ld))) for ld in loads]
    a, am = run_gpu(phys, loads, 20, capi.FP64)
    b, bm = run_gpu(phys, perm, 20, capi.FP64)
    for x, y in zip(a, b):
        x, y = by_id(x), by_id(y)
        for k in x:
            np.testing.assert_array_equal(x[k], y[k])
    np.testing.assert_array_equal(am["E"], bm["E"])


def test_magnetized_source_with_ionization_fp64_parity():
    """Boris push, volume re-injection, elastic + ionization + charge exchange."""
    phys = W.magnetized_source(ncells=64, ppc=40, seed=2, nu=0.2, capacity_factor=3.0)
    loads = W.initial_load(phys, seed=2)
    steps = 100
    g, gm = run_gpu(phys, loads, steps, capi.FP64, sort_interval=10)
    o, om = run_oracle(phys, loads, steps)
    assert om["collisions"][1] > 0  # some ionization happened
    np.testing.assert_array_equal(gm["collisions"], om["collisions"])
    np.testing.assert_array_equal(gm["wall_count"], om["wall_count"])
    np.testing.assert_array_equal(gm["live"], om["live"])
    assert gm["next_id"] == 2 * phys.ncells * 40 + 2 * int(om["collisions"][1])
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < 1e-12 and ev < 1e-12, (s, ex, ev)
    assert_same_clocks(g, o)


def test_thousands_of_ionizations_a_step_number_children_like_the_oracle():
    """Several thousand ionizations a step with ids past 2^16: the children's ids (the
    rank of each parent id among the step's events) come from a multi-tile, three-pass
    sort of the parent ids and must equal the oracle's, particle by particle."""
    phys = W.magnetized_source(ncells=512, ppc=100, seed=12, nu=3.0, capacity_factor=3.0)
    loads = W.initial_load(phys, seed=12)
    steps = 6
    g, gm = run_gpu(phys, loads, steps, capi.FP64, sort_interval=4)
    o, om = run_oracle(phys, loads, steps)
    assert int(om["collisions"][1]) > 3 * 4096  # several tiles of events a step
    np.testing.assert_array_equal(gm["collisions"], om["collisions"])
    np.testing.assert_array_equal(gm["live"], om["live"])
    assert gm["next_id"] == 2 * phys.ncells * 100 + 2 * int(om["collisions"][1])
    assert 2 * phys.ncells * 100 > 1 << 16  # three passes of the sort
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < 1e-12 and ev < 1e-12, (s, ex, ev)
    assert_same_clocks(g, o)


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_checkpoint_restart_is_bit_identical(precision):
    """particles (cell units + collision clocks) + step + next ids reloaded into a
    fresh handle continue exactly like the uninterrupted run."""
    ensure_built()
    phys = W.magnetized_source(ncells=48, ppc=30, seed=8, nu=0.3, capacity_factor=3.0)
    loads = W.initial_load(phys, seed=8)
    ref = capi.Sim(phys, precision=precision, sort_interval=7)
    ref.load_all(loads)
    ref.step(45)
    want = [by_id(ref.particles(0, s, cell_units=True)) for s in range(2)]
    ref.close()

    a = capi.Sim(phys, precision=precision, sort_interval=7)
    a.load_all(loads)
    a.step(25)
    snap = [a.particles(0, s, cell_units=True) for s in range(2)]
    m = a.moments(0)
    a.close()
    b = capi.Sim(phys, precision=precision, sort_interval=7)
    for s, p in enumerate(snap):
        b.load(0, s, W.Load(p["cell"], p["off"], p["vx"], p["vy"], p["vz"], p["id"], p["state"]),
               cell_units=True)
    b.restore_counters(m["step"], [m["next_id"]])
    b.step(20)
    got = [by_id(b.particles(0, s, cell_units=True)) for s in range(2)]
    b.close()
    for x, y in zip(want, got):
        for k in x:
            np.testing.assert_array_equal(x[k], y[k])


@pytest.mark.parametrize("B", [2.0, 0.0])
def test_magnetized_source_fp32_parity(B):
    # B = 0: the plain push, and in a batch large enough (or with the tests' setting) the
    # mover pair, whose queued clock tests include re-injected particles and products
    phys = W.magnetized_source(ncells=64, ppc=40, seed=4, nu=0.2, capacity_factor=3.0, B=B)
    loads = W.initial_load(phys, seed=4)
    g, gm = run_gpu(phys, loads, 10, capi.FP32, sort_interval=5)
    o, om = run_oracle(phys, loads, 10)
    np.testing.assert_array_equal(gm["live"], om["live"])
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < 1e-5 and ev < 1e-5, (s, ex, ev)


@pytest.mark.parametrize("precision", [capi.FP64, capi.FP32])
def test_edge_cases_empty_single_cell_and_ragged(precision):
    # a single cell; an empty species; counts that are not multiples of 4 or a tile
    sp = [W.Species("e", -1.0, 1.0, 0.1, 1.0, 3), W.Species("i", 1.0, 100.0, 0.1, 1.0, 0)]
    phys = W.Physics(ncells=1, dx=0.5, dt=0.05, species=sp,
                     processes=[W.Process(W.PROC_ELASTIC, 0, 0.5)], m_neutral=100.0, seed=3)
    loads = W.initial_load(phys, seed=3)
    g, gm = run_gpu(phys, loads, 30, precision)
    o, om = run_oracle(phys, loads, 30)
    np.testing.assert_array_equal(gm["live"], om["live"])
    np.testing.assert_array_equal(gm["wall_count"], om["wall_count"])
    tol = 1e-12 if precision == capi.FP64 else 1e-5
    for ex, ev in particle_errors(phys, g, o):
        assert ex < tol and ev < tol
    # ragged: 1, 5, 1027 particles
    for n in (1, 5, 1027):
        phys = W.bounded_small(ncells=50, ppc=max(1, -(-n // 50)), seed=n)
        ld = W.initial_load(phys, seed=n)
        ld = [x.take(np.arange(min(n, len(x)))) for x in ld]
        g, gm = run_gpu(phys, ld, 12, precision)
        o, om = run_oracle(phys, ld, 12)
        np.testing.assert_array_equal(gm["live"], om["live"])
        for ex, ev in particle_errors(phys, g, o):
            assert ex < tol and ev < tol


def test_invalid_load_is_reported_then_state_is_sticky():
    ensure_built()
    phys = W.bounded_small(ncells=16, ppc=4)
    loads = W.initial_load(phys)
    loads[0].cell[3] = 99  # outside [0, 16)
    sim = capi.Sim(phys, precision=capi.FP32)
    sim.load_all(loads)
    with pytest.raises(capi.PicError) as e:
        sim.sync()
    assert e.value.code == -1
    with pytest.raises(capi.PicError) as e:
        sim.step(1)
    assert e.value.code == -7
    sim.close()


@pytest.mark.parametrize("sort", [0, 3])
def test_capacity_overflow_is_reported(sort):
    ensure_built()
    phys = W.magnetized_source(ncells=16, ppc=20, nu=5.0, capacity_factor=1.0)
    loads = W.initial_load(phys)
    sim = capi.Sim(phys, precision=capi.FP32, sort_interval=sort)
    sim.load_all(loads)
    sim.step(40)
    with pytest.raises(capi.PicError) as e:
        sim.sync()
    assert e.value.code == -4
    sim.close()


def test_fp64_move_rounds_exactly_like_the_oracle():
    """With no field and no collisions the FP64 step is the move alone: f' = f + u and
    f' - floor(f').  For -1 < f' < 2 the GPU reads the floor from the bits and forms
    f' - floor(f') as one addition of 0 or +-1; that must round exactly as the
    subtraction does, so after many crossings in both directions, landings close to a
    cell edge and moves of more than a cell, every position is the oracle's bit for
    bit."""
    ensure_built()
    n = 400
    sp = [W.Species("e", -1.0, 1.0, 0.5 / n, 30.0, n)]  # |u| ~ 0.55 cells per step
    phys = W.Physics(ncells=64, dx=0.5, dt=0.05, species=sp, processes=[],
                     bc=W.BC_PERIODIC, field=W.FIELD_NONE, seed=11)
    loads = W.initial_load(phys, seed=11)
    g, _ = run_gpu(phys, loads, 60, capi.FP64, sort_interval=7)
    o, _ = run_oracle(phys, loads, 60)
    g, o = by_id(g[0]), by_id(o[0])
    np.testing.assert_array_equal(g["id"], o["id"])
    np.testing.assert_array_equal(g["cell"], o["cell"])
    np.testing.assert_array_equal(g["off"].view(np.uint64), o["off"].view(np.uint64))
    np.testing.assert_array_equal(g["vx"], o["vx"])
    assert (np.abs(loads[0].vx) * phys.dt / phys.dx > 1).any()  # some move past a cell


@pytest.mark.parametrize("case", ["bounded", "source", "target"])
def test_mover_pair_changes_no_result(monkeypatch, case):
    """Plain FP32 steps of large batches use the mover pair: on the clock-test steps
    (multiples of 127) and after a load the variant with the collision-clock draw
    inline, on the others the variant that queues the few clocks needing a draw for the
    event kernel (after a candidate, and for re-injected particles and ionization
    products, which start with a fresh clock).  Both orders of work give the same state,
    bit for bit: over 260 steps (clock-test steps, graph-replayed sort cycles) and, but
    for the neutral-target case (its subcycled neutrals never draw), a reload of the
    state."""
    ensure_built()
    if case == "bounded":
        phys = W.bounded_small(ncells=200, ppc=60, seed=4)
    elif case == "source":  # volume source and ionization without magnetic field
        phys = W.magnetized_source(ncells=64, ppc=60, seed=4, B=0.0, nu=0.05, capacity_factor=3.0)
    else:  # the paper's case: neutral particle targets moved on the sort steps
        phys = W.ionization_case(ncells=300, ppc=40, seed=4, nu_iz=0.05)
    loads = W.initial_load(phys, seed=4)
    K = phys.sort_interval if case == "target" else 20

    def run(min_slots):
        monkeypatch.setenv("BITPIC_PAIR_MIN_SLOTS", str(min_slots))
        a = capi.Sim(phys, precision=capi.FP32, sort_interval=K)
        a.load_all(loads)
        if case == "target":
            a.step(260)
            out = [by_id(a.particles(0, s, cell_units=True)) for s in range(len(phys.species))]
            mm = a.moments(0)
            a.close()
            return out, mm
        a.step(150)
        snap = [a.particles(0, s, cell_units=True) for s in range(2)]
        m = a.moments(0)
        a.close()
        b = capi.Sim(phys, precision=capi.FP32, sort_interval=K)
        for s, p in enumerate(snap):
            b.load(0, s, W.Load(p["cell"], p["off"], p["vx"], p["vy"], p["vz"], p["id"],
                                p["state"]), cell_units=True)
        b.restore_counters(m["step"], [m["next_id"]])
        b.step(110)
        out = [by_id(b.particles(0, s, cell_units=True)) for s in range(2)]
        mm = b.moments(0)
        b.close()
        return out, mm

    a, ma = run(0)
    b, mb = run(1 << 62)
    for x, y in zip(a, b):
        assert set(x) == set(y)
        for k in x:
            np.testing.assert_array_equal(x[k], y[k], err_msg=k)
    for k in ("wall_count", "collisions", "live", "density", "E"):
        np.testing.assert_array_equal(ma[k], mb[k], err_msg=k)
    assert ma["collisions"].sum() > 0


def _wall_flood(n_per_cell):
    """Four cells, one species so hot (|u| ~ 100 cells/step) that nearly every particle
    reaches a wall in the first step: the rare-event queue takes one entry per particle."""
    sp = [W.Species("e", -1.0, 1.0, 0.5 / n_per_cell, 1.0e6, n_per_cell)]
    return W.Physics(ncells=4, dx=0.5, dt=0.05, species=sp, processes=[],
                     field=W.FIELD_NONE, seed=5)


@pytest.mark.parametrize("sort", [0, 2])
def test_wall_flood_within_the_queue_matches_oracle(sort):
    # 60,000 particles: within the queue's 65,536-entry floor; with sort interval 2 the
    # second step is a sort step
    ensure_built()
    phys = _wall_flood(15000)
    loads = W.initial_load(phys, seed=5)
    g, gm = run_gpu(phys, loads, 2, capi.FP64, sort_interval=sort)
    o, om = run_oracle(phys, loads, 2)
    np.testing.assert_array_equal(gm["live"], om["live"])
    np.testing.assert_array_equal(gm["wall_count"], om["wall_count"])
    assert gm["wall_count"].sum() > 0.95 * 60000
    np.testing.assert_allclose(gm["wall_energy"], om["wall_energy"], rtol=1e-12)


def test_rare_event_queue_overflow_is_reported():
    # 300,000 particles hitting the walls in one step overflow the queue (65,536 + a
    # sixteenth of the capacity): the step reports PIC_ECAPACITY, nothing is dropped silently
    ensure_built()
    phys = _wall_flood(75000)
    loads = W.initial_load(phys, seed=5)
    sim = capi.Sim(phys, precision=capi.FP32)
    sim.load_all(loads)
    sim.step(1)
    with pytest.raises(capi.PicError) as e:
        sim.sync()
    assert e.value.code == -4
    assert "rare-event queue" in str(e.value)
    sim.close()


@pytest.mark.parametrize("precision,steps,tol", [(capi.FP64, 100, 1e-12), (capi.FP32, 10, 1e-5)])
def test_magnetized_source_full_size(precision, steps, tol):
    """The magnetized workload at its full size: 4096 cells x 200 particles/cell/species
    (1,638,400 particles), oblique B, volume source, elastic + ionization + charge
    exchange.  FP64 bound 1e-12, FP32 1e-5, for every particle."""
    ensure_built()
    phys = W.magnetized_source(seed=1)
    loads = W.initial_load(phys, seed=1)
    sim = capi.Sim(phys, precision=precision, sort_interval=20)
    sim.load_all(loads)
    sim.step(steps)
    g = [sim.particles(0, s) for s in range(2)]
    gm = sim.moments(0)
    sim.close()
    o, om = run_oracle(phys, loads, steps)
    np.testing.assert_array_equal(gm["live"], om["live"])
    if precision == capi.FP64:
        np.testing.assert_array_equal(gm["collisions"], om["collisions"])
        np.testing.assert_array_equal(gm["wall_count"], om["wall_count"])
    assert om["collisions"][1] > 0  # ionization happened
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < tol and ev < tol, (s, ex, ev)
    assert_same_clocks(g, o)
