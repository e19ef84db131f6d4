"""Host data in single precision: pic_load_particles_f32 and pic_get_particles_f32.

The float entry points move 24 instead of 40 bytes per particle through the host link.
They must be the double entry points with the values rounded to float and nothing
else: a run loaded from float arrays is bit-identical to one loaded from the same
values widened to double, and a float read-back is the double read-back rounded once.
"""
import numpy as np
import pytest

from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W
from tests.gpu_common import by_id, ensure_built, requires_gpu

pytestmark = [pytest.mark.gpu, requires_gpu]


def _float_loads(phys, seed):
    """The workload's load with offsets and velocities representable in float."""
    out = []
    for ld in W.initial_load(phys, seed=seed):
        off = np.minimum(ld.off.astype(np.float32), np.float32(1.0) - np.float32(2.0 ** -24))
        out.append(W.Load(ld.cell, off, ld.vx.astype(np.float32), ld.vy.astype(np.float32),
                          ld.vz.astype(np.float32), ld.id))
    return out


def _widened(loads):
    return [W.Load(ld.cell, ld.off.astype(np.float64), ld.vx.astype(np.float64),
                   ld.vy.astype(np.float64), ld.vz.astype(np.float64), ld.id) for ld in loads]


@pytest.mark.parametrize("precision", [capi.FP32, capi.FP64])
def test_float_load_equals_double_load(precision):
    ensure_built()
    phys = W.magnetized_source(ncells=96, ppc=40, seed=3, nu=0.1, capacity_factor=3.0)
    f32 = _float_loads(phys, 3)
    runs = []
    for loads in (f32, _widened(f32)):
        sim = capi.Sim(phys, precision=precision, sort_interval=6)
        sim.load_all(loads)
        sim.step(25)
        runs.append(([by_id(sim.particles(0, s, cell_units=True)) for s in range(2)],
                     sim.moments(0)))
        sim.close()
    (a, ma), (b, mb) = runs
    for x, y in zip(a, b):
        for k in x:
            np.testing.assert_array_equal(x[k], y[k], err_msg=k)
    for k in ("live", "wall_count", "collisions", "density", "E"):
        np.testing.assert_array_equal(ma[k], mb[k], err_msg=k)


@pytest.mark.parametrize("precision", [capi.FP32, capi.FP64])
@pytest.mark.parametrize("cell_units", [False, True])
def test_float_read_back_is_the_double_read_back_rounded(precision, cell_units):
    ensure_built()
    phys = W.bounded_small(ncells=80, ppc=30, seed=5)
    sim = capi.Sim(phys, precision=precision, sort_interval=5)
    sim.load_all(W.initial_load(phys, seed=5))
    sim.step(12)
    for s in range(2):
        d = sim.particles(0, s, cell_units=cell_units)
        f = sim.particles(0, s, cell_units=cell_units, dtype=np.float32)
        for k in ("cell", "id", "state"):
            np.testing.assert_array_equal(d[k], f[k])
        for k in ("off", "vx", "vy", "vz"):
            assert f[k].dtype == np.float32
            want = d[k].astype(np.float32)
            if k == "off":  # an offset that rounds up to 1 stays just below it
                want = np.minimum(want, np.float32(1.0) - np.float32(2.0 ** -24))
            np.testing.assert_array_equal(want, f[k], err_msg=k)
    sim.close()


def test_fp64_offset_next_to_one_reads_back_reloadable():
    """An FP64-form offset of 1 - 2^-30 rounds to 1.0f; the float read-back keeps the
    particle in its cell at the largest float below 1, and loads again."""
    ensure_built()
    sp = [W.Species("e", -1.0, 1.0, 0.1, 1.0, 0)]
    phys = W.Physics(ncells=8, dx=0.5, dt=0.05, species=sp, processes=[],
                     field=W.FIELD_NONE, bc=W.BC_PERIODIC, seed=2)
    off = np.array([1.0 - 2.0 ** -30, 0.25, 1.0 - 2.0 ** -24, 0.0])
    z = np.zeros(4)
    ld = W.Load(np.array([3, 4, 7, 0], np.int32), off, z.copy(), z.copy(), z.copy(),
                np.arange(4, dtype=np.uint32))
    a = capi.Sim(phys, precision=capi.FP64)
    a.load_all([ld])
    f = by_id(a.particles(0, 0, dtype=np.float32))
    a.close()
    np.testing.assert_array_equal(f["cell"], [3, 4, 7, 0])
    np.testing.assert_array_equal(f["off"], np.array([1.0 - 2.0 ** -24, 0.25, 1.0 - 2.0 ** -24,
                                                      0.0], np.float32))
    b = capi.Sim(phys, precision=capi.FP64)
    b.load_all([W.Load(f["cell"], f["off"], f["vx"], f["vy"], f["vz"], f["id"])])
    b.sync()
    g = by_id(b.particles(0, 0))
    b.close()
    np.testing.assert_array_equal(g["cell"], [3, 4, 7, 0])
    assert (g["off"] < 1.0).all()


def test_float_offset_of_one_is_rejected():
    ensure_built()
    phys = W.bounded_small(ncells=8, ppc=4, seed=2)
    loads = _float_loads(phys, 2)
    loads[0].off[3] = np.float32(1.0)
    sim = capi.Sim(phys, precision=capi.FP32)
    sim.load_all(loads)
    with pytest.raises(capi.PicError) as e:
        sim.sync()
    assert e.value.code == -1
    sim.close()
