"""GPU parity of the density smoother (Section 2's "Density Smoother" phase, read as
the 1-2-1 filter of the interior node densities, walls kept).  The GPU filters the
integer node charges exactly (times 4, the 1/4 in the field scale); the oracle filters
the FP64 densities.  Same tolerances as the other parity tests."""
import numpy as np
import pytest

from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W
from tests.gpu_common import (assert_same_clocks, particle_errors, requires_gpu, run_gpu,
                              run_oracle)

pytestmark = [pytest.mark.gpu, requires_gpu]


@pytest.mark.parametrize("precision,steps,tol", [(capi.FP64, 100, 1e-12), (capi.FP32, 10, 1e-5)])
def test_smoothed_bounded_plasma(precision, steps, tol):
    phys = W.bounded_small()
    phys.smooth = 1
    loads = W.initial_load(phys, seed=1)
    g, gm = run_gpu(phys, loads, steps, precision, sort_interval=20)
    o, om = run_oracle(phys, loads, steps)
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < tol and ev < tol, (s, ex, ev)
    assert_same_clocks(g, o)
    scale = np.abs(om["E"]).max()
    if precision == capi.FP64:
        np.testing.assert_array_equal(gm["wall_count"], om["wall_count"])
        np.testing.assert_array_equal(gm["collisions"], om["collisions"])
        np.testing.assert_allclose(gm["E"], om["E"], rtol=0, atol=1e-11 * scale)
        np.testing.assert_allclose(gm["phi"], om["phi"], rtol=0, atol=1e-11 * np.abs(om["phi"]).max())
    else:
        np.testing.assert_allclose(gm["E"], om["E"], rtol=0, atol=1e-5 * scale)


def test_smoother_changes_the_field():
    """The smoothed field is not the unsmoothed one (the filter is applied), and both
    match their own oracle runs."""
    phys = W.bounded_small(ncells=64, ppc=20, seed=3)
    loads = W.initial_load(phys, seed=3)
    _, gm0 = run_gpu(phys, loads, 1, capi.FP64)
    phys.smooth = 1
    _, gm1 = run_gpu(phys, loads, 1, capi.FP64)
    _, om1 = run_oracle(phys, loads, 1)
    assert np.abs(gm1["E"] - gm0["E"]).max() > 1e-3 * np.abs(gm0["E"]).max()
    np.testing.assert_allclose(gm1["E"], om1["E"], rtol=0, atol=1e-12 * np.abs(om1["E"]).max())


def test_smoothed_magnetized_source_fp64():
    phys = W.magnetized_source(ncells=64, ppc=40, seed=2, nu=0.2, capacity_factor=3.0)
    phys.smooth = 1
    loads = W.initial_load(phys, seed=2)
    g, gm = run_gpu(phys, loads, 60, capi.FP64, sort_interval=10)
    o, om = run_oracle(phys, loads, 60)
    np.testing.assert_array_equal(gm["collisions"], om["collisions"])
    np.testing.assert_array_equal(gm["live"], om["live"])
    for s, (ex, ev) in enumerate(particle_errors(phys, g, o)):
        assert ex < 1e-12 and ev < 1e-12, (s, ex, ev)
