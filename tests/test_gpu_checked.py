"""The bounds-checked device build (-DPIC_CHECKED) on GPU workloads.

In that build every index a kernel computes into a particle store, a node array, a
queue or a staging buffer is checked, and a refusal latches a status bit that the next
synchronising call reports.  The normal workloads (the 256-cell plasma in both forms,
the magnetized source with ionization, subcycling, the y drift, the separate sort and
the paper's neutral-target case) must run through it without a single refusal and give
the normal build's results bit for bit; its self-probe shows that a refusal is latched.
Each library runs in a subprocess of its own (a process loads one of them).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.gpu_common import requires_gpu
from tests.helpers import ROOT

pytestmark = [pytest.mark.gpu, requires_gpu]


def _run(lib, out):
    env = dict(os.environ, BITPIC_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "tests.checked_run", str(out)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return dict(np.load(out))


def test_checked_build_refuses_nothing_and_changes_nothing(tmp_path):
    from paper_2404_10270_gb300 import build
    normal = build.build()
    checked = build.build(checked=True)
    a = _run(checked, tmp_path / "checked.npz")
    b = _run(normal, tmp_path / "normal.npz")
    assert int(a.pop("probe")) == 0      # the check refuses an index past its range
    assert int(b.pop("probe")) == -1     # the normal build has no checks
    assert set(a) == set(b)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
