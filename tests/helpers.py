"""Small helpers shared by the tests (no method arithmetic)."""
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def read_kat(name="philox4x32_10_kat.txt"):
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def positions(parts, dx):
    """Physical positions x = (j + f) dx of a particle dict."""
    return (parts["cell"].astype(np.float64) + parts["off"]) * dx
