import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Plain FP32 steps of large batches move particles with a pair of mover variants (the
# one that leaves collision-clock draws to the event kernel, and the one with the draw
# inline on the common test steps).  The tests' batches are small: let them take that
# path too, so the parity checks cover the code the large workloads run.
os.environ.setdefault("BITPIC_PAIR_MIN_SLOTS", "0")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running")
