"""GB300-native PIC Monte Carlo particle mover (arXiv 2404.10270, the BIT1 mover).

The compute path lives in a C-ABI shared library of hand-written sm_103a CUDA
kernels (``csrc/``); :mod:`.capi` is its ctypes binding and :class:`.capi.Sim` the
user-facing handle.  :mod:`.workloads` defines the seeded synthetic workloads.
"""
