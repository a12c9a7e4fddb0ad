"""GB300 (sm_103a) implementation of the per-time-step hot path of the combined multi-phase-field /
lattice-Boltzmann method for capillary-driven particle motion (arXiv:1902.10432).

The compute lives in the CUDA library ``_lib/libcbl.so`` behind the C ABI of ``include/cbl.h``;
``cbl`` is its ctypes binding and ``workloads`` builds the seeded synthetic inputs.
"""
from . import cbl  # noqa: F401
