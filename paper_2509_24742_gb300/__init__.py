"""GB300-native SRBE (symmetry-preserving random batch Ewald) for constant-potential slabs.

The compute path lives in libsrbe.so (hand-written CUDA for sm_103a behind the C ABI of
include/srbe.h); `srbe` is its thin binding and `workloads` makes seeded synthetic inputs.
"""
from . import build, workloads  # noqa: F401

__all__ = ["build", "workloads", "srbe"]
