"""GB300-native two-level Schwarz / H_k-GenEO / FGMRES solver for the indefinite
Helmholtz problem (arXiv 2406.06283).

The compute path is the CUDA library `libhkgeneo.so` (C ABI, header
`include/hkgeneo.h`); `paper_2406_06283_gb300.hk` is its thin ctypes binding.
`paper_2406_06283_gb300.workloads` generates the seeded synthetic inputs.
Importing the package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""
__all__ = ["hk", "workloads"]
