"""GB300 (sm_103a) CheFSI hot path for real-space Kohn-Sham DFT (arXiv 2303.00790).

The compute lives in libkscf.so (C ABI in include/kscf.h, CUDA kernels in csrc/);
`paper_2303_00790_gb300.kscf` is its ctypes binding.  Build with
`paper_2303_00790_gb300.build.build()`.
"""
__all__ = ["kscf", "build"]
