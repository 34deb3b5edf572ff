"""GB300 (sm_103a) Z4c right-hand side + RK4 over a pack of MeshBlocks.

The compute path is the CUDA library libz4c_gb300.so (C ABI in
include/z4c.h); ``paper_2409_10383_gb300.z4c`` is a thin ctypes binding with
the same function names.  PyTorch only provides device memory and streams.
"""
__all__ = ["z4c", "inputs"]
