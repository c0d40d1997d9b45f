"""GPU-stream-enqueued MPI communication among virtual ranks on one GB300.

The product is the C-ABI library `libmpx.so` (include/mpx.h); `mpx` is a thin
ctypes binding with the same function names.  Build with
`paper_2208_13707_gb300.build.build()`.
"""
