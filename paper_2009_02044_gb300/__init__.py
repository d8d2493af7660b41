"""GB300 library for the laboratory-frame 3+1D Glasma time step with CPIC
charges (Mueller & Ipp, arXiv:2009.02044).

The compute path is the C ABI of include/glasma.h, implemented by the CUDA
kernels under csrc/ and built into _lib/libglasma.so; the submodule
`glasma` is its ctypes binding and `build` compiles it.
"""
