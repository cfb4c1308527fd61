"""GB300-native semi-Lagrangian level-set surface reconstruction.

Implements the hot path of Preda & Semplice, "Surface reconstruction from
point cloud using a semi-Lagrangian scheme with local interpolator" (arXiv
2410.22205) as hand-written sm_103a CUDA kernels behind the C ABI of
include/slr.h (libslr.so). ``slr`` is the Python binding (argument
marshalling only; it also wraps the batched form, slr_batch_evolve, and the
served form, slr_server_*), ``synth`` the seeded synthetic inputs and
``build`` the nvcc build of the library. Importing the package loads
nothing; the CUDA library is loaded on first use and its absence is an
error.
"""
__all__ = ["slr", "synth"]
