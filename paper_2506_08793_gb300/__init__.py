"""GB300 (sm_103a) CUDA implementation of the PDE-based dehazing method of
arXiv 2506.08793: dark-channel-prior front end and the fixed-point solver of
-div(D(grad u) grad u) + lambda(t) G(u) = Phi(I, t, A).

The compute lives in libdehaze.so (C ABI: include/dehaze.h); `_native` binds
it one function per entry point, `api` adds torch-tensor conveniences.
Importing this package does not load CUDA or torch.
"""
__all__ = ["api", "scenes"]
