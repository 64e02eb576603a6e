"""GB300-native engine for weighted Gerchberg-Saxton (GSW) holograms by direct superposition.

Importing the package is cheap: the CUDA library is loaded by ``paper_0907_4027_gb300.hot``
(the ctypes binding of the C ABI declared in ``include/hot.h``), which raises if the
library has not been built.  ``paper_0907_4027_gb300.workloads`` holds the seeded synthetic
input generators and no arithmetic of the method; ``autograd`` wraps the forward field and its
adjoint in a ``torch.autograd.Function``; ``sharded`` holds the multi-GPU drivers (replicas and
row bands).
"""
__all__ = ["hot", "workloads", "autograd", "sharded"]
