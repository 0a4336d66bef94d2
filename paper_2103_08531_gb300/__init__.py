"""GB300-native free-space Poisson solver: Hockney-Eastwood and Vico-Greengard-Ferrando.

The solve is a zero-padded FFT convolution computed by hand-written CUDA kernels
for sm_103a in libfsp.so (C ABI in include/fsp.h); this package only marshals
torch tensors into that ABI.  See Plan, FspSolve, Batch and solve_batched.
"""
from ._lib import FspError, load  # noqa: F401
from .solver import Batch, FspSolve, HostPipeline, Plan, solve, solve_batched, tuned_variant  # noqa: F401

__all__ = ["Plan", "FspSolve", "Batch", "HostPipeline", "solve", "solve_batched", "tuned_variant", "FspError", "load"]
