"""GES (Gaussian-enhanced Surfels) renderer for GB300 (sm_103a).

The CUDA library ``libges.so`` implements the two-pass render of Sec. 3
(surfel z-buffer, depth-tested sorting-free Gaussian accumulation, Eq. 5
composite), its backward pass for the joint optimisation stage (Sec. 4.2) and
batched multi-view rendering, behind the C ABI of ``include/ges.h``.
``native`` is the ctypes binding with the ABI's names; ``render`` (imported
on demand: ``from paper_2504_17545_gb300 import render``) is the thin PyTorch
layer (device memory, streams, autograd).
"""
from . import build, native  # noqa: F401

__all__ = ["build", "native"]
