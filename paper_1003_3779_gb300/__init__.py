"""GB300-native discrete-time coined quantum walk (Sawerwain & Gielerak,
arXiv:1003.3779): the step U = S (I (x) C) on the cycle and the torus, its
marginal probabilities, batched walks and the adjoint gradient, computed by
hand-written sm_103a CUDA kernels behind the C ABI declared in ``include/qw.h``.

Importing the package does not load the CUDA library; ``paper_1003_3779_gb300.qw``
loads it on first use and raises if it is missing (there is no CPU fallback).
"""
__all__ = ["qw", "inputs"]
