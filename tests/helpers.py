"""Shared helpers of the GPU parity tests: tolerances derived from the arithmetic.

Rounding model: every step forms each output amplitude with a short chain of
fused multiply-adds over one coin row; with |psi| <= 1 and a unitary coin that
adds at most ~4 units in the last place per step, and unitary propagation does
not amplify earlier errors.  So after T steps the amplitude error is bounded by
T * 4 * u, u the unit roundoff of the arithmetic (2^-24 float, 2^-53 double,
2^-44 for the double-float form, whose products keep ~2^-48).  bfloat16
storage adds one rounding of 2^-8 relative per HBM round trip.
"""
import math

import numpy as np

U = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "comp": 2.0 ** -44, "bf16": 2.0 ** -24}

# probability tolerances stated for the method: FP64 path <= 1e-12 (L1 of P);
# FP32 path <= 1e-4 L1 at T = 4096
L1_F64 = 1e-12
L1_F32 = 1e-4


def amp_tol(prec, T, k=1):
    t = max(T, 1) * 4 * U[prec] + 1e-15
    if prec == "bf16":
        t += (math.ceil(max(T, 1) / max(k, 1)) + 1) * 2.0 ** -8
    return t


def p_l1_tol(prec, T, nsites, k=1):
    if prec == "f64":
        return max(L1_F64, 4 * T * U["f64"] * 10)
    if prec == "f32":
        return L1_F32
    if prec == "comp":
        return 1e-10
    # bf16: |P - P'| <= 2|psi||d| + |d|^2 summed: 2 * sqrt(d*ns) * dmax bound (loose)
    dmax = amp_tol(prec, T, k)
    return 2 * math.sqrt(4 * nsites) * dmax + 4 * nsites * dmax * dmax


def l1(a, b):
    return float(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)).sum())


def maxabs(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max()) if np.size(a) else 0.0
