"""Exact Gaussian-integer Hadamard walk on a cycle.

With H = (1/sqrt2)[[1, 1], [1, -1]] and psi_0 = |x0> (x) (|0> + i|1>)/sqrt2, every
amplitude after t steps is a Gaussian integer divided by 2^{(t+1)/2}.  This
module carries the Gaussian integers a_t exactly (Python big integers in numpy
object arrays): a step adds/subtracts the two coin components (H without its
1/sqrt2) and moves coin 0 to x-1 and coin 1 to x+1 (periodic), per the 1D walk
of Sec. 2.2 with U = S (I (x) C) of Sec. 2.1.  P_T(x) = (|a0|^2 + |a1|^2) / 2^{T+1}.
"""
from fractions import Fraction

import numpy as np


def hadamard_walk_exact(N: int, T: int, x0: int = 0):
    """Return (re0, im0, re1, im1) Gaussian-integer planes after T steps."""
    z = np.zeros(N, dtype=object)
    z[:] = 0
    re0, im0, re1, im1 = z.copy(), z.copy(), z.copy(), z.copy()
    re0[x0] = 1          # coin 0 amplitude 1
    im1[x0] = 1          # coin 1 amplitude i
    for _ in range(T):
        p_re0, p_im0 = re0 + re1, im0 + im1      # H row 0 (unnormalised)
        p_re1, p_im1 = re0 - re1, im0 - im1      # H row 1
        # coin 0 moves x -> x-1: new[x] = phi[x+1]; coin 1 moves x -> x+1
        re0, im0 = np.roll(p_re0, -1), np.roll(p_im0, -1)
        re1, im1 = np.roll(p_re1, 1), np.roll(p_im1, 1)
    return re0, im0, re1, im1


def exact_probabilities(N: int, T: int, x0: int = 0):
    """Integer numerators num[x] with P_T(x) = num[x] / 2^{T+1}, and the denominator."""
    re0, im0, re1, im1 = hadamard_walk_exact(N, T, x0)
    num = re0 * re0 + im0 * im0 + re1 * re1 + im1 * im1
    return num, 1 << (T + 1)


def as_float(num, den):
    return np.array([float(Fraction(int(n), den)) for n in num])


def exact_state(N: int, T: int, x0: int = 0):
    """The state as complex128 (each amplitude correctly rounded per component)."""
    re0, im0, re1, im1 = hadamard_walk_exact(N, T, x0)
    scale = 2.0 ** (-(T + 1) / 2.0)
    # exact only when (T+1) is even; otherwise one rounding of sqrt(2) enters
    out = np.empty((2, N), dtype=np.complex128)
    for c, (r, i) in enumerate(((re0, im0), (re1, im1))):
        out[c] = np.array([complex(float(int(a)) * scale, float(int(b)) * scale)
                           for a, b in zip(r, i)])
    return out
