"""Fourier-space closed form of a walk with one global coin on the cycle or torus.

Translation invariance makes U block-diagonal in momentum: with the DFT
psi^(k) = sum_x psi(x) e^{-2 pi i k.x/n}, a shift of coin plane c by e_c
multiplies psi^_c(k) by e^{-2 pi i k.e_c/n}, so psi^_T(k) = (D(k) C)^T psi^_0(k)
(moving shift), or (X D(k) C)^T psi^_0(k) with X swapping coins c <-> c xor 1
(flip-flop shift).  Computed with numpy's FFT and a stacked matrix power --
a method independent of stepping in real space.
"""
import numpy as np

# displacement (dx, dy) of each coin: 1D coin 0 -> -1, coin 1 -> +1;
# 2D coin 0 +x, 1 -x, 2 +y, 3 -y
DIR_1D = [(-1, 0), (1, 0)]
DIR_2D = [(1, 0), (-1, 0), (0, 1), (0, -1)]
DIR_DIAG = [(1, 1), (1, -1), (-1, 1), (-1, -1)]   # coin c = 2j+k moves ((-1)^j, (-1)^k)


def evolve_fourier(psi, coin, T, flipflop=False, diagonal=False):
    psi = np.asarray(psi, dtype=np.complex128)
    coin = np.asarray(coin, dtype=np.complex128)
    if psi.ndim == 2:
        d, N = psi.shape
        dirs = DIR_1D
        hat = np.fft.fft(psi, axis=1)                   # (d, N)
        k = np.arange(N)
        phase = np.stack([np.exp(-2j * np.pi * k * dx / N) for dx, _ in dirs])  # (d, N)
        spatial_shape = (N,)
    else:
        d, Ly, Lx = psi.shape
        dirs = DIR_DIAG if diagonal else DIR_2D
        hat = np.fft.fft2(psi, axes=(1, 2))             # (d, Ly, Lx)
        ky = np.arange(Ly)[:, None]
        kx = np.arange(Lx)[None, :]
        phase = np.stack([np.exp(-2j * np.pi * (kx * dx / Lx + ky * dy / Ly))
                          for dx, dy in dirs])         # (d, Ly, Lx)
        spatial_shape = (Ly, Lx)
    nk = int(np.prod(spatial_shape))
    ph = phase.reshape(d, nk).T                         # (nk, d)
    M = ph[:, :, None] * coin[None, :, :]               # D(k) C
    if flipflop:
        perm = [c ^ 1 for c in range(d)]
        M = M[:, perm, :]                               # X D(k) C
    MT = np.linalg.matrix_power(M, int(T))
    v = hat.reshape(d, nk).T[:, :, None]                # (nk, d, 1)
    out_hat = (MT @ v)[:, :, 0].T.reshape((d,) + spatial_shape)
    if psi.ndim == 2:
        return np.fft.ifft(out_hat, axis=1)
    return np.fft.ifft2(out_hat, axes=(1, 2))
