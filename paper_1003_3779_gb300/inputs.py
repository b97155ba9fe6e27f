"""Seeded synthetic inputs for the quantum-walk workloads.

This module holds no arithmetic of the walk itself: it only draws seeded random
numbers and writes down the named coin matrices and initial states that are the
*inputs* of a walk.  Both the CUDA path and the CPU oracle receive the same
arrays from here.

Layout of a state: ``d`` coin-major planes, numpy shape ``(2, N)`` on the cycle
and ``(4, L, L)`` on the torus (row ``y``, column ``x``).  Directions (the coin
basis): 1D coin 0 -> x-1, coin 1 -> x+1; 2D coin 0 +x, 1 -x, 2 +y, 3 -y.

Workloads (sizes and distributions follow the paper's lattices, Sec. 2.2/3, and
the scenarios the library is built for):

* ``hadamard_1d``      cycle N=2001, Hadamard coin, |0>(x)(|0>+i|1>)/sqrt2, T=1000
* ``su2_1d``           cycle N=2^27, SU(2) coin theta=pi/4, random state (seed 1), T=4096
* ``torus_2d``         8192^2 torus, Grover or H(x)H, moving or flip-flop, T=1024
* ``batch_1d``         4096 walks, N~U[256,65536], T~U[64,4096], theta~U[0,pi/2]
* ``region_grad_2d``   1024^2 torus, Grover.diag(e^{i phi}), phi~U[-0.1,0.1], T=512
* graphs (Sec. 2.1)    a random 4-regular graph (configuration model, 2^26
                       vertices), the 8192^2 torus as a graph, and a power-law
                       (Chung-Lu) graph with skewed degrees; Grover coin

A graph walk's state is one amplitude per arc (vertex, edge end) in the arc
form: the arcs of vertex v are off[v] .. off[v+1]-1 and partner[a] is the arc at
the other end of a's edge.
"""
from __future__ import annotations

import math

import numpy as np

SQ2 = math.sqrt(2.0)


# ---------------------------------------------------------------- coins
def hadamard() -> np.ndarray:
    """H = (1/sqrt2) [[1, 1], [1, -1]] (the default coin of Sec. 3)."""
    return np.array([[1, 1], [1, -1]], dtype=np.complex128) / SQ2


def su2(theta: float, xi: float = 0.0, zeta: float = 0.0) -> np.ndarray:
    """C = [[e^{i xi} cos t, e^{i zeta} sin t], [-e^{-i zeta} sin t, e^{-i xi} cos t]]."""
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[np.exp(1j * xi) * c, np.exp(1j * zeta) * s],
                     [-np.exp(-1j * zeta) * s, np.exp(-1j * xi) * c]], dtype=np.complex128)


def grover(d: int = 4) -> np.ndarray:
    """Grover coin G = (2/d) J - I (Sec. 3 names it)."""
    return (2.0 / d) * np.ones((d, d), dtype=np.complex128) - np.eye(d, dtype=np.complex128)


def hadamard2() -> np.ndarray:
    """H (x) H on the two coin qubits, coin index c = 2 j + k (Sec. 3 state)."""
    return np.kron(hadamard(), hadamard())


def fourier(d: int = 4) -> np.ndarray:
    """Fourier coin F[j, k] = w^{jk} / sqrt(d), w = e^{2 pi i / d} (Sec. 3 names it)."""
    j = np.arange(d)
    return np.exp(2j * np.pi * np.outer(j, j) / d) / math.sqrt(d)


def random_unitary(d: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-like random unitary (QR of a complex Gaussian matrix, phases fixed)."""
    z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


# ---------------------------------------------------------------- states
def localized_1d(N: int, x0: int = 0, coin_state=(1 / SQ2, 1j / SQ2)) -> np.ndarray:
    psi = np.zeros((2, N), dtype=np.complex128)
    psi[0, x0] = coin_state[0]
    psi[1, x0] = coin_state[1]
    return psi


GROVER_SPREAD_STATE = (0.5, -0.5, -0.5, 0.5)


def localized_2d(L: int, x0: int = 0, y0: int = 0, coin_state=GROVER_SPREAD_STATE,
                 Ly: int | None = None) -> np.ndarray:
    Ly = L if Ly is None else Ly
    psi = np.zeros((4, Ly, L), dtype=np.complex128)
    for c in range(4):
        psi[c, y0, x0] = coin_state[c]
    return psi


def random_state(shape, seed: int, dtype=np.complex128) -> np.ndarray:
    """i.i.d. complex Gaussian amplitudes (re, im standard normal, PCG64(seed)),
    divided by their FP64 norm.  ``shape`` is the plane shape with the coin axis
    first, e.g. (2, N) or (4, L, L).  With dtype complex64 the normals are drawn
    in float32 and the normalised values rounded once to float32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(np.prod(shape))
    if np.dtype(dtype) == np.complex64:
        raw = rng.standard_normal(2 * n, dtype=np.float32)
        ss = 0.0
        step = 1 << 24
        for i in range(0, raw.size, step):
            blk = raw[i:i + step].astype(np.float64)
            ss += float(np.dot(blk, blk))
        scale = 1.0 / math.sqrt(ss)
        out = np.empty(n, dtype=np.complex64)
        ov = out.view(np.float32)
        for i in range(0, raw.size, step):
            ov[i:i + step] = (raw[i:i + step].astype(np.float64) * scale).astype(np.float32)
        return out.reshape(shape)
    re = rng.standard_normal(n)
    im = rng.standard_normal(n)
    z = re + 1j * im
    z /= math.sqrt(float(np.sum(re * re) + np.sum(im * im)))
    return z.reshape(shape)


# ---------------------------------------------------------------- workloads
def batch_1d_params(nwalks: int = 4096, seed: int = 3, n_lo: int = 256, n_hi: int = 65536,
                    t_lo: int = 64, t_hi: int = 4096):
    """Per-walk (N, T, theta, x0) for the batched workload: N~U[n_lo,n_hi],
    T~U[t_lo,t_hi] (integers, inclusive), theta~U[0,pi/2], x0~U[0,N)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = rng.integers(n_lo, n_hi + 1, size=nwalks, dtype=np.int64)
    T = rng.integers(t_lo, t_hi + 1, size=nwalks, dtype=np.int64)
    theta = rng.uniform(0.0, math.pi / 2, size=nwalks)
    x0 = (rng.uniform(0.0, 1.0, size=nwalks) * N).astype(np.int64)
    x0 = np.minimum(x0, N - 1)
    return N, T, theta, x0


BATCH_COIN_STATE = (1 / SQ2, 1j / SQ2)


def region_grad_phases(L: int = 1024, seed: int = 4, amp: float = 0.1) -> np.ndarray:
    """phi_{v,k} ~ U[-amp, amp], shape (L, L, 4) (site-major, 4 reals per site)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-amp, amp, size=(L, L, 4))


def region_rect(L: int = 1024, centre=(256, 256), size: int = 64):
    """(x0, y0, w, h) of the size x size square centred at ``centre``."""
    return (centre[0] - size // 2, centre[1] - size // 2, size, size)


# ---------------------------------------------------------------- graphs
def random_regular_arcs(nvert: int, degree: int, seed: int):
    """Arc form (off, partner) of a random degree-regular multigraph by the
    configuration model: vertex v owns arcs v*degree .. v*degree+degree-1 (its
    edge ends), and a uniformly random perfect matching pairs all arcs into
    edges (loops and parallel edges are kept).  nvert*degree must be even."""
    A = int(nvert) * int(degree)
    if A % 2:
        raise ValueError("nvert * degree must be even")
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = rng.permutation(A).astype(np.int64)
    partner = np.empty(A, dtype=np.int64)
    partner[perm[0::2]] = perm[1::2]
    partner[perm[1::2]] = perm[0::2]
    off = np.arange(0, A + 1, degree, dtype=np.int64)
    return off, partner


def lattice_graph_arcs(Lx: int, Ly: int | None = None):
    """The cycle Z_Lx (Ly None) or the torus Z_Lx x Z_Ly as a graph in arc form,
    with the lattice's coin slots as arc slots: on the cycle vertex x has slot 0
    (edge to x-1) and slot 1 (edge to x+1); on the torus vertex y*Lx + x has
    slots +x, -x, +y, -y.  The graph walk on it is the flip-flop lattice walk."""
    if Ly is None:
        x = np.arange(Lx, dtype=np.int64)
        partner = np.empty(2 * Lx, dtype=np.int64)
        partner[2 * x] = 2 * ((x - 1) % Lx) + 1
        partner[2 * x + 1] = 2 * ((x + 1) % Lx)
        return np.arange(0, 2 * Lx + 1, 2, dtype=np.int64), partner
    y, x = np.divmod(np.arange(Lx * Ly, dtype=np.int64), Lx)
    right, left = y * Lx + (x + 1) % Lx, y * Lx + (x - 1) % Lx
    up, down = ((y + 1) % Ly) * Lx + x, ((y - 1) % Ly) * Lx + x
    v = y * Lx + x
    partner = np.empty(4 * Lx * Ly, dtype=np.int64)
    partner[4 * v] = 4 * right + 1
    partner[4 * v + 1] = 4 * left
    partner[4 * v + 2] = 4 * up + 3
    partner[4 * v + 3] = 4 * down + 2
    return np.arange(0, 4 * Lx * Ly + 1, 4, dtype=np.int64), partner


def chung_lu_edges(nvert: int, mean_degree: float, exponent: float, seed: int) -> np.ndarray:
    """Edge list (nedges, 2) of a Chung-Lu graph with power-law expected
    degrees: vertex v has weight (v + 1)^(-1/(exponent - 1)); nvert*mean_degree/2
    edges, each joining two vertices drawn in proportion to their weights
    (loops, parallel edges and isolated vertices are kept)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = (np.arange(nvert, dtype=np.float64) + 1.0) ** (-1.0 / (exponent - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    m = int(round(nvert * mean_degree / 2))
    ends = np.searchsorted(cdf, rng.uniform(0.0, 1.0, size=2 * m), side="right")
    return np.minimum(ends, nvert - 1).astype(np.int64).reshape(m, 2)
