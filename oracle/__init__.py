"""FP64 CPU oracle for the coined quantum walk (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
and reference arms may import this package.  It shares no code with the CUDA
library: the arithmetic lives in ``qw_oracle.c`` (plain C99, FP64,
``-ffp-contract=off``), written from the definitions of Sawerwain & Gielerak,
arXiv:1003.3779, Sec. 2.1 (U = S(I (x) C), S|v,e> = |v',e>), Sec. 2.2 (the Z^1 and
Z^2 walks) and Sec. 3 (two-qubit coin, shift operator, broken links).

State layout everywhere: ``d`` coin-major planes of ``nsites`` complex numbers,
as a numpy complex128 array of shape ``(d, nsites)`` (1D) or ``(d, Ly, Lx)`` (2D).

Every function here is pinned by tests that do not call it to check itself
(exact Gaussian-integer arithmetic, a Fourier-space closed form, the dense
unitary built explicitly, invariants) -- see ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBS: dict = {}
_LOCK = threading.Lock()

BC_PERIODIC, BC_SEGMENT, BC_LINE = 0, 1, 2
SHIFT_MOVING, SHIFT_FLIPFLOP, SHIFT_DIAGONAL = 0, 1, 2


def build(openmp: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` and return the path."""
    os.makedirs(_BUILD, exist_ok=True)
    name = "liboracle_omp.so" if openmp else "liboracle.so"
    out = os.path.join(_BUILD, name)
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", out + ".tmp", "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def _lib(openmp: bool = False):
    with _LOCK:
        if openmp not in _LIBS:
            lib = ctypes.CDLL(build(openmp))
            P = ctypes.c_void_p
            lib.oracle_evolve.argtypes = [ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P,
                                          ctypes.c_int, ctypes.c_int, P, P, P,
                                          ctypes.c_int64, ctypes.c_int, P]
            lib.oracle_probabilities.argtypes = [ctypes.c_int, P, P, P, P]
            lib.oracle_region_grad.argtypes = [P, ctypes.c_int, P, P, P, ctypes.c_int64,
                                               P, P, P]
            lib.oracle_num_threads.argtypes = []
            lib.oracle_philox4x32_10.argtypes = [P, P, P]
            lib.oracle_philox4x32_10.restype = None
            lib.oracle_link_masks.argtypes = [ctypes.c_int, P, ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.c_int64, ctypes.c_int64, P]
            lib.oracle_graph_arcs.argtypes = [ctypes.c_int64, ctypes.c_int64, P, P, P]
            lib.oracle_graph_evolve.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, P, P,
                                                ctypes.c_int64, ctypes.c_int, P]
            lib.oracle_graph_probabilities.argtypes = [ctypes.c_int64, P, P, P, P]
            _LIBS[openmp] = lib
        return _LIBS[openmp]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _dims(psi):
    psi = np.asarray(psi)
    if psi.ndim == 2:
        return 1, np.array([psi.shape[1]], dtype=np.int64)
    if psi.ndim == 3:
        return 2, np.array([psi.shape[2], psi.shape[1]], dtype=np.int64)
    raise ValueError("state must have shape (2, N) or (4, Ly, Lx)")


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"{what} failed with status {st}")


def num_threads(openmp: bool = False) -> int:
    return int(_lib(openmp).oracle_num_threads())


def evolve(psi, coin, T, *, shift=SHIFT_MOVING, bc=BC_PERIODIC, coin_mode=None,
           phi=None, closed=None, closed_per_step=False, adjoint=False,
           openmp=False):
    """Return U^T psi (or (U^dagger)^T psi).

    coin: (d, d) complex for one global coin; (nsites, d, d) for one matrix per
    site; with ``phi`` (nsites, d) real, the per-site coin is coin . diag(e^{i phi}).
    closed: optional uint8 link flags, shape (ndim, nsites) or (T, ndim, nsites).
    """
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    ndim, dims = _dims(psi)
    d = 2 * ndim
    if psi.shape[0] != d:
        raise ValueError("coin dimension must be 2 in 1D and 4 in 2D")
    nsites = int(np.prod(dims))
    coin = np.ascontiguousarray(coin, dtype=np.complex128)
    if coin_mode is None:
        coin_mode = 2 if phi is not None else (1 if coin.ndim == 3 else 0)
    if coin_mode in (0, 2) and coin.shape != (d, d):
        raise ValueError("global/base coin must be d x d")
    if coin_mode == 1 and coin.shape != (nsites, d, d):
        raise ValueError("per-site coins must be (nsites, d, d)")
    phi_a = None
    if coin_mode == 2:
        phi_a = np.ascontiguousarray(phi, dtype=np.float64).reshape(nsites, d)
    cl = None
    if closed is not None:
        cl = np.ascontiguousarray(closed, dtype=np.uint8)
        want = (int(T), ndim, nsites) if closed_per_step else (ndim, nsites)
        if cl.size != int(np.prod(want)):
            raise ValueError(f"closed mask must have {want} entries")
    out = np.empty_like(psi)
    st = _lib(openmp).oracle_evolve(ndim, _ptr(dims), int(shift), int(bc), _ptr(cl),
                                    int(bool(closed_per_step)), int(coin_mode),
                                    _ptr(coin), _ptr(phi_a), _ptr(psi), int(T),
                                    int(bool(adjoint)), _ptr(out))
    _check(st, "oracle_evolve")
    return out


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon et al., SC 2011): four 32-bit words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    _lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def link_threshold(p):
    """The 32-bit threshold of closing probability p (a link closes when a
    Philox word is below it)."""
    return min(int(p * 4294967296.0), 4294967295)


def link_masks(plane_shape, seed, p, t0, T):
    """Closed-link masks of steps t0 .. t0+T-1 (Sec. 3, links broken at random at
    every step): uint8 array (T, ndim, nsites) for evolve(..., closed_per_step=True)."""
    shape = tuple(int(x) for x in plane_shape)
    ndim = len(shape)
    dims = np.array(shape[::-1], dtype=np.int64)   # (nx,) or (nx, ny)
    ns = int(np.prod(shape))
    out = np.empty((int(T), ndim, ns), dtype=np.uint8)
    st = _lib().oracle_link_masks(ndim, _ptr(dims), int(seed), link_threshold(p), int(t0), int(T), _ptr(out))
    _check(st, "oracle_link_masks")
    return out


def probabilities(psi, openmp=False):
    """Return (P, norm): P(v) = sum_c |psi(v,c)|^2 shaped like one plane."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    ndim, dims = _dims(psi)
    P = np.empty(psi.shape[1:], dtype=np.float64)
    norm = ctypes.c_double(0.0)
    st = _lib(openmp).oracle_probabilities(ndim, _ptr(dims), _ptr(psi), _ptr(P),
                                           ctypes.cast(ctypes.pointer(norm), ctypes.c_void_p))
    _check(st, "oracle_probabilities")
    return P, norm.value


def region_grad(psi0, base, phi, T, rect, *, shift=SHIFT_MOVING, openmp=False):
    """Loss and gradient of the mass in rect=(x0, y0, w, h) after T steps
    (2D torus, C_v = base . diag(e^{i phi_v})).  Returns (loss, grad (Ly, Lx, 4))."""
    psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
    ndim, dims = _dims(psi0)
    if ndim != 2:
        raise ValueError("region_grad is defined on the 2D torus")
    nsites = int(np.prod(dims))
    base = np.ascontiguousarray(base, dtype=np.complex128)
    phi_a = np.ascontiguousarray(phi, dtype=np.float64).reshape(nsites, 4)
    r = np.ascontiguousarray(rect, dtype=np.int64)
    grad = np.empty((nsites, 4), dtype=np.float64)
    loss = ctypes.c_double(0.0)
    st = _lib(openmp).oracle_region_grad(_ptr(dims), int(shift), _ptr(base), _ptr(phi_a),
                                         _ptr(psi0), int(T), _ptr(r),
                                         ctypes.cast(ctypes.pointer(loss), ctypes.c_void_p),
                                         _ptr(grad))
    _check(st, "oracle_region_grad")
    return loss.value, grad.reshape(int(dims[1]), int(dims[0]), 4)


GRAPH_COIN_GROVER, GRAPH_COIN_PER_VERTEX = 0, 1


def graph_arcs(nvert, edges):
    """Arc form (off, partner) of a graph given as an edge list (Sec. 2.1): the
    arcs of vertex v are off[v] .. off[v+1]-1, in the order the vertex's edge
    ends appear in the list; partner[a] is the arc at the other end of a's edge."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int64).reshape(-1, 2))
    off = np.empty(int(nvert) + 1, dtype=np.int64)
    partner = np.empty(2 * len(e), dtype=np.int64)
    st = _lib().oracle_graph_arcs(int(nvert), len(e), _ptr(e), _ptr(off), _ptr(partner))
    _check(st, "oracle_graph_arcs")
    return off, partner


def graph_evolve(off, partner, psi, T, *, coins=None, adjoint=False, openmp=False):
    """U^T psi (or (U^dagger)^T psi) for the walk on a general graph in arc form
    (Sec. 2.1, U = S (I (x) C), S|v,e> = |v',e>).  coins None: the Grover coin
    (2/d) J - I at every vertex; else a list of per-vertex d(v) x d(v) matrices,
    or one d x d matrix for a d-regular graph."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    partner = np.ascontiguousarray(partner, dtype=np.int64)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    nvert = len(off) - 1
    if psi.shape != (int(off[-1]),):
        raise ValueError("psi must hold one amplitude per arc")
    mode, flat = GRAPH_COIN_GROVER, None
    if coins is not None:
        mode = GRAPH_COIN_PER_VERTEX
        deg = np.diff(off)
        if isinstance(coins, np.ndarray) and coins.ndim == 2:
            if np.any(deg != coins.shape[0]):
                raise ValueError("one matrix for all vertices needs a regular graph of that degree")
            flat = np.ascontiguousarray(np.tile(coins.astype(np.complex128).ravel(), nvert))
        else:
            parts = [np.asarray(c, dtype=np.complex128).ravel() for c in coins]
            if len(parts) != nvert or any(p.size != d * d for p, d in zip(parts, deg)):
                raise ValueError("one d(v) x d(v) matrix per vertex")
            flat = np.ascontiguousarray(np.concatenate(parts) if parts else np.zeros(0, complex))
    out = np.empty_like(psi)
    st = _lib(openmp).oracle_graph_evolve(nvert, _ptr(off), _ptr(partner), mode, _ptr(flat),
                                          _ptr(psi), int(T), int(bool(adjoint)), _ptr(out))
    _check(st, "oracle_graph_evolve")
    return out


def graph_probabilities(off, psi):
    """Return (P, norm): P(v) = sum over the arcs of v of |psi(a)|^2."""
    off = np.ascontiguousarray(off, dtype=np.int64)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    P = np.empty(len(off) - 1, dtype=np.float64)
    norm = ctypes.c_double(0.0)
    st = _lib().oracle_graph_probabilities(len(off) - 1, _ptr(off), _ptr(psi), _ptr(P),
                                           ctypes.cast(ctypes.pointer(norm), ctypes.c_void_p))
    _check(st, "oracle_graph_probabilities")
    return P, norm.value
