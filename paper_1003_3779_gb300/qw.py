"""Python binding of the C ABI in ``include/qw.h`` (argument marshalling only).

Every function named ``qw_*`` here calls the library function of the same name
through ctypes; the classes ``Walk`` and ``Batch`` and the autograd Function
``RegionMass`` only hold handles and pass ``tensor.data_ptr()`` and the current
torch CUDA stream.  All arithmetic of the walk runs in the library's kernels;
there is no CPU fallback: if ``libqw.so`` is missing, loading raises.

The walk (Sawerwain & Gielerak, arXiv:1003.3779, Sec. 2.1): one step is
U = S (I (x) C) on the cycle (coin dim 2) or torus (coin dim 4).
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libqw.so")

QW_OK, QW_EINVAL, QW_ENOMEM, QW_ECUDA, QW_ESTATE, QW_ETIMEOUT, QW_EUNSUPPORTED = range(7)
BC_PERIODIC, BC_SEGMENT, BC_LINE = 0, 1, 2
SHIFT_MOVING, SHIFT_FLIPFLOP, SHIFT_DIAGONAL = 0, 1, 2
F64, F32, F32_BF16STORE, F32_COMP = 0, 1, 2, 3
C128, C64 = 0, 1
R64, R32 = 0, 1

PRECISIONS = {"f64": F64, "f32": F32, "bf16": F32_BF16STORE, "comp": F32_COMP}

_lib = None


class QWError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


def lib():
    """Load libqw.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libqw.so not found at {LIB_PATH}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    P, I, I64, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "qw_create": (I, [I, P, I, I, I, I, P, P]),
        "qw_destroy": (I, [P]),
        "qw_set_coin": (I, [P, P, I, I]),
        "qw_set_coin_phases": (I, [P, P, P, I]),
        "qw_set_links": (I, [P, P, I]),
        "qw_set_link_noise": (I, [P, ctypes.c_double, ctypes.c_uint64, I64]),
        "qw_run_host_batch": (I, [P, I, P, I64, I, I64, P, I64, I, P]),
        "qw_get_link_step": (I, [P, P]),
        "qw_set_state": (I, [P, P, I, I]),
        "qw_get_state": (I, [P, P, I, I]),
        "qw_step": (I, [P, I64]),
        "qw_step_adjoint": (I, [P, I64]),
        "qw_probabilities": (I, [P, P, I, I, P]),
        "qw_set_plan": (I, [P, I, I]),
        "qw_get_plan": (I, [P, P, P]),
        "qw_set_plan_ex": (I, [P, I, I, I]),
        "qw_get_plan_ex": (I, [P, P, P, P]),
        "qw_autotune": (I, [P, ctypes.c_char_p, S]),
        "qw_nsites": (I64, [P]),
        "qw_describe": (I, [P, ctypes.c_char_p, S]),
        "qw_set_clipping": (I, [P, I]),
        "qw_synchronize": (I, [P]),
        "qw_backward": (I, [P, P, I64, I64, P, P, I]),
        "qw_batch_create": (I, [I, P, P, P, P, P, I, P, P]),
        "qw_batch_step": (I, [P]),
        "qw_batch_probabilities": (I, [P, P, I, P]),
        "qw_batch_get_state": (I, [P, I, P, I]),
        "qw_batch_destroy": (I, [P]),
        "qw_batch_set_plan": (I, [P, I]),
        "qw_batch_get_plan": (I, [P, P, P]),
        "qw_batch_autotune": (I, [P, ctypes.c_char_p, S]),
        "qw_batch_set_plan_ex": (I, [P, I, I]),
        "qw_batch_set_cta_walks": (I, [P, I]),
        "qw_batch_cta_walks": (I, [P]),
        "qw_batch_get_plan_ex": (I, [P, P, P, P]),
        "qw_graph_arcs": (I, [I64, I64, P, P, P]),
        "qw_gwalk_create": (I, [I64, P, P, I, P, P]),
        "qw_gwalk_destroy": (I, [P]),
        "qw_gwalk_set_coin": (I, [P, I, P, I]),
        "qw_gwalk_set_state": (I, [P, P, I, I]),
        "qw_gwalk_get_state": (I, [P, P, I, I]),
        "qw_gwalk_step": (I, [P, I64]),
        "qw_gwalk_step_adjoint": (I, [P, I64]),
        "qw_gwalk_probabilities": (I, [P, P, I, I, P]),
        "qw_gwalk_set_variant": (I, [P, I]),
        "qw_gwalk_get_variant": (I, [P, P]),
        "qw_gwalk_set_window": (I, [P, S]),
        "qw_gwalk_autotune": (I, [P, ctypes.c_char_p, S]),
        "qw_gwalk_synchronize": (I, [P]),
        "qw_gwalk_narcs": (I64, [P]),
        "qw_gwalk_last_error": (ctypes.c_char_p, [P]),
        "qw_status_string": (ctypes.c_char_p, [I]),
        "qw_last_error": (ctypes.c_char_p, [P]),
        "qw_batch_last_error": (ctypes.c_char_p, [P]),
        "qw_version": (ctypes.c_char_p, []),
        "qw_debug_bounded_wait": (I, [I64, P]),
        "qw_probabilities_noalloc": (I, [P, I, I, I64, P, I, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def declared_symbols():
    """Entry points the binding expects (matches include/qw.h)."""
    lib()
    return sorted(n for n in dir(_lib) if n.startswith("qw_"))


def _check(st, handle=None, batch=False):
    if st == QW_OK:
        return
    L = lib()
    msg = L.qw_status_string(st).decode()
    if handle is not None:
        err = {False: L.qw_last_error, True: L.qw_batch_last_error, "graph": L.qw_gwalk_last_error}[batch]
        detail = err(handle).decode()
        if detail:
            msg = f"{msg}: {detail}"
    raise QWError(st, msg)


def _ptr(x):
    """Pointer of a numpy array or torch tensor (or None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(x.data_ptr())


def _on_device(x):
    return 0 if isinstance(x, np.ndarray) else int(x.is_cuda)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ---------------------------------------------------------------- raw ABI
def qw_version():
    return lib().qw_version().decode()


def qw_create(ndim, dims, coin_dim, bc=BC_PERIODIC, shift=SHIFT_MOVING, prec=F32, stream=None):
    d = np.ascontiguousarray(dims, dtype=np.int64)
    h = ctypes.c_void_p()
    st = lib().qw_create(int(ndim), _ptr(d), int(coin_dim), int(bc), int(shift), int(prec),
                         stream if stream is not None else _stream(), ctypes.byref(h))
    _check(st)
    return h


def qw_destroy(h):
    _check(lib().qw_destroy(h))


def qw_set_coin(h, coin, per_site=False):
    if isinstance(coin, np.ndarray):
        coin = np.ascontiguousarray(coin, dtype=np.complex128)
    _check(lib().qw_set_coin(h, _ptr(coin), int(per_site), _on_device(coin)), h)


def qw_set_coin_phases(h, base, phi):
    base = np.ascontiguousarray(base, dtype=np.complex128)
    if isinstance(phi, np.ndarray):
        phi = np.ascontiguousarray(phi, dtype=np.float32)
    _check(lib().qw_set_coin_phases(h, _ptr(base), _ptr(phi), _on_device(phi)), h)


def qw_set_links(h, closed):
    if isinstance(closed, np.ndarray):
        closed = np.ascontiguousarray(closed, dtype=np.uint8)
    _check(lib().qw_set_links(h, _ptr(closed), _on_device(closed) if closed is not None else 0), h)


def qw_set_link_noise(h, p, seed, step=0):
    _check(lib().qw_set_link_noise(h, float(p), int(seed) & 0xFFFFFFFFFFFFFFFF, int(step)), h)


def qw_get_link_step(h):
    t = ctypes.c_int64(0)
    _check(lib().qw_get_link_step(h, ctypes.byref(t)), h)
    return t.value


def _cdtype(x):
    if isinstance(x, np.ndarray):
        return C64 if x.dtype == np.complex64 else C128
    import torch
    return C64 if x.dtype == torch.complex64 else C128


def qw_set_state(h, amp):
    if isinstance(amp, np.ndarray) and amp.dtype not in (np.complex64, np.complex128):
        amp = amp.astype(np.complex128)
    if isinstance(amp, np.ndarray):
        amp = np.ascontiguousarray(amp)
    _check(lib().qw_set_state(h, _ptr(amp), _cdtype(amp), _on_device(amp)), h)


def qw_get_state(h, out):
    _check(lib().qw_get_state(h, _ptr(out), _cdtype(out), _on_device(out)), h)
    return out


def qw_step(h, T):
    _check(lib().qw_step(h, int(T)), h)


def qw_step_adjoint(h, T):
    _check(lib().qw_step_adjoint(h, int(T)), h)


def qw_probabilities(h, P_out=None, want_norm=True):
    norm = ctypes.c_double(0.0)
    pd = R64
    if P_out is not None:
        if isinstance(P_out, np.ndarray):
            pd = R32 if P_out.dtype == np.float32 else R64
        else:
            import torch
            pd = R32 if P_out.dtype == torch.float32 else R64
    st = lib().qw_probabilities(h, _ptr(P_out), pd, _on_device(P_out) if P_out is not None else 0,
                                ctypes.byref(norm) if want_norm else None)
    _check(st, h)
    return norm.value if want_norm else None


def qw_set_plan(h, k, tile=0):
    _check(lib().qw_set_plan(h, int(k), int(tile)), h)


def qw_get_plan(h):
    k, t = ctypes.c_int(), ctypes.c_int()
    _check(lib().qw_get_plan(h, ctypes.byref(k), ctypes.byref(t)), h)
    return k.value, t.value


def qw_set_plan_ex(h, k, tile=0, variant=0):
    _check(lib().qw_set_plan_ex(h, int(k), int(tile), int(variant)), h)


def qw_get_plan_ex(h):
    k, t, v = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().qw_get_plan_ex(h, ctypes.byref(k), ctypes.byref(t), ctypes.byref(v)), h)
    return k.value, t.value, v.value


def qw_autotune(h):
    buf = ctypes.create_string_buffer(512)
    _check(lib().qw_autotune(h, buf, 512), h)
    return buf.value.decode()


def qw_describe(h):
    import json
    buf = ctypes.create_string_buffer(1024)
    _check(lib().qw_describe(h, buf, 1024), h)
    return json.loads(buf.value.decode())


def qw_set_clipping(h, on):
    _check(lib().qw_set_clipping(h, int(bool(on))), h)


def qw_synchronize(h):
    _check(lib().qw_synchronize(h), h)


def qw_backward(h, rect, T, K, grad_out):
    r = np.ascontiguousarray(rect, dtype=np.int64)
    loss = ctypes.c_double(0.0)
    _check(lib().qw_backward(h, _ptr(r), int(T), int(K), ctypes.byref(loss), _ptr(grad_out),
                             _on_device(grad_out)), h)
    return loss.value


def qw_probabilities_noalloc(amp, P_out=None, norm_out=None, stream=None):
    """Marginals and norm of a caller-owned device state without any library
    allocation (see include/qw.h).  amp: contiguous torch complex64/complex128
    tensor of shape (d, ...) on the GPU, d = 2 or 4; P_out: contiguous
    float32/float64 tensor with at least one element per site, or None;
    norm_out: float64 tensor with at least one element, or None.  All on the
    same GPU.  Returns the status.  Raises ValueError on any other argument:
    the library reads and writes these pointers as device memory of exactly
    those types and sizes, so a host tensor, a strided view or a short output
    would be an out-of-bounds access on the GPU."""
    import torch
    if not isinstance(amp, torch.Tensor) or not amp.is_cuda:
        raise ValueError("amp must be a CUDA tensor")
    if amp.dtype not in (torch.complex64, torch.complex128):
        raise ValueError(f"amp must be complex64 or complex128, not {amp.dtype}")
    if not amp.is_contiguous() or amp.dim() < 2:
        raise ValueError("amp must be a contiguous tensor of shape (d, sites...)")
    d = int(amp.shape[0])
    ns = int(amp[0].numel())
    dev = amp.device
    if P_out is not None:
        if not isinstance(P_out, torch.Tensor) or not P_out.is_cuda or P_out.device != dev:
            raise ValueError("P_out must be a CUDA tensor on the device of amp")
        if P_out.dtype not in (torch.float32, torch.float64):
            raise ValueError(f"P_out must be float32 or float64, not {P_out.dtype}")
        if not P_out.is_contiguous() or P_out.numel() < ns:
            raise ValueError(f"P_out must be contiguous with at least {ns} elements")
    if norm_out is not None:
        if not isinstance(norm_out, torch.Tensor) or not norm_out.is_cuda or norm_out.device != dev:
            raise ValueError("norm_out must be a CUDA tensor on the device of amp")
        if norm_out.dtype != torch.float64 or norm_out.numel() < 1:
            raise ValueError("norm_out must be a float64 tensor with at least one element")
    dt = C64 if amp.dtype == torch.complex64 else C128
    pd = R32 if (P_out is not None and P_out.dtype == torch.float32) else R64
    return lib().qw_probabilities_noalloc(_ptr(amp), dt, d, ns, _ptr(P_out), pd, _ptr(norm_out),
                                          stream if stream is not None else _stream())


def qw_debug_bounded_wait(spins, stream=None):
    return lib().qw_debug_bounded_wait(int(spins), stream if stream is not None else _stream())


# ---------------------------------------------------------------- convenience
class Walk:
    """A walk handle: the lattice, its coin and its state live on the GPU.

    ``Walk((N,))`` is the cycle Z_N (coin dim 2); ``Walk((Lx, Ly))`` the torus
    (coin dim 4).  ``prec`` is one of "f64", "f32", "bf16", "comp".
    """

    def __init__(self, dims, prec="f32", shift=SHIFT_MOVING, bc=BC_PERIODIC, stream=None):
        dims = tuple(int(x) for x in dims)
        self.ndim = len(dims)
        self.dims = dims
        self.d = 2 * self.ndim
        self.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        self.h = qw_create(self.ndim, dims, self.d, bc, shift, self.prec, stream)
        self.nsites = int(np.prod(dims))

    @property
    def plane_shape(self):
        return (self.nsites,) if self.ndim == 1 else (self.dims[1], self.dims[0])

    def close(self):
        if getattr(self, "h", None):
            qw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_coin(self, coin, per_site=False):
        qw_set_coin(self.h, coin, per_site)
        return self

    def set_coin_phases(self, base, phi):
        qw_set_coin_phases(self.h, base, phi)
        return self

    def set_links(self, closed):
        qw_set_links(self.h, closed)
        return self

    def run_host_batch(self, states, T, count=None, P_out=None, norms=False):
        """Independent runs of T steps from host states, copies overlapping the
        steps (qw_run_host_batch).  states: (count, d, ...) numpy array, or one
        state (d, ...) reused `count` times.  P_out: (count, ...) or one plane
        shape (reused, the last run's P remains); float32 or float64, allocated
        if None.  Returns P_out (and the norms if `norms`)."""
        states = np.ascontiguousarray(states)
        if count is None:
            count, in_stride = states.shape[0], states[0].nbytes
        else:
            in_stride = 0
        if P_out is None:
            P_out = np.empty((count,) + self.plane_shape, dtype=np.float64)
        p_stride = P_out[0].nbytes if P_out.shape != self.plane_shape else 0
        nrm = np.empty(max(count, 1), dtype=np.float64) if norms else None
        _check(lib().qw_run_host_batch(self.h, int(count), _ptr(states), int(in_stride), _cdtype(states), int(T),
                                       _ptr(P_out), int(p_stride), R32 if P_out.dtype == np.float32 else R64,
                                       _ptr(nrm)), self.h)
        return (P_out, nrm[:count]) if norms else P_out

    def set_link_noise(self, p, seed, step=0):
        """Links broken at random afresh at every step with probability p."""
        qw_set_link_noise(self.h, p, seed, step)
        return self

    def link_step(self):
        return qw_get_link_step(self.h)

    def set_state(self, amp):
        qw_set_state(self.h, amp)
        return self

    def state(self, dtype=np.complex128):
        out = np.empty((self.d,) + self.plane_shape, dtype=dtype)
        qw_get_state(self.h, out)
        return out

    def step(self, T):
        qw_step(self.h, T)
        return self

    def step_adjoint(self, T):
        qw_step_adjoint(self.h, T)
        return self

    def probabilities(self, dtype=np.float64):
        P = np.empty(self.plane_shape, dtype=dtype)
        norm = qw_probabilities(self.h, P)
        return P, norm

    def norm(self):
        return qw_probabilities(self.h, None)

    def set_plan(self, k, tile=0):
        qw_set_plan(self.h, k, tile)
        return self

    def plan(self):
        return qw_get_plan(self.h)

    def set_plan_ex(self, k, tile=0, variant=0):
        qw_set_plan_ex(self.h, k, tile, variant)
        return self

    def plan_ex(self):
        return qw_get_plan_ex(self.h)

    def autotune(self):
        return qw_autotune(self.h)

    def describe(self):
        return qw_describe(self.h)

    def set_clipping(self, on):
        """Light-cone clipping of localised states (on by default; see qw_set_clipping)."""
        qw_set_clipping(self.h, on)
        return self

    def synchronize(self):
        qw_synchronize(self.h)


class Batch:
    """Many independent walks on cycles, advanced in one persistent launch.

    N, T, x0: integer arrays (one entry per walk); coins: (nwalks, 2, 2)
    complex; coin_state: the two coin amplitudes at x0; prec "f32", "bf16" or
    "comp" (double-float).
    """

    def __init__(self, N, T, coins, x0, coin_state=(2 ** -0.5, 1j * 2 ** -0.5), prec="f32",
                 stream=None):
        self.N = np.ascontiguousarray(N, dtype=np.int64)
        self.T = np.ascontiguousarray(T, dtype=np.int64)
        self.x0 = np.ascontiguousarray(x0, dtype=np.int64)
        c = np.ascontiguousarray(coins, dtype=np.complex128).reshape(len(self.N), 2, 2)
        cs = np.ascontiguousarray(coin_state, dtype=np.complex128)
        self.nwalks = len(self.N)
        self.offsets = np.concatenate([[0], np.cumsum(self.N)]).astype(np.int64)
        h = ctypes.c_void_p()
        st = lib().qw_batch_create(self.nwalks, _ptr(self.N), _ptr(self.T), _ptr(c), _ptr(self.x0),
                                   _ptr(cs), PRECISIONS[prec] if isinstance(prec, str) else int(prec),
                                   stream if stream is not None else _stream(), ctypes.byref(h))
        _check(st)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().qw_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self):
        _check(lib().qw_batch_step(self.h), self.h, batch=True)
        return self

    def set_plan(self, k):
        _check(lib().qw_batch_set_plan(self.h, int(k)), self.h, batch=True)
        return self

    def plan(self):
        k, t = ctypes.c_int(), ctypes.c_int()
        _check(lib().qw_batch_get_plan(self.h, ctypes.byref(k), ctypes.byref(t)), self.h, batch=True)
        return k.value, t.value

    def set_plan_ex(self, k, variant):
        """variant 0: warp tiles with halos; 1: light-cone window sweep."""
        _check(lib().qw_batch_set_plan_ex(self.h, int(k), int(variant)), self.h, batch=True)
        return self

    def set_cta_walks(self, n):
        """Variant 1: the n walks with the most light-cone work run on a whole
        CTA each, the rest on one warp each."""
        _check(lib().qw_batch_set_cta_walks(self.h, int(n)), self.h, batch=True)
        return self

    def cta_walks(self):
        return int(lib().qw_batch_cta_walks(self.h))

    def plan_ex(self):
        k, t, v = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().qw_batch_get_plan_ex(self.h, ctypes.byref(k), ctypes.byref(t), ctypes.byref(v)),
               self.h, batch=True)
        return k.value, t.value, v.value

    def autotune(self):
        buf = ctypes.create_string_buffer(256)
        _check(lib().qw_batch_autotune(self.h, buf, 256), self.h, batch=True)
        return buf.value.decode()

    def probabilities(self, out=None):
        """(P_concat, norms): P of walk i is P_concat[offsets[i]:offsets[i+1]]."""
        if out is None:
            out = np.empty(int(self.offsets[-1]), dtype=np.float32)
        norms = np.empty(self.nwalks, dtype=np.float64)
        _check(lib().qw_batch_probabilities(self.h, _ptr(out), _on_device(out), _ptr(norms)),
               self.h, batch=True)
        return out, norms

    def state(self, walk, dtype=np.complex128):
        out = np.empty((2, int(self.N[walk])), dtype=dtype)
        _check(lib().qw_batch_get_state(self.h, int(walk), _ptr(out),
                                        C64 if dtype == np.complex64 else C128), self.h, batch=True)
        return out


def _region_mass_function():
    import torch

    class RegionMass(torch.autograd.Function):
        """loss = probability mass in rect after T steps on the torus, as a
        function of the per-site coin phases phi (nsites x 4, float32, CUDA);
        C_v = base . diag(e^{i phi_v}).  Forward and backward both come from one
        qw_backward call (forward pass with checkpoints every K steps, then the
        U^dagger sweep); backward returns grad_output * dL/dphi."""

        @staticmethod
        def forward(ctx, phi, walk, base, psi0, rect, T, K):
            qw_set_coin_phases(walk.h, base, phi)
            qw_set_state(walk.h, psi0)
            grad = torch.empty((walk.nsites, 4), dtype=torch.float64, device=phi.device)
            loss = qw_backward(walk.h, rect, T, K, grad)
            ctx.save_for_backward(grad)
            return torch.tensor(loss, dtype=torch.float64, device=phi.device)

        @staticmethod
        def backward(ctx, grad_output):
            (grad,) = ctx.saved_tensors
            return (grad_output * grad).to(torch.float32), None, None, None, None, None, None

    return RegionMass


def region_mass(phi, walk, base, psi0, rect, T, K=64):
    """Differentiable region mass (see RegionMass)."""
    return _region_mass_function().apply(phi, walk, base, psi0, rect, T, K)


# ---------------------------------------------------------------- graphs
GCOIN_GROVER, GCOIN_UNIFORM, GCOIN_PER_VERTEX = 0, 1, 2


def graph_arcs(nvert, edges):
    """Arc form (off, partner) of an edge list, built by the library
    (qw_graph_arcs): vertex v's arcs are off[v] .. off[v+1]-1 in the order its
    edge ends appear, partner[a] the arc at the other end of a's edge."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int64).reshape(-1, 2))
    off = np.empty(int(nvert) + 1, dtype=np.int64)
    partner = np.empty(2 * len(e), dtype=np.int64)
    _check(lib().qw_graph_arcs(int(nvert), len(e), _ptr(e), _ptr(off), _ptr(partner)))
    return off, partner


class GraphWalk:
    """The walk on a general graph (Sec. 2.1) in arc form: one amplitude per
    (vertex, edge end); ``prec`` "f64" or "f32".  The default coin is Grover."""

    def __init__(self, off, partner, prec="f32", stream=None):
        off = np.ascontiguousarray(off, dtype=np.int64)
        partner = np.ascontiguousarray(partner, dtype=np.int64)
        self.nvert = len(off) - 1
        self.narcs = int(off[-1])
        self.deg = np.diff(off)
        self.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        h = ctypes.c_void_p()
        _check(lib().qw_gwalk_create(self.nvert, _ptr(off), _ptr(partner), self.prec,
                                     stream if stream is not None else _stream(), ctypes.byref(h)))
        self.h = h

    def _ck(self, st):
        _check(st, self.h, batch="graph")

    def close(self):
        if getattr(self, "h", None):
            lib().qw_gwalk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_coin(self, coins=None):
        """None: Grover; one d x d matrix (regular graph); or a list of
        per-vertex d(v) x d(v) matrices; or a flat complex array (host or
        device) of the concatenated per-vertex matrices."""
        if coins is None:
            self._ck(lib().qw_gwalk_set_coin(self.h, GCOIN_GROVER, None, 0))
            return self
        if isinstance(coins, np.ndarray) and coins.ndim == 2:
            c = np.ascontiguousarray(coins, dtype=np.complex128)
            self._ck(lib().qw_gwalk_set_coin(self.h, GCOIN_UNIFORM, _ptr(c), 0))
            return self
        if isinstance(coins, (list, tuple)):
            parts = [np.asarray(m, dtype=np.complex128).ravel() for m in coins]
            coins = np.concatenate(parts) if parts else np.zeros(0, np.complex128)
        if isinstance(coins, np.ndarray):
            coins = np.ascontiguousarray(coins, dtype=np.complex128)
            if coins.size == 0:
                coins = np.zeros(1, np.complex128)
        self._ck(lib().qw_gwalk_set_coin(self.h, GCOIN_PER_VERTEX, _ptr(coins), _on_device(coins)))
        return self

    def set_state(self, amp):
        if isinstance(amp, np.ndarray):
            amp = np.ascontiguousarray(amp if amp.dtype in (np.complex64, np.complex128) else amp.astype(np.complex128))
        self._ck(lib().qw_gwalk_set_state(self.h, _ptr(amp), _cdtype(amp), _on_device(amp)))
        return self

    def state(self, dtype=np.complex128, out=None):
        if out is None:
            out = np.empty(self.narcs, dtype=dtype)
        self._ck(lib().qw_gwalk_get_state(self.h, _ptr(out), _cdtype(out), _on_device(out)))
        return out

    def step(self, T):
        self._ck(lib().qw_gwalk_step(self.h, int(T)))
        return self

    def step_adjoint(self, T):
        self._ck(lib().qw_gwalk_step_adjoint(self.h, int(T)))
        return self

    def probabilities(self, dtype=np.float64):
        P = np.empty(self.nvert, dtype=dtype)
        norm = ctypes.c_double(0.0)
        self._ck(lib().qw_gwalk_probabilities(self.h, _ptr(P), R32 if P.dtype == np.float32 else R64, 0,
                                              ctypes.byref(norm)))
        return P, norm.value

    def set_variant(self, v):
        self._ck(lib().qw_gwalk_set_variant(self.h, int(v)))
        return self

    def set_window(self, nbytes):
        """Output bytes per destination bucket of the two-pass forms."""
        self._ck(lib().qw_gwalk_set_window(self.h, int(nbytes)))
        return self

    def variant(self):
        v = ctypes.c_int(0)
        self._ck(lib().qw_gwalk_get_variant(self.h, ctypes.byref(v)))
        return v.value

    def autotune(self):
        buf = ctypes.create_string_buffer(512)
        self._ck(lib().qw_gwalk_autotune(self.h, buf, 512))
        return json.loads(buf.value.decode())

    def synchronize(self):
        self._ck(lib().qw_gwalk_synchronize(self.h))
