"""The allocation-free marginals entry point (qw_probabilities_noalloc).

It serves callers that cannot call cudaMalloc (a thread running while another
holds a global-mode stream capture, an application whose allocator already
holds the device memory, a latency-critical path).  Checked through the C ABI
against qw_probabilities on the same state and against the FP64 oracle's
marginals, on two calls in a row, with the same tolerances as the other
FP32/FP64 parity tests.  This file is collected last, so a run that stops at
the first failure has run everything else.
"""
import ctypes
import gc

import numpy as np
import pytest

import oracle
from paper_1003_3779_gb300 import inputs

pytestmark = pytest.mark.gpu


def _reference(qw, psi, dims, prec):
    w = qw.Walk(dims, prec=prec).set_state(psi)
    P, norm = w.probabilities()
    w.close()
    return P.reshape(-1), norm


def _ptol(pdt, cdt):
    """|P_gpu - P| bound relative to max P: one float rounding of P for float32
    output, else the rounding of complex64 inputs' squares summed in double."""
    if pdt == "f32":
        return 2.0 ** -23
    return 1e-14


@pytest.mark.parametrize("cdt", ["c64", "c128"])
@pytest.mark.parametrize("pdt", ["f32", "f64"])
@pytest.mark.parametrize("dims", [(1 << 20,), (37, 29)])
def test_noalloc_matches_probabilities_and_oracle_on_two_calls(cdt, pdt, dims):
    import torch
    import paper_1003_3779_gb300.qw as qw
    d = 2 * len(dims)
    shape = (d, dims[0]) if len(dims) == 1 else (d, dims[1], dims[0])
    npdt = np.complex64 if cdt == "c64" else np.complex128
    tdt = torch.float32 if pdt == "f32" else torch.float64
    prec = "f32" if cdt == "c64" else "f64"
    for call in range(2):
        psi = inputs.random_state(shape, seed=40 + call).astype(npdt)
        # the oracle on the same (rounded) amplitudes, and the handle-based entry point
        want_P, want_norm = oracle.probabilities(psi.astype(np.complex128))
        want_P = want_P.reshape(-1)
        lib_P, lib_norm = _reference(qw, psi, dims, prec)
        amp = torch.from_numpy(psi).cuda()
        P = torch.full((int(np.prod(dims)),), -1.0, dtype=tdt, device="cuda")
        norm = torch.zeros(1, dtype=torch.float64, device="cuda")
        assert qw.qw_probabilities_noalloc(amp, P, norm) == qw.QW_OK
        torch.cuda.synchronize()
        got = P.cpu().numpy().astype(np.float64)
        tol = _ptol(pdt, cdt) * want_P.max()
        assert np.abs(got - want_P).max() <= tol
        assert np.abs(got - lib_P).max() <= tol + _ptol("f32" if prec == "f32" else "f64", cdt) * want_P.max()
        # the norm: double sums of the same squares in two fixed orders
        assert abs(norm.item() - want_norm) < 1e-12
        assert abs(norm.item() - lib_norm) < 1e-12


def test_noalloc_on_a_side_stream():
    import torch
    import paper_1003_3779_gb300.qw as qw
    psi = inputs.random_state((4, 300, 200), seed=7).astype(np.complex64)
    want_P, want_norm = oracle.probabilities(psi.astype(np.complex128))
    side = torch.cuda.Stream()
    amp = torch.from_numpy(psi).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        P = torch.empty(300 * 200, dtype=torch.float32, device="cuda")
        norm = torch.zeros(1, dtype=torch.float64, device="cuda")
        st = qw.qw_probabilities_noalloc(amp, P, norm, stream=ctypes.c_void_p(side.cuda_stream))
    assert st == qw.QW_OK
    side.synchronize()
    assert np.abs(P.cpu().numpy() - want_P.reshape(-1)).max() <= 2.0 ** -23 * want_P.max()
    assert abs(norm.item() - want_norm) < 1e-12


def test_noalloc_allocates_no_device_memory():
    """After a first call (which looks up the scratch address and loads the
    kernels), calls leave the device's free memory unchanged."""
    import torch
    import paper_1003_3779_gb300.qw as qw
    psi = inputs.random_state((2, 1 << 16), seed=9).astype(np.complex128)
    amp = torch.from_numpy(psi).cuda()
    P32 = torch.empty(1 << 16, dtype=torch.float32, device="cuda")
    P64 = torch.empty(1 << 16, dtype=torch.float64, device="cuda")
    norm = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert qw.qw_probabilities_noalloc(amp, P32, norm) == qw.QW_OK
    torch.cuda.synchronize()
    # no garbage collection in between: a collected handle of an earlier test
    # would free its device memory and move the count
    gc.collect()
    gc.disable()
    try:
        free0, _ = torch.cuda.mem_get_info()
        for P in (P64, P32, None):
            assert qw.qw_probabilities_noalloc(amp, P, norm) == qw.QW_OK
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    finally:
        gc.enable()
    assert free1 == free0
    want_P, want_norm = oracle.probabilities(psi)
    assert abs(norm.item() - want_norm) < 1e-12
    assert np.abs(P32.cpu().numpy() - want_P).max() <= 2.0 ** -23 * want_P.max()


def test_noalloc_odd_size_then_smaller_and_limits():
    import torch
    import paper_1003_3779_gb300.qw as qw
    for n in (100003, 5):   # the second, smaller call must not see the first call's partials
        psi = inputs.random_state((2, n), seed=n).astype(np.complex64)
        want_P, want_norm = oracle.probabilities(psi.astype(np.complex128))
        amp = torch.from_numpy(psi).cuda()
        norm = torch.zeros(1, dtype=torch.float64, device="cuda")
        assert qw.qw_probabilities_noalloc(amp, None, norm) == qw.QW_OK
        torch.cuda.synchronize()
        assert abs(norm.item() - want_norm) < 1e-12
    # beyond the scratch array: rejected before any launch (no buffer that large is touched)
    L = qw.lib()
    small = torch.zeros(2, 8, dtype=torch.complex64, device="cuda")
    st = L.qw_probabilities_noalloc(qw._ptr(small), qw.C64, 2, (1 << 27) + 1, None, qw.R32, None, None)
    assert st == qw.QW_EINVAL
    assert L.qw_probabilities_noalloc(None, qw.C64, 2, 8, None, qw.R32, None, None) == qw.QW_EINVAL


def test_noalloc_binding_rejects_what_the_kernel_cannot_take():
    """The binding refuses, before any launch, arguments the library would read
    or write out of bounds: host tensors, strided views, other dtypes, short
    outputs."""
    import torch
    import paper_1003_3779_gb300.qw as qw
    amp = torch.zeros(2, 64, dtype=torch.complex64, device="cuda")
    ok_P = torch.empty(64, dtype=torch.float32, device="cuda")
    ok_n = torch.zeros(1, dtype=torch.float64, device="cuda")
    bad = [
        dict(amp=amp.cpu()),
        dict(amp=torch.zeros(2, 128, dtype=torch.complex64, device="cuda")[:, ::2]),
        dict(amp=torch.zeros(2, 64, dtype=torch.float32, device="cuda")),
        dict(amp=amp, P_out=ok_P.cpu()),
        dict(amp=amp, P_out=torch.empty(64, dtype=torch.float16, device="cuda")),
        dict(amp=amp, P_out=torch.empty(63, dtype=torch.float32, device="cuda")),
        dict(amp=amp, norm_out=ok_n.cpu()),
        dict(amp=amp, norm_out=torch.zeros(1, dtype=torch.float32, device="cuda")),
    ]
    for kw in bad:
        with pytest.raises(ValueError):
            qw.qw_probabilities_noalloc(**kw)
    assert qw.qw_probabilities_noalloc(amp, ok_P, ok_n) == qw.QW_OK
    torch.cuda.synchronize()
