"""The allocation-free marginals entry point (qw_probabilities_noalloc).

It serves callers that cannot call cudaMalloc (a thread running while another
holds a global-mode stream capture, an application whose allocator already
holds the device memory, a latency-critical path).  Checked through the C ABI
against qw_probabilities on the same state, on two calls in a row, with the
same tolerance as the other FP32/FP64 parity tests.  This file is collected
last, so a run that stops at the first failure has run everything else.
"""
import numpy as np
import pytest

from paper_1003_3779_gb300 import inputs

pytestmark = pytest.mark.gpu


def _reference(qw, psi, dims, prec):
    w = qw.Walk(dims, prec=prec).set_state(psi)
    P, norm = w.probabilities()
    w.close()
    return P.reshape(-1), norm


@pytest.mark.parametrize("case", [("f32", (1 << 20,)), ("f64", (37, 29))])
def test_noalloc_matches_probabilities_on_two_calls(case):
    import torch
    import paper_1003_3779_gb300.qw as qw
    prec, dims = case
    d = 2 * len(dims)
    shape = (d, dims[0]) if len(dims) == 1 else (d, dims[1], dims[0])
    cdt = np.complex64 if prec == "f32" else np.complex128
    tdt = torch.float32 if prec == "f32" else torch.float64
    tol_p = 1e-6 if prec == "f32" else 1e-14
    for call in range(2):
        psi = inputs.random_state(shape, seed=40 + call).astype(cdt)
        want_P, want_norm = _reference(qw, psi, dims, prec)
        amp = torch.from_numpy(psi).cuda()
        P = torch.full((int(np.prod(dims)),), -1.0, dtype=tdt, device="cuda")
        norm = torch.zeros(1, dtype=torch.float64, device="cuda")
        st = qw.qw_probabilities_noalloc(amp, P, norm)
        assert st == qw.QW_OK
        torch.cuda.synchronize()
        assert np.abs(P.cpu().numpy().astype(np.float64) - want_P).max() < tol_p * max(1.0, want_P.max())
        assert abs(norm.item() - want_norm) < 1e-12


def test_noalloc_odd_size_then_smaller_and_limits():
    import torch
    import paper_1003_3779_gb300.qw as qw
    for n in (100003, 5):   # the second, smaller call must not see the first call's partials
        psi = inputs.random_state((2, n), seed=n).astype(np.complex64)
        want_P, want_norm = _reference(qw, psi, (n,), "f32")
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
