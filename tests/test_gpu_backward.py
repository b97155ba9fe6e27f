"""The adjoint gradient of a region's mass with respect to per-site coin phases
(qw_backward): against the FP64 stored-trajectory oracle gradient, central
finite differences of the FP64 GPU forward, and exact zeros outside the past
light cone."""
import numpy as np
import pytest

import oracle
from paper_1003_3779_gb300 import inputs
from tests.helpers import maxabs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qw():
    import paper_1003_3779_gb300.qw as qw
    qw.lib()
    return qw


def gpu_grad(qw, psi0, base, phi, T, K, rect, prec, shift=0):
    d, Ly, Lx = psi0.shape
    w = qw.Walk((Lx, Ly), prec=prec, shift=shift)
    w.set_coin_phases(base, phi.reshape(-1, 4).astype(np.float32)).set_state(psi0)
    grad = np.empty((Lx * Ly, 4))
    loss = qw.qw_backward(w.h, rect, T, K, grad)
    end = w.state()
    w.close()
    return loss, grad.reshape(Ly, Lx, 4), end


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("coin", ["grover", "complex"])
def test_small_torus_against_oracle_gradient(qw, prec, shift, coin):
    rng = np.random.default_rng(7)
    Lx, Ly, T, K = 16, 12, 13, 4
    base = inputs.grover() if coin == "grover" else inputs.random_unitary(4, rng)
    phi = rng.uniform(-0.5, 0.5, size=(Ly, Lx, 4)).astype(np.float32).astype(np.float64)
    psi0 = inputs.random_state((4, Ly, Lx), seed=8)
    rect = (3, 2, 4, 3)
    want_loss, want = oracle.region_grad(psi0, base, phi, T, rect, shift=shift)
    loss, got, end = gpu_grad(qw, psi0, base, phi, T, K, rect, prec, shift)
    tol = 1e-12 if prec == "f64" else 2e-5
    assert abs(loss - want_loss) < tol
    assert maxabs(got, want) < tol * max(1.0, np.abs(want).max())
    # the walk is left at psi_T
    psiT = oracle.evolve(psi0, base, T, shift=shift, phi=phi.reshape(-1, 4))
    assert maxabs(end, psiT) < (1e-12 if prec == "f64" else 1e-5)


def test_64_torus_T512_against_oracle_gradient(qw):
    """The gradient configuration scaled to a 64 x 64 torus: T = 512, K = 64,
    the 4 x 4 square centred at (16, 16), FP32 adjoint vs the FP64 oracle."""
    L, T, K = 64, 512, 64
    phi = inputs.region_grad_phases(L).astype(np.float32).astype(np.float64)
    psi0 = inputs.localized_2d(L)
    rect = inputs.region_rect(L, centre=(16, 16), size=4)
    want_loss, want = oracle.region_grad(psi0, inputs.grover(), phi, T, rect)
    loss, got, _ = gpu_grad(qw, psi0, inputs.grover(), phi, T, K, rect, "f32")
    assert abs(loss - want_loss) < 1e-5 * max(want_loss, 1e-3)
    assert maxabs(got, want) < 1e-4 * np.abs(want).max()


@pytest.mark.slow
def test_full_size_finite_differences_and_light_cone(qw):
    """1024^2 torus, Grover . diag(e^{i phi}), phi ~ U[-0.1, 0.1], T = 512, K = 64,
    region 64 x 64 centred at (256, 256): the FP32 adjoint gradient against
    central differences of the FP64 GPU forward at 32 phases inside the past
    light cone, and exact zeros outside it."""
    import torch
    L, T, K = 1024, 512, 64
    phi = inputs.region_grad_phases(L).astype(np.float32)
    psi0 = inputs.localized_2d(L)
    rect = inputs.region_rect(L)
    loss, grad, _ = gpu_grad(qw, psi0, inputs.grover(), phi.astype(np.float64), T, K, rect, "f32")
    x0, y0, w_, h_ = rect
    yy, xx = np.mgrid[0:L, 0:L]
    def tdist(a, lo, hi):
        # circular distance from coordinate a to the interval [lo, hi - 1]
        def circ(u, v):
            d = np.abs(u - v)
            return np.minimum(d, L - d)
        inside = (a >= lo) & (a <= hi - 1)
        return np.where(inside, 0, np.minimum(circ(a, lo), circ(a, hi - 1)))
    dist = tdist(xx, x0, x0 + w_) + tdist(yy, y0, y0 + h_)
    assert np.all(grad[dist > T] == 0.0)

    f64 = qw.Walk((L, L), prec="f64")
    def fwd(ph):
        f64.set_coin_phases(inputs.grover(), ph.reshape(-1, 4)).set_state(psi0)
        f64.step(T)
        P, _ = f64.probabilities()
        return float(P[y0:y0 + h_, x0:x0 + w_].sum())
    rng = np.random.default_rng(9)
    cand = np.argwhere((dist <= 300) & (dist >= 1))
    picks = cand[rng.choice(len(cand), size=32, replace=False)]
    h = np.float32(1e-3)
    scale = np.abs(grad).max()
    for (y, x) in picks:
        k = int(rng.integers(0, 4))
        pp, pm = phi.copy(), phi.copy()
        pp[y, x, k] += h
        pm[y, x, k] -= h
        fd = (fwd(pp) - fwd(pm)) / (float(pp[y, x, k]) - float(pm[y, x, k]))
        assert abs(fd - grad[y, x, k]) < 1e-3 * scale + 1e-7, (y, x, k, fd, grad[y, x, k])
    f64.close()


def test_autograd_function(qw):
    import torch
    L, T, K = 32, 40, 8
    rng = np.random.default_rng(10)
    phi = torch.tensor(rng.uniform(-0.1, 0.1, size=(L * L, 4)), dtype=torch.float32,
                       device="cuda", requires_grad=True)
    psi0 = inputs.localized_2d(L, 16, 16)
    w = qw.Walk((L, L), prec="f32")
    rect = (18, 18, 6, 6)
    loss = qw.region_mass(phi, w, inputs.grover(), psi0, rect, T, K)
    loss.backward()
    want_loss, want = oracle.region_grad(psi0, inputs.grover(),
                                         phi.detach().cpu().numpy().astype(np.float64), T, rect)
    assert abs(loss.item() - want_loss) < 1e-5
    assert maxabs(phi.grad.cpu().numpy().reshape(L, L, 4), want) < 1e-4 * max(1e-3, np.abs(want).max())
    w.close()
