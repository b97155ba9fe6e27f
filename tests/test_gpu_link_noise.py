"""GPU parity for links broken at random afresh at every step (Sec. 3, the RBL
function resampled per step): the generic kernel draws each link's state from
Philox4x32-10 on the device; the oracle draws the same masks from its own
Philox and applies them step by step."""
import numpy as np
import pytest

import oracle
from paper_1003_3779_gb300 import inputs
from tests.helpers import amp_tol, maxabs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qw():
    import paper_1003_3779_gb300.qw as qw
    qw.lib()
    return qw


def make_walk(qw, shape, prec, shift, bc):
    if len(shape) == 2:
        return qw.Walk((shape[1],), prec=prec, shift=shift, bc=bc)
    return qw.Walk((shape[2], shape[1]), prec=prec, shift=shift, bc=bc)


@pytest.mark.parametrize("prec", ["f64", "f32", "comp"])
@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("ndim", [1, 2])
@pytest.mark.parametrize("p", [0.05, 0.5])
def test_random_links_forward(qw, prec, bc, shift, ndim, p):
    rng = np.random.default_rng(100 + bc + 3 * shift + 7 * ndim)
    shape = (2, 301) if ndim == 1 else (4, 13, 17)
    C = inputs.random_unitary(2 * ndim, rng)
    psi0 = inputs.random_state(shape, seed=31)
    T, seed, t0 = 19, 0x1234_5678_9ABC_DEF0 + ndim, 5
    masks = oracle.link_masks(shape[1:], seed, p, t0, T)
    want = oracle.evolve(psi0, C, T, shift=shift, bc=bc, closed=masks, closed_per_step=True)
    w = make_walk(qw, shape, prec, shift, bc).set_coin(C).set_link_noise(p, seed, t0).set_state(psi0)
    assert w.describe()["path"] == "generic"
    w.step(T)
    assert w.link_step() == t0 + T
    assert maxabs(w.state(), want) < amp_tol(prec, T)
    w.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("ndim", [1, 2])
def test_random_links_adjoint_and_inverse(qw, prec, ndim):
    """The adjoint counts the step index down before each step: from index T it
    applies (U_{T-1} ... U_0)^dagger, the oracle's adjoint over masks 0..T-1, and
    a forward run followed by its adjoint returns the initial state."""
    rng = np.random.default_rng(140 + ndim)
    shape = (2, 257) if ndim == 1 else (4, 11, 19)
    C = inputs.random_unitary(2 * ndim, rng)
    psi0 = inputs.random_state(shape, seed=32)
    T, seed, p = 23, 77, 0.3
    masks = oracle.link_masks(shape[1:], seed, p, 0, T)
    want = oracle.evolve(psi0, C, T, closed=masks, closed_per_step=True, adjoint=True)
    w = make_walk(qw, shape, prec, 0, 0).set_coin(C).set_link_noise(p, seed, T).set_state(psi0)
    w.step_adjoint(T)
    assert w.link_step() == 0
    assert maxabs(w.state(), want) < amp_tol(prec, T)
    w.set_state(psi0)
    w.step(T)
    assert w.link_step() == T
    w.step_adjoint(T)
    assert maxabs(w.state(), psi0) < 2 * amp_tol(prec, T)
    w.close()


@pytest.mark.parametrize("ndim", [1, 2])
def test_random_links_or_fixed_mask(qw, ndim):
    """A link is closed when the fixed mask or the step's random draw closes it."""
    rng = np.random.default_rng(150 + ndim)
    shape = (2, 300) if ndim == 1 else (4, 16, 16)
    ns = int(np.prod(shape[1:]))
    fixed = (rng.uniform(size=(ndim, ns)) < 0.2).astype(np.uint8)
    C = inputs.random_unitary(2 * ndim, rng)
    psi0 = inputs.random_state(shape, seed=33)
    T, seed, p = 17, 2024, 0.1
    masks = oracle.link_masks(shape[1:], seed, p, 0, T) | fixed[None]
    want = oracle.evolve(psi0, C, T, closed=masks, closed_per_step=True)
    w = make_walk(qw, shape, "f64", 0, 0).set_coin(C).set_links(fixed).set_link_noise(p, seed).set_state(psi0)
    w.step(T)
    assert maxabs(w.state(), want) < 1e-12
    w.close()


def test_random_links_counter_wraps(qw):
    """The step index enters the counter modulo 2^32."""
    shape = (4, 9, 10)
    C = inputs.grover()
    psi0 = inputs.random_state(shape, seed=34)
    T, seed, p, t0 = 8, 5, 0.25, (1 << 32) - 3
    masks = oracle.link_masks(shape[1:], seed, p, t0, T)
    assert np.array_equal(masks[3:], oracle.link_masks(shape[1:], seed, p, 0, T - 3))
    want = oracle.evolve(psi0, C, T, closed=masks, closed_per_step=True)
    w = make_walk(qw, shape, "f64", 0, 0).set_coin(C).set_link_noise(p, seed, t0).set_state(psi0)
    w.step(T)
    assert maxabs(w.state(), want) < 1e-12
    w.close()


def test_random_links_extremes(qw):
    """p = 0 is the plain walk on the periodic kernels; p = 1 closes every link,
    so each step reflects every amplitude in place (the oracle's all-closed mask)."""
    rng = np.random.default_rng(160)
    shape = (4, 12, 20)
    C = inputs.random_unitary(4, rng)
    psi0 = inputs.random_state(shape, seed=35)
    T = 9
    w = make_walk(qw, shape, "f64", 0, 0).set_coin(C).set_link_noise(0.0, 1).set_state(psi0)
    assert w.describe()["path"] != "generic"
    w.step(T)
    assert maxabs(w.state(), oracle.evolve(psi0, C, T)) < 1e-12
    w.set_link_noise(1.0, 1).set_state(psi0)
    w.step(T)
    allclosed = np.ones((T, 2, 240), dtype=np.uint8)
    assert np.array_equal(oracle.link_masks(shape[1:], 1, 1.0, 0, T), allclosed)
    assert maxabs(w.state(), oracle.evolve(psi0, C, T, closed=allclosed, closed_per_step=True)) < 1e-12
    w.close()


def test_random_links_rejections(qw):
    w = qw.Walk((64,), prec="f64").set_coin(inputs.hadamard())
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(qw.QWError):
            w.set_link_noise(bad, 1)
    w.close()
    w = qw.Walk((16, 16), prec="f64", shift=qw.SHIFT_DIAGONAL).set_coin(inputs.hadamard2())
    with pytest.raises(qw.QWError):
        w.set_link_noise(0.1, 1)
    w.close()
    w = qw.Walk((16, 16), prec="f32")
    w.set_coin_phases(inputs.grover(), np.zeros((256, 4), dtype=np.float32)).set_link_noise(0.1, 1)
    w.set_state(inputs.localized_2d(16))
    with pytest.raises(qw.QWError):
        qw.qw_backward(w.h, (4, 4, 4, 4), 4, 2, np.zeros((256, 4), dtype=np.float64))
    w.close()
