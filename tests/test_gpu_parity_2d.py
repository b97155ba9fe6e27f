"""GPU parity on the torus (coin dim 4) and for the general boundary / broken-link
path: the CUDA path through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1003_3779_gb300 import inputs
from tests.helpers import amp_tol, l1, maxabs, p_l1_tol

pytestmark = pytest.mark.gpu

PRECS = ["f64", "f32", "bf16", "comp"]


@pytest.fixture(scope="module")
def qw():
    import paper_1003_3779_gb300.qw as qw
    qw.lib()
    return qw


def coin_named(name, rng):
    if name == "grover":
        return inputs.grover()
    if name == "hh":
        return inputs.hadamard2()
    if name == "fourier":
        return inputs.fourier()
    if name == "real":
        q, _ = np.linalg.qr(rng.standard_normal((4, 4)))
        return q.astype(np.complex128)
    return inputs.random_unitary(4, rng)


def gpu_run(qw, psi0, coin, T, prec, shift=0, adjoint=False, per_site=False, phases=None, bc=0,
            links=None):
    d, Ly, Lx = psi0.shape
    w = qw.Walk((Lx, Ly), prec=prec, shift=shift, bc=bc)
    if phases is not None:
        w.set_coin_phases(coin, phases)
    else:
        w.set_coin(coin, per_site=per_site)
    if links is not None:
        w.set_links(links)
    w.set_state(psi0)
    (w.step_adjoint if adjoint else w.step)(T)
    out = w.state()
    P, norm = w.probabilities()
    w.close()
    return out, P, norm


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("coin", ["grover", "hh", "real", "complex", "fourier"])
@pytest.mark.parametrize("shift", [0, 1])
def test_torus_coins_shifts(qw, prec, coin, shift):
    rng = np.random.default_rng(["grover", "hh", "real", "complex", "fourier"].index(coin) * 2 + shift)
    C = coin_named(coin, rng)
    Lx, Ly, T = 136, 18, 23          # 136 = one full 128-site segment + a ragged tail
    psi0 = inputs.random_state((4, Ly, Lx), seed=21)
    want = oracle.evolve(psi0, C, T, shift=shift)
    got, P, _ = gpu_run(qw, psi0, C, T, prec, shift=shift)
    assert maxabs(got, want) < amp_tol(prec, T)
    assert l1(P, oracle.probabilities(want)[0]) < p_l1_tol(prec, T, Lx * Ly)


@pytest.mark.parametrize("prec", PRECS)
def test_grover_from_origin_symmetry(qw, prec):
    L, T = 256, 100
    psi0 = inputs.localized_2d(L)
    want = oracle.evolve(psi0, inputs.grover(), T)
    got, P, norm = gpu_run(qw, psi0, inputs.grover(), T, prec)
    assert maxabs(got, want) < amp_tol(prec, T)
    if prec != "bf16":
        neg = (-np.arange(L)) % L
        assert maxabs(P, P.T) < 1e-6 and maxabs(P, P[neg][:, neg]) < 1e-6
        y, x = np.mgrid[0:L, 0:L]
        assert np.all(P[(x + y - T) % 2 != 0] == 0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("coin", ["grover", "hh", "complex", "real"])
@pytest.mark.parametrize("shift", [0, 1])
def test_torus_adjoint(qw, prec, coin, shift):
    rng = np.random.default_rng(31)
    C = coin_named(coin, rng)
    Lx, Ly, T = 260, 7, 15
    psi0 = inputs.random_state((4, Ly, Lx), seed=22)
    want = oracle.evolve(psi0, C, T, shift=shift, adjoint=True)
    got, _, _ = gpu_run(qw, psi0, C, T, prec, shift=shift, adjoint=True)
    assert maxabs(got, want) < amp_tol(prec, T)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_phase_coin_2d(qw, prec, shift, adjoint):
    Lx, Ly, T = 128, 40, 12
    rng = np.random.default_rng(41)
    phi = rng.uniform(-0.5, 0.5, size=(Ly, Lx, 4)).astype(np.float32)
    psi0 = inputs.random_state((4, Ly, Lx), seed=23)
    want = oracle.evolve(psi0, inputs.grover(), T, shift=shift, phi=phi.reshape(-1, 4).astype(np.float64),
                         adjoint=adjoint)
    got, _, _ = gpu_run(qw, psi0, inputs.grover(), T, prec, shift=shift, adjoint=adjoint,
                        phases=phi.reshape(-1, 4))
    assert maxabs(got, want) < amp_tol(prec, T) + (T * 2e-7 if prec in ("f32", "bf16") else 0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_per_site_matrices_2d(qw, prec):
    Lx, Ly, T = 9, 6, 7
    rng = np.random.default_rng(51)
    coins = np.stack([inputs.random_unitary(4, rng) for _ in range(Lx * Ly)])
    psi0 = inputs.random_state((4, Ly, Lx), seed=24)
    for shift in (0, 1):
        for adj in (False, True):
            want = oracle.evolve(psi0, coins, T, shift=shift, adjoint=adj)
            got, _, _ = gpu_run(qw, psi0, coins, T, prec, shift=shift, per_site=True, adjoint=adj)
            assert maxabs(got, want) < amp_tol(prec, T)


@pytest.mark.parametrize("prec", ["f64", "f32", "comp"])
@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("ndim", [1, 2])
def test_boundaries_and_broken_links(qw, prec, bc, shift, ndim):
    rng = np.random.default_rng(61 + bc + 3 * shift + 7 * ndim)
    shape = (2, 301) if ndim == 1 else (4, 13, 17)
    ns = int(np.prod(shape[1:]))
    closed = (rng.uniform(size=(ndim, ns)) < 0.15).astype(np.uint8)
    C = inputs.random_unitary(2 * ndim, rng)
    psi0 = inputs.random_state(shape, seed=25)
    T = 19
    for adj in (False, True):
        want = oracle.evolve(psi0, C, T, shift=shift, bc=bc, closed=closed, adjoint=adj)
        if ndim == 1:
            w = qw.Walk((shape[1],), prec=prec, shift=shift, bc=bc)
        else:
            w = qw.Walk((shape[2], shape[1]), prec=prec, shift=shift, bc=bc)
        w.set_coin(C).set_links(closed).set_state(psi0)
        (w.step_adjoint if adj else w.step)(T)
        assert maxabs(w.state(), want) < amp_tol(prec, T)
        w.close()


@pytest.mark.parametrize("L", [1, 2, 3, 6])
def test_tiny_torus(qw, L):
    rng = np.random.default_rng(L)
    C = inputs.random_unitary(4, rng)
    psi0 = inputs.random_state((4, L, L), seed=L)
    want = oracle.evolve(psi0, C, 9)
    got, _, _ = gpu_run(qw, psi0, C, 9, "f64")
    assert maxabs(got, want) < 1e-12


@pytest.mark.parametrize("k", [4, 8])
@pytest.mark.parametrize("coin", ["grover", "hh", "real", "complex"])
@pytest.mark.parametrize("shift", [0, 1, 2])
@pytest.mark.parametrize("dims", [(200, 37), (64, 300), (48, 9)])
def test_torus_temporal_blocking(qw, k, coin, shift, dims):
    """The streaming kernel (k steps per HBM round trip) against the oracle:
    strips and row chunks with ragged ends, wrap in x and y, T not a multiple
    of k; moving, flip-flop and diagonal-lattice shifts."""
    rng = np.random.default_rng(["grover", "hh", "real", "complex"].index(coin) + 10 * k)
    C = coin_named(coin, rng)
    Lx, Ly = dims
    T = 3 * k + 3
    psi0 = inputs.random_state((4, Ly, Lx), seed=26)
    want = oracle.evolve(psi0, C, T, shift=shift)
    w = qw.Walk((Lx, Ly), prec="f32", shift=shift).set_coin(C).set_plan(k)
    assert w.describe()["path"] == "k_step2d_tb"
    w.set_state(psi0)
    w.step(T)
    assert maxabs(w.state(), want) < amp_tol("f32", T)
    w.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("coin", ["hh", "fourier", "grover", "complex"])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("dims", [(136, 18), (9, 7)])
def test_diagonal_lattice(qw, prec, coin, adjoint, dims):
    """The diagonal lattice (each coin qubit drives one axis) against the oracle,
    forward and adjoint, full segments plus ragged tails and a tiny torus."""
    rng = np.random.default_rng(["hh", "fourier", "grover", "complex"].index(coin) + 50)
    C = coin_named(coin, rng)
    Lx, Ly = dims
    T = 21
    psi0 = inputs.random_state((4, Ly, Lx), seed=27)
    want = oracle.evolve(psi0, C, T, shift=2, adjoint=adjoint)
    w = qw.Walk((Lx, Ly), prec=prec, shift=qw.SHIFT_DIAGONAL).set_coin(C).set_state(psi0)
    (w.step_adjoint if adjoint else w.step)(T)
    assert maxabs(w.state(), want) < amp_tol(prec, T)
    w.close()


def test_diagonal_hadamard_factorises_on_gpu(qw):
    """H (x) H on the diagonal lattice from a product start: P(x, y) = P1(-x) P1(-y)
    with P1 the Hadamard walk on the cycle (exact factorisation of the walk)."""
    L, T = 256, 100
    a = (0.6, 0.8j)
    b = (1 / np.sqrt(2), -1 / np.sqrt(2))
    psi = np.zeros((4, L, L), dtype=complex)
    for j in range(2):
        for k in range(2):
            psi[2 * j + k, 0, 0] = a[j] * b[k]
    w = qw.Walk((L, L), prec="f64", shift=qw.SHIFT_DIAGONAL).set_coin(inputs.hadamard2()).set_state(psi)
    w.step(T)
    P, _ = w.probabilities()
    Px, _ = oracle.probabilities(oracle.evolve(inputs.localized_1d(L, 0, a), inputs.hadamard(), T))
    Py, _ = oracle.probabilities(oracle.evolve(inputs.localized_1d(L, 0, b), inputs.hadamard(), T))
    neg = (-np.arange(L)) % L
    assert np.abs(P - np.outer(Py[neg], Px[neg])).max() < 1e-13
    w.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("dims", [(200, 37), (3, 5)])
@pytest.mark.parametrize("coin", ["per_site", "phase"])
def test_tiled_generic_step_site_coins(qw, prec, bc, shift, dims, coin):
    """The tiled generic step with per-site matrices or phase coins, several
    tiles, boundaries and both kinds of broken links, against the oracle."""
    Lx, Ly = dims
    ns = Lx * Ly
    rng = np.random.default_rng(Lx + 5 * bc + 3 * shift + len(coin))
    fixed = (rng.uniform(size=(2, ns)) < 0.1).astype(np.uint8)
    psi0 = inputs.random_state((4, Ly, Lx), seed=30)
    T, seed, p = 9, 97, 0.2
    masks = oracle.link_masks((Ly, Lx), seed, p, 0, T) | fixed[None]
    w = qw.Walk((Lx, Ly), prec=prec, shift=shift, bc=bc)
    tol = amp_tol(prec, T)
    if coin == "per_site":
        coins = np.stack([inputs.random_unitary(4, rng) for _ in range(ns)])
        want = oracle.evolve(psi0, coins, T, shift=shift, bc=bc, closed=masks, closed_per_step=True)
        w.set_coin(coins, per_site=True)
    else:
        phi = rng.uniform(-0.5, 0.5, size=(ns, 4)).astype(np.float32)
        want = oracle.evolve(psi0, inputs.grover(), T, shift=shift, bc=bc, phi=phi.astype(np.float64),
                             closed=masks, closed_per_step=True)
        w.set_coin_phases(inputs.grover(), phi)
        tol += T * 2e-7 if prec in ("f32", "bf16") else 0
    w.set_links(fixed).set_link_noise(p, seed).set_state(psi0)
    w.step(T)
    assert maxabs(w.state(), want) < tol
    w.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("dims", [(200, 37), (129, 70), (3, 5)])
def test_tiled_generic_step_multi_tile(qw, prec, bc, shift, dims):
    """The tiled generic step (64 x 8 sites per block, one-site halo
    in shared memory): several tiles with ragged edges, wrap-around, a fixed
    mask and links broken at random per step, against the oracle; the adjoint
    (the per-site kernel) undoes it."""
    Lx, Ly = dims
    rng = np.random.default_rng(Lx + 7 * bc + 3 * shift)
    C = inputs.random_unitary(4, rng)
    fixed = (rng.uniform(size=(2, Lx * Ly)) < 0.1).astype(np.uint8)
    psi0 = inputs.random_state((4, Ly, Lx), seed=28)
    T, seed, p = 11, 99, 0.2
    masks = oracle.link_masks((Ly, Lx), seed, p, 0, T) | fixed[None]
    want = oracle.evolve(psi0, C, T, shift=shift, bc=bc, closed=masks, closed_per_step=True)
    w = qw.Walk((Lx, Ly), prec=prec, shift=shift, bc=bc).set_coin(C).set_links(fixed).set_link_noise(p, seed)
    w.set_state(psi0)
    w.step(T)
    assert maxabs(w.state(), want) < amp_tol(prec, T)
    if bc != 2 and prec in ("f64", "comp"):
        w.step_adjoint(T)
        assert maxabs(w.state(), psi0) < 2 * amp_tol(prec, T)
    w.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("N", [3 * 1024 + 77, 1024, 5])
def test_tiled_generic_step_cycle(qw, prec, bc, shift, N):
    """The tiled generic step on the cycle (1024 sites per block, one-site halo):
    several tiles, a ragged last one, wrap-around, a fixed mask and links broken
    at random per step, against the oracle."""
    rng = np.random.default_rng(N + 7 * bc + 3 * shift)
    C = inputs.random_unitary(2, rng)
    fixed = (rng.uniform(size=(1, N)) < 0.1).astype(np.uint8)
    psi0 = inputs.random_state((2, N), seed=29)
    T, seed, p = 13, 98, 0.2
    masks = oracle.link_masks((N,), seed, p, 0, T) | fixed[None]
    want = oracle.evolve(psi0, C, T, shift=shift, bc=bc, closed=masks, closed_per_step=True)
    w = qw.Walk((N,), prec=prec, shift=shift, bc=bc).set_coin(C).set_links(fixed).set_link_noise(p, seed)
    w.set_state(psi0)
    w.step(T)
    assert maxabs(w.state(), want) < amp_tol(prec, T)
    w.close()


@pytest.mark.parametrize("prec", ["f64"])
@pytest.mark.parametrize("name", ["grover", "hadamard2"])
def test_near_grover_and_hh_coins_run_as_given_in_double(qw, prec, name):
    """A Grover or H (x) H coin scaled by 1 + 1.8e-15 (every entry moved by
    about 8 ulps, within 1e-15) is applied as given in the double form: after
    T = 1024 steps the state follows the oracle of the scaled coin, far closer
    than the scaling moved it.  The unscaled coin, H (x) H built as
    kron(H, H) of the rounded 1/sqrt2 included, keeps its own kernel."""
    L, T = 32, 1024
    base = inputs.grover() if name == "grover" else inputs.hadamard2()
    C = base * (1 + 1.8e-15)
    psi0 = inputs.random_state((4, L, L), seed=62)
    want = oracle.evolve(psi0, C, T)
    exact = oracle.evolve(psi0, base, T)
    gap = maxabs(want, exact)
    w = qw.Walk((L, L), prec=prec).set_coin(C)
    assert w.describe()["coin_kind"] == "real"
    w.set_state(psi0).step(T)
    got = w.state()
    P, _ = w.probabilities()
    w.close()
    assert maxabs(got, want) < gap / 8, (maxabs(got, want), gap)
    if prec == "f64":
        assert l1(P, oracle.probabilities(want)[0]) < 1e-12
    w = qw.Walk((L, L), prec=prec).set_coin(base)
    assert w.describe()["coin_kind"] == name
    w.close()
