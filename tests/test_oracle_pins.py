"""Pins of the FP64 oracle against things other than itself.

Each test fixes the oracle to an independent fact: exact Gaussian-integer
arithmetic, the Fourier-space closed form, the dense unitary built explicitly,
or an invariant the walk must obey (Sec. 2.1-3 of the paper).  The set is
chosen so that a transposed coin, a wrong direction, a dropped phase, a wrong
reflection slot or a wrong adjoint each fail at least one test (see
``test_planted_mistakes_are_caught``).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1003_3779_gb300 import inputs
from tests.pins import dense, exact, fourier


def signed(x, N):
    return np.where(x <= N // 2, x, x - N)


# ------------------------------------------------------------ exact Hadamard walk
def test_exact_hadamard_cycle_2001_T1000():
    """Hadamard walk on the cycle N=2001, T=1000 from |0>(x)(|0>+i|1>)/sqrt2:
    oracle probabilities equal the exact rational values to ~1e-15 relative."""
    N, T = 2001, 1000
    num, den = exact.exact_probabilities(N, T)
    assert sum(int(v) for v in num) == den            # norm exactly 1
    p_exact = exact.as_float(num, den)
    psi = oracle.evolve(inputs.localized_1d(N), inputs.hadamard(), T)
    P, norm = oracle.probabilities(psi)
    # the rounded 1/sqrt2 makes each step scale the norm by 1 + O(eps):
    # bound T * 4 * eps
    assert abs(norm - 1.0) < T * 4 * np.finfo(float).eps
    big = p_exact > 1e-30
    rel = np.abs(P[big] - p_exact[big]) / p_exact[big]
    assert rel.max() < T * 4 * np.finfo(float).eps
    # exact invariants: parity zeros and left/right symmetry
    xs = signed(np.arange(N), N)
    odd = (xs - T) % 2 != 0
    assert all(int(num[i]) == 0 for i in np.nonzero(odd)[0])
    assert np.all(P[odd] == 0.0)
    for x in range(1, 1001):
        assert num[x] == num[N - x]


def test_exact_state_amplitudes_small():
    """Amplitudes (not only probabilities) of the Hadamard walk, T odd (exact scale)."""
    N, T = 101, 41
    want = exact.exact_state(N, T)
    got = oracle.evolve(inputs.localized_1d(N), inputs.hadamard(), T)
    # |amplitude| <= 1; each step adds at most a few eps of rounding
    assert np.abs(got - want).max() < T * 4 * np.finfo(float).eps


def test_hadamard_variance_asymptotics():
    """Loose textbook check (Nayak & Vishwanath): Var(x)/T^2 -> 1 - 1/sqrt2."""
    N, T = 2001, 1000
    P, _ = oracle.probabilities(oracle.evolve(inputs.localized_1d(N), inputs.hadamard(), T))
    xs = signed(np.arange(N), N).astype(float)
    mean = (P * xs).sum()
    var = (P * xs * xs).sum() - mean * mean
    assert abs(var / T**2 - (1 - 1 / math.sqrt(2))) < 0.01


# ------------------------------------------------------------ Fourier closed form
@pytest.mark.parametrize("flipflop", [False, True])
@pytest.mark.parametrize("N,T", [(257, 50), (64, 200)])
def test_fourier_closed_form_1d(N, T, flipflop):
    rng = np.random.default_rng(11)
    C = inputs.random_unitary(2, rng)
    psi0 = inputs.random_state((2, N), seed=5)
    want = fourier.evolve_fourier(psi0, C, T, flipflop=flipflop)
    got = oracle.evolve(psi0, C, T, shift=int(flipflop))
    assert np.abs(got - want).max() < 1e-11


@pytest.mark.parametrize("flipflop", [False, True])
def test_fourier_closed_form_2d(flipflop):
    rng = np.random.default_rng(12)
    C = inputs.random_unitary(4, rng)
    psi0 = inputs.random_state((4, 10, 12), seed=6)   # Ly=10, Lx=12: x/y not symmetric
    want = fourier.evolve_fourier(psi0, C, 23, flipflop=flipflop)
    got = oracle.evolve(psi0, C, 23, shift=int(flipflop))
    assert np.abs(got - want).max() < 1e-11


@pytest.mark.parametrize("coin", ["grover", "hh", "fourier"])
def test_fourier_named_coins_2d(coin):
    C = {"grover": inputs.grover(), "hh": inputs.hadamard2(), "fourier": inputs.fourier()}[coin]
    psi0 = inputs.random_state((4, 16, 16), seed=7)
    for ff in (False, True):
        want = fourier.evolve_fourier(psi0, C, 31, flipflop=ff)
        got = oracle.evolve(psi0, C, 31, shift=int(ff))
        assert np.abs(got - want).max() < 1e-11


# ------------------------------------------------------------ dense brute force
def _check_dense(dims, coins, T, flipflop=False, bc=0, closed=None, phi=None, base=None):
    ns = int(np.prod(dims))
    d = 2 * len(dims)
    shape = (d, ns) if len(dims) == 1 else (d, dims[1], dims[0])
    if phi is not None:
        cm = np.einsum("rc,vc->vrc", base, np.exp(1j * phi))   # B . diag(e^{i phi_v})
    else:
        cm = coins
    U = dense.walk_matrix(dims, cm, flipflop=flipflop, bc=bc, closed=closed)
    if bc != 2:
        assert np.abs(U.conj().T @ U - np.eye(d * ns)).max() < 1e-12
    psi0 = inputs.random_state(shape, seed=ns + T)
    want = dense.apply_power(U, psi0, T)
    if phi is not None:
        got = oracle.evolve(psi0, base, T, shift=int(flipflop), bc=bc, closed=closed, phi=phi)
    else:
        got = oracle.evolve(psi0, coins, T, shift=int(flipflop), bc=bc, closed=closed)
    assert np.abs(got - want).max() < 1e-12
    want_adj = dense.apply_power(U.conj().T, psi0, T)
    if phi is not None:
        got_adj = oracle.evolve(psi0, base, T, shift=int(flipflop), bc=bc, closed=closed,
                                phi=phi, adjoint=True)
    else:
        got_adj = oracle.evolve(psi0, coins, T, shift=int(flipflop), bc=bc, closed=closed,
                                adjoint=True)
    assert np.abs(got_adj - want_adj).max() < 1e-12


@pytest.mark.parametrize("flipflop", [False, True])
def test_dense_per_site_coins_1d(flipflop):
    rng = np.random.default_rng(21)
    N = 9
    coins = np.stack([inputs.random_unitary(2, rng) for _ in range(N)])
    _check_dense((N,), coins, 7, flipflop=flipflop)


@pytest.mark.parametrize("flipflop", [False, True])
def test_dense_per_site_coins_2d(flipflop):
    rng = np.random.default_rng(22)
    dims = (4, 3)
    coins = np.stack([inputs.random_unitary(4, rng) for _ in range(12)])
    _check_dense(dims, coins, 5, flipflop=flipflop)


@pytest.mark.parametrize("flipflop", [False, True])
def test_dense_phase_coins_2d(flipflop):
    rng = np.random.default_rng(23)
    dims = (4, 5)
    phi = rng.uniform(-1, 1, size=(20, 4))
    _check_dense(dims, None, 6, flipflop=flipflop, phi=phi, base=inputs.grover())


@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("flipflop", [False, True])
@pytest.mark.parametrize("ndim", [1, 2])
def test_dense_broken_links_and_boundaries(bc, flipflop, ndim):
    rng = np.random.default_rng(30 + bc + 3 * flipflop + 7 * ndim)
    dims = (11,) if ndim == 1 else (4, 5)
    ns = int(np.prod(dims))
    d = 2 * ndim
    closed = (rng.uniform(size=(ndim, ns)) < 0.3).astype(np.uint8)
    C = inputs.random_unitary(d, rng)
    _check_dense(dims, C, 6, flipflop=flipflop, bc=bc, closed=closed)


def test_dense_closed_per_step():
    rng = np.random.default_rng(41)
    N, T = 10, 5
    masks = (rng.uniform(size=(T, 1, N)) < 0.4).astype(np.uint8)
    C = inputs.random_unitary(2, rng)
    psi0 = inputs.random_state((2, N), seed=3)
    want = psi0.reshape(-1)
    for t in range(T):
        want = dense.walk_matrix((N,), C, closed=masks[t]) @ want
    got = oracle.evolve(psi0, C, T, closed=masks, closed_per_step=True)
    assert np.abs(got.reshape(-1) - want).max() < 1e-12
    back = oracle.evolve(got, C, T, closed=masks, closed_per_step=True, adjoint=True)
    assert np.abs(back - psi0).max() < 1e-12


# ------------------------------------------------------------ links broken at random each step
def test_philox_known_answers():
    """The oracle's Philox4x32-10 reproduces the generator's published
    known-answer vectors (tests/golden/philox4x32_10_kat.txt)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        got = oracle.philox4x32_10(v[0:4], v[4:6])
        assert list(got) == v[6:10]


def test_link_masks_rate_and_independence():
    """Per-step masks: each link closes with probability p (binomial bound), the
    masks of different steps, axes and seeds differ, and the same (seed, step)
    gives the same mask."""
    p, shape = 0.3, (40, 50)
    m = oracle.link_masks(shape, seed=12345, p=p, t0=7, T=6)
    assert m.shape == (6, 2, 2000)
    n = m.size
    assert abs(m.mean() - p) < 5 * np.sqrt(p * (1 - p) / n)
    assert not np.array_equal(m[0], m[1]) and not np.array_equal(m[0, 0], m[0, 1])
    again = oracle.link_masks(shape, seed=12345, p=p, t0=8, T=1)
    assert np.array_equal(again[0], m[1])
    other = oracle.link_masks(shape, seed=12346, p=p, t0=7, T=1)
    assert not np.array_equal(other[0], m[0])
    assert oracle.link_masks(shape, seed=1, p=0.0, t0=0, T=2).sum() == 0
    assert oracle.link_masks(shape, seed=1, p=1.0, t0=0, T=1).all()


def test_link_masks_draw_words_from_the_known_answer_vector():
    """The mask of site 0 at step 0 with seed 0 comes from counter (0, 0, 0, 0)
    and key (0, 0), whose published Philox4x32-10 output starts 6627e8d5
    e169c58d: the x-link takes word 0 and the y-link word 1, each closed exactly
    when the threshold floor(p 2^32) exceeds its word."""
    rows = [ln.split() for ln in open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    zero = [r for r in rows if all(int(x, 16) == 0 for x in r[:6])][0]
    words = [int(zero[6], 16), int(zero[7], 16)]
    for axis, wd in enumerate(words):
        at = oracle.link_masks((1, 1), seed=0, p=wd / 2.0 ** 32, t0=0, T=1)[0, axis, 0]
        above = oracle.link_masks((1, 1), seed=0, p=(wd + 1) / 2.0 ** 32, t0=0, T=1)[0, axis, 0]
        assert (at, above) == (0, 1), axis
    # on the cycle the single link of a site is word 0
    assert oracle.link_masks((1,), seed=0, p=(words[0] + 1) / 2.0 ** 32, t0=0, T=1)[0, 0, 0] == 1
    assert oracle.link_masks((1,), seed=0, p=words[0] / 2.0 ** 32, t0=0, T=1)[0, 0, 0] == 0


# ------------------------------------------------------------ invariants
def test_norm_every_step_and_reversibility():
    rng = np.random.default_rng(51)
    C = inputs.random_unitary(4, rng)
    psi = inputs.random_state((4, 12, 12), seed=8)
    psi0 = psi.copy()
    for _ in range(20):
        psi = oracle.evolve(psi, C, 1)
        _, norm = oracle.probabilities(psi)
        assert abs(norm - 1.0) < 1e-13
    back = oracle.evolve(psi, C, 20, adjoint=True)
    assert np.abs(back - psi0).max() < 1e-13


def test_inner_products_preserved():
    rng = np.random.default_rng(52)
    C = inputs.random_unitary(2, rng)
    a = inputs.random_state((2, 300), seed=9)
    b = inputs.random_state((2, 300), seed=10)
    Ua, Ub = oracle.evolve(a, C, 37), oracle.evolve(b, C, 37)
    assert abs(np.vdot(Ua, Ub) - np.vdot(a, b)) < 1e-13
    # adjoint identity <lambda, U psi> = <U^dagger lambda, psi>
    assert abs(np.vdot(b, Ua) - np.vdot(oracle.evolve(b, C, 37, adjoint=True), a)) < 1e-13


def test_2d_parity_and_symmetry_grover():
    """Grover walk from the origin with (|0>-|1>-|2>+|3>)/2, moving shift, even L:
    amplitude only where x+y = T (mod 2).  Swapping x<->y maps the coin state to
    minus itself, and so does the point inversion (x,y)->(-x,-y); the Grover coin
    commutes with both relabellings, so P(x,y) = P(y,x) = P(-x,-y).  (The mirror
    x->-x alone does not map the state to +-itself and is not a symmetry.)"""
    L, T = 64, 30
    psi = oracle.evolve(inputs.localized_2d(L), inputs.grover(), T)
    P, norm = oracle.probabilities(psi)
    assert abs(norm - 1) < 1e-13
    y, x = np.mgrid[0:L, 0:L]
    assert np.all(P[(x + y - T) % 2 != 0] == 0)
    neg = (-np.arange(L)) % L
    assert np.abs(P - P.T).max() < 1e-15
    assert np.abs(P - P[neg][:, neg]).max() < 1e-15
    # the maximally spreading state of this basis, (|0>+|1>-|2>-|3>)/2, has the
    # full D4 symmetry and leaves almost nothing at the origin
    psi = oracle.evolve(inputs.localized_2d(L, coin_state=(.5, .5, -.5, -.5)), inputs.grover(), T)
    P, _ = oracle.probabilities(psi)
    assert np.abs(P - P[:, neg]).max() < 1e-15
    assert np.abs(P - P.T).max() < 1e-15
    assert P[0, 0] < 1e-3


def test_paper_coin_labelling_matches_after_permutation():
    """The paper's shift equation labels coin (j,k), c=2j+k, with moves
    (0,0)->+n, (0,1)->+m, (1,0)->-m, (1,1)->-n.  With (m,n) = (x,y) this is our
    walk after relabelling the coin basis: paper c -> ours pi[c]."""
    paper_dirs = [(0, 1), (1, 0), (-1, 0), (0, -1)]
    pi = [2, 0, 1, 3]
    rng = np.random.default_rng(61)
    Cp = inputs.random_unitary(4, rng)
    dims = (5, 4)
    psi_p = inputs.random_state((4, 4, 5), seed=12)
    want = dense.apply_power(dense.walk_matrix(dims, Cp, dirs=paper_dirs), psi_p, 6)
    Pm = np.zeros((4, 4))
    for c in range(4):
        Pm[pi[c], c] = 1
    C_ours = Pm @ Cp @ Pm.T
    psi_ours = np.empty_like(psi_p)
    for c in range(4):
        psi_ours[pi[c]] = psi_p[c]
    got = oracle.evolve(psi_ours, C_ours, 6)
    for c in range(4):
        assert np.abs(got[pi[c]] - want[c]).max() < 1e-12


def test_light_cone_window_equals_full_lattice():
    """psi_T at one site depends only on the 2T+1 sites around it: a cycle
    (torus) of side 2T+1 cut out around it gives the same value exactly."""
    rng = np.random.default_rng(71)
    C = inputs.random_unitary(2, rng)
    N, T, x = 500, 40, 17
    psi0 = inputs.random_state((2, N), seed=13)
    full = oracle.evolve(psi0, C, T)
    idx = (x + np.arange(-T, T + 1)) % N
    win = oracle.evolve(psi0[:, idx], C, T)
    assert np.abs(win[:, T] - full[:, x]).max() < 1e-14
    C4 = inputs.random_unitary(4, rng)
    L, T2, (x2, y2) = 40, 8, (3, 30)
    psi2 = inputs.random_state((4, L, L), seed=14)
    full2 = oracle.evolve(psi2, C4, T2)
    ix = (x2 + np.arange(-T2, T2 + 1)) % L
    iy = (y2 + np.arange(-T2, T2 + 1)) % L
    win2 = oracle.evolve(psi2[:, iy][:, :, ix], C4, T2)
    assert np.abs(win2[:, T2, T2] - full2[:, y2, x2]).max() < 1e-14


# ------------------------------------------------------------ gradient
def _loss(psi0, base, phi, T, rect):
    psi = oracle.evolve(psi0, base, T, phi=phi.reshape(-1, 4))
    x0, y0, w, h = rect
    return float((np.abs(psi[:, y0:y0 + h, x0:x0 + w]) ** 2).sum())


def test_region_grad_matches_central_differences():
    L, T = 8, 6
    rng = np.random.default_rng(81)
    phi = rng.uniform(-0.5, 0.5, size=(L, L, 4))
    psi0 = inputs.random_state((4, L, L), seed=15)
    base = inputs.grover()
    rect = (2, 3, 3, 2)
    loss, g = oracle.region_grad(psi0, base, phi, T, rect)
    assert abs(loss - _loss(psi0, base, phi, T, rect)) < 1e-14
    h = 1e-5
    for (y, x, k) in [(0, 0, 0), (3, 2, 1), (5, 7, 2), (4, 4, 3), (1, 6, 1), (7, 3, 0)]:
        pp, pm = phi.copy(), phi.copy()
        pp[y, x, k] += h
        pm[y, x, k] -= h
        fd = (_loss(psi0, base, pp, T, rect) - _loss(psi0, base, pm, T, rect)) / (2 * h)
        assert abs(fd - g[y, x, k]) < 1e-8


def test_region_grad_zero_outside_past_light_cone():
    L, T = 32, 5
    phi = inputs.region_grad_phases(L, seed=3)
    psi0 = inputs.random_state((4, L, L), seed=16)
    rect = (14, 14, 4, 4)
    _, g = oracle.region_grad(psi0, inputs.grover(), phi, T, rect)
    y, x = np.mgrid[0:L, 0:L]
    # a phase at v can only influence sites within distance T-1 ... T of v
    dist = np.maximum(np.maximum(14 - x, x - 17), 0) + np.maximum(np.maximum(14 - y, y - 17), 0)
    far = dist > T
    assert np.all(g[far] == 0.0)
    assert np.abs(g[~far]).max() > 1e-6


# ------------------------------------------------------------ the pins have teeth
MUTATIONS = {
    "transposed_coin": ("acc += C[r * d + c] * in[(size_t)v * d + c];",
                        "acc += C[c * d + r] * in[(size_t)v * d + c];"),
    "wrong_direction_1d": ("sgn = (c == 0) ? -1 : +1; }", "sgn = (c == 0) ? +1 : -1; }"),
    "dropped_phase": ("cplx e = cos(a) + I * sin(a);", "cplx e = 1.0;"),
    "reflect_wrong_slot": ("*co = L->shift == 1 ? c : (c ^ 1); return 1; }",
                           "*co = c; return 1; }"),
    "adjoint_no_conj": ("acc += conj(C[c * d + r]) * g[c];", "acc += C[c * d + r] * g[c];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes_are_caught(name, tmp_path, monkeypatch):
    """Plant one mistake in a copy of the oracle source (CPU only) and check
    that the pins above reject it."""
    import ctypes
    import subprocess
    src = open(oracle._SRC).read()
    old, new = MUTATIONS[name]
    assert old in src
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-std=c11", "-O1", "-ffp-contract=off", "-fPIC", "-shared",
                    str(mut), "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    real = oracle._lib(False)
    lib.oracle_evolve.argtypes = real.oracle_evolve.argtypes
    lib.oracle_probabilities.argtypes = real.oracle_probabilities.argtypes
    lib.oracle_region_grad.argtypes = real.oracle_region_grad.argtypes
    monkeypatch.setitem(oracle._LIBS, False, lib)
    checks = [
        lambda: test_fourier_closed_form_1d(64, 20, False),
        lambda: test_fourier_closed_form_2d(False),
        lambda: test_dense_phase_coins_2d(False),
        lambda: test_dense_broken_links_and_boundaries(1, False, 1),
        lambda: test_dense_per_site_coins_1d(False),
    ]
    failures = 0
    for chk in checks:
        try:
            chk()
        except AssertionError:
            failures += 1
    assert failures > 0, f"mutation {name} passed every pin"


# ------------------------------------------------------------ diagonal lattice
def test_diagonal_lattice_factorises_for_hadamard_coins():
    """H (x) H on the diagonal lattice: qubit j drives x, qubit k drives y, so a
    product start stays a product of two 1D Hadamard walks (each mirrored: coin 0
    moves +1 here, -1 on the cycle):  P(x, y) = P1(-x) P1(-y)."""
    L, T = 41, 17
    a = (0.6, 0.8j)
    b = (1 / np.sqrt(2), -1 / np.sqrt(2))
    psi = np.zeros((4, L, L), dtype=complex)
    for j in range(2):
        for k in range(2):
            psi[2 * j + k, 0, 0] = a[j] * b[k]
    P, _ = oracle.probabilities(oracle.evolve(psi, inputs.hadamard2(), T, shift=2))
    Px, _ = oracle.probabilities(oracle.evolve(inputs.localized_1d(L, 0, a), inputs.hadamard(), T))
    Py, _ = oracle.probabilities(oracle.evolve(inputs.localized_1d(L, 0, b), inputs.hadamard(), T))
    neg = (-np.arange(L)) % L
    assert np.abs(P - np.outer(Py[neg], Px[neg])).max() < 1e-14


@pytest.mark.parametrize("coin", ["fourier", "grover", "random"])
def test_diagonal_lattice_fourier_and_dense(coin):
    rng = np.random.default_rng(91)
    C = {"fourier": inputs.fourier(), "grover": inputs.grover(),
         "random": inputs.random_unitary(4, rng)}[coin]
    psi0 = inputs.random_state((4, 6, 9), seed=92)
    want = fourier.evolve_fourier(psi0, C, 13, diagonal=True)
    got = oracle.evolve(psi0, C, 13, shift=2)
    assert np.abs(got - want).max() < 1e-12
    U = dense.diagonal_shift_matrix((9, 6)) @ dense.coin_matrix(C, 54, 4)
    assert np.abs(dense.apply_power(U, psi0, 5) - oracle.evolve(psi0, C, 5, shift=2)).max() < 1e-12
    assert np.abs(dense.apply_power(U.conj().T, psi0, 5) -
                  oracle.evolve(psi0, C, 5, shift=2, adjoint=True)).max() < 1e-12
