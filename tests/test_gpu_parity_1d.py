"""GPU parity on the cycle: the CUDA path (through the C ABI) against the FP64
oracle, element by element, on seeded inputs."""
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


def run_gpu(qw, psi0, coin, T, prec, shift=0, plan=None, per_site=False, phases=None, adjoint=False):
    w = qw.Walk((psi0.shape[1],), prec=prec, shift=shift)
    if phases is not None:
        w.set_coin_phases(coin, phases)
    else:
        w.set_coin(coin, per_site=per_site)
    if plan is not None:
        w.set_plan(*plan)
    w.set_state(psi0)
    if adjoint:
        w.step_adjoint(T)
    else:
        w.step(T)
    out = w.state()
    P, norm = w.probabilities()
    k = w.plan()[0]
    w.close()
    return out, P, norm, k


@pytest.mark.parametrize("prec", PRECS)
def test_hadamard_cycle_2001_T1000(qw, prec):
    N, T = 2001, 1000
    psi0 = inputs.localized_1d(N)
    want = oracle.evolve(psi0, inputs.hadamard(), T)
    Pw, _ = oracle.probabilities(want)
    got, P, norm, k = run_gpu(qw, psi0, inputs.hadamard(), T, prec)
    assert maxabs(got, want) < amp_tol(prec, T, k)
    assert l1(P, Pw) < p_l1_tol(prec, T, N, k)
    if prec in ("f64", "comp", "f32"):
        # parity zeros are exact on every path: zero amplitudes stay zero
        xs = np.where(np.arange(N) <= N // 2, np.arange(N), np.arange(N) - N)
        assert np.all(P[(xs - T) % 2 != 0] == 0.0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [1, 2, 5, 63, 1000, 5003, 70001])
def test_random_state_complex_coin(qw, prec, N):
    rng = np.random.default_rng(N)
    C = inputs.random_unitary(2, rng)
    psi0 = inputs.random_state((2, N), seed=N + 1)
    T = 37
    want = oracle.evolve(psi0, C, T)
    got, P, _, k = run_gpu(qw, psi0, C, T, prec)
    assert maxabs(got, want) < amp_tol(prec, T, k)
    assert l1(P, oracle.probabilities(want)[0]) < p_l1_tol(prec, T, N, k)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("plan", [(1, 0), (3, 0), (5, "A"), ("max", "A"), ("max", "B")])
def test_plans_and_shifts(qw, prec, shift, plan):
    N, T = 9001, 101
    ta, tb = (4, 8) if prec in ("f64", "comp") else (8, 16)
    tile = {0: 0, "A": ta, "B": tb}[plan[1]]
    k = plan[0]
    if k == "max":
        k = 8 * (tile or (8 if prec == "f64" else 4 if prec == "comp" else 16))
    C = inputs.su2(0.3, 0.2, -0.5)
    psi0 = inputs.random_state((2, N), seed=3)
    want = oracle.evolve(psi0, C, T, shift=shift)
    got, P, _, kk = run_gpu(qw, psi0, C, T, prec, shift=shift, plan=(k, tile))
    assert kk == k
    assert maxabs(got, want) < amp_tol(prec, T, k)


@pytest.mark.parametrize("prec", PRECS)
def test_real_coin_su2_theta_pi4(qw, prec):
    N, T = 20000, 300
    C = inputs.su2(np.pi / 4)
    psi0 = inputs.random_state((2, N), seed=1)
    want = oracle.evolve(psi0, C, T)
    got, P, _, k = run_gpu(qw, psi0, C, T, prec)
    assert maxabs(got, want) < amp_tol(prec, T, k)
    assert l1(P, oracle.probabilities(want)[0]) < p_l1_tol(prec, T, N, k)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shift", [0, 1])
def test_per_site_coins(qw, prec, shift):
    N, T = 777, 25
    rng = np.random.default_rng(5)
    coins = np.stack([inputs.random_unitary(2, rng) for _ in range(N)])
    psi0 = inputs.random_state((2, N), seed=6)
    want = oracle.evolve(psi0, coins, T, shift=shift)
    got, _, _, k = run_gpu(qw, psi0, coins, T, prec, shift=shift, per_site=True)
    assert maxabs(got, want) < amp_tol(prec, T, k)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_phase_coins_1d(qw, prec):
    N, T = 513, 40
    rng = np.random.default_rng(8)
    phi = rng.uniform(-1, 1, size=(N, 2)).astype(np.float32)
    base = inputs.hadamard()
    psi0 = inputs.random_state((2, N), seed=9)
    want = oracle.evolve(psi0, base, T, phi=phi.astype(np.float64))
    got, _, _, k = run_gpu(qw, psi0, base, T, prec, phases=phi)
    assert maxabs(got, want) < amp_tol(prec, T, k) + T * 1e-7  # phases are float inputs


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("per_site", [False, True])
def test_adjoint_matches_oracle_and_inverts(qw, prec, shift, per_site):
    N, T = 3001, 50
    rng = np.random.default_rng(10)
    C = (np.stack([inputs.random_unitary(2, rng) for _ in range(N)]) if per_site
         else inputs.random_unitary(2, rng))
    psi0 = inputs.random_state((2, N), seed=11)
    want = oracle.evolve(psi0, C, T, shift=shift, adjoint=True)
    got, _, _, k = run_gpu(qw, psi0, C, T, prec, shift=shift, per_site=per_site, adjoint=True)
    assert maxabs(got, want) < amp_tol(prec, T, k)
    # U^T then (U^dagger)^T returns the start
    w = qw.Walk((N,), prec=prec, shift=shift).set_coin(C, per_site=per_site).set_state(psi0)
    w.step(T).step_adjoint(T)
    assert maxabs(w.state(), psi0) < 2 * amp_tol(prec, T, k)
    w.close()


def test_step_zero_and_norm_reproducible(qw):
    N = 4096
    psi0 = inputs.random_state((2, N), seed=12)
    w = qw.Walk((N,), prec="f32").set_coin(inputs.hadamard()).set_state(psi0)
    w.step(0)
    assert maxabs(w.state(), psi0) < 1e-7
    w.step(333)
    n1, n2 = w.norm(), w.norm()
    assert n1 == n2   # fixed-order double reduction: bitwise identical
    # random rounding only: the coin's systematic drift is compensated
    assert abs(n1 - 1) < 333 * 4 * 2.0 ** -24
    w.close()


def test_device_buffers_and_streams(qw):
    import torch
    N, T = 10000, 64
    C = inputs.su2(0.7)
    psi0 = inputs.random_state((2, N), seed=13)
    want = oracle.evolve(psi0, C, T)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        dev = torch.from_numpy(psi0.astype(np.complex64)).cuda()
        w = qw.Walk((N,), prec="f32").set_coin(C)
        w.set_state(dev)
        w.step(T)
        out = torch.empty_like(dev)
        qw.qw_get_state(w.h, out)
        P = torch.empty(N, dtype=torch.float32, device="cuda")
        norm = qw.qw_probabilities(w.h, P)
    s.synchronize()
    assert maxabs(out.cpu().numpy(), want) < amp_tol("f32", T)
    assert l1(P.cpu().numpy(), oracle.probabilities(want)[0]) < 1e-4
    assert abs(norm - 1) < 1e-5
    w.close()


def test_autotune_keeps_state_and_picks_a_valid_plan(qw):
    N = 1 << 20
    psi0 = inputs.random_state((2, N), seed=14)
    w = qw.Walk((N,), prec="f32").set_coin(inputs.su2(np.pi / 4)).set_state(psi0)
    rep = w.autotune()
    assert '"tuned": true' in rep
    k, tile, variant = w.plan_ex()
    # the tile kernel takes k <= 8 * tile; the sweep kernel k < chunk / 2 = 16 * tile
    assert 1 <= k <= (8 * tile if variant == 0 else 16 * tile - 1)
    assert maxabs(w.state(), psi0) < 1e-7   # tuning wrote only the scratch buffer
    w.close()


def test_bounded_wait_times_out_without_hanging(qw):
    assert qw.qw_debug_bounded_wait(2000) == qw.QW_ETIMEOUT
    # the context is still usable afterwards
    w = qw.Walk((64,), prec="f32").set_coin(inputs.hadamard()).set_state(inputs.localized_1d(64))
    w.step(3)
    assert abs(w.norm() - 1) < 1e-6
    w.close()


SIGN_PATTERNS = [(a, b, c) for a in (1, -1) for b in (1, -1) for c in (1, -1)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("m00,m01,m10", SIGN_PATTERNS)
def test_hadamard_class_coins(qw, prec, m00, m01, m10):
    """Coins lambda * M with M a +-1 matrix take the addition-only kernel; every
    sign pattern, forward and backward, several depths, against the oracle."""
    M = np.array([[m00, m01], [m10, -m10 * m01 * m00]], dtype=float)
    C = (M / np.sqrt(2)).astype(np.complex128)
    N, T = 4099, 77
    psi0 = inputs.random_state((2, N), seed=15)
    for adj in (False, True):
        want = oracle.evolve(psi0, C, T, adjoint=adj)
        for k in (1, 2, 7, 32):
            w = qw.Walk((N,), prec=prec).set_coin(C).set_plan(k)
            assert w.describe()["coin_kind"] == "hadamard_class"
            w.set_state(psi0)
            (w.step_adjoint if adj else w.step)(T)
            assert maxabs(w.state(), want) < amp_tol(prec, T, k), (adj, k)
            w.close()


def test_describe_reports_the_kernel_path(qw):
    w = qw.Walk((1000,), prec="f32").set_coin(inputs.su2(np.pi / 4))
    assert w.describe()["path"] == "k_step1d_sweep"      # at least one 512-site chunk
    w.close()
    w = qw.Walk((300,), prec="f32").set_coin(inputs.su2(np.pi / 4))
    d = w.describe()
    assert d["coin_kind"] == "hadamard_class" and d["path"] == "k_step1d"
    w.set_coin(inputs.su2(0.3))
    assert w.describe()["coin_kind"] == "real"
    w.set_coin(inputs.su2(0.3, 0.1))
    assert w.describe()["coin_kind"] == "complex"
    w.close()
    w = qw.Walk((1000,), prec="f32", shift=1).set_coin(inputs.hadamard())
    assert w.describe()["coin_kind"] == "real"    # flip-flop keeps the general kernel
    w.close()


@pytest.mark.parametrize("theta", [np.pi / 4, 0.3])
def test_norm_drift_compensated_long_run(qw, theta):
    """FP32 at T = 4096: the rounded coin's systematic norm drift is removed."""
    N, T = 1 << 16, 4096
    psi0 = inputs.random_state((2, N), seed=16)
    w = qw.Walk((N,), prec="f32").set_coin(inputs.su2(theta)).set_state(psi0)
    w.step(T)
    # unbiased rounding only: well inside T * u
    assert abs(w.norm() - 1) < 4096 * 2.0 ** -24 / 4
    w.close()


# (precision, N, sites per lane): both compiled tiles of the float forms (chunks
# of 512 and 1024 sites), several segments with a short last one, one-chunk cycles,
# and cycles whose last chunk runs past site N - 1 (odd N too)
SWEEP_CASES = [("f32", 512 * 37, 16), ("f32", 512, 16), ("f32", 1024 * 19, 32), ("f32", 1024, 32),
               ("f32", 1024 * 19 + 333, 32), ("f32", 512 * 3 + 1, 16), ("f32", 1024 + 7, 32),
               ("bf16", 512 * 21, 16), ("bf16", 1024 * 11, 32), ("bf16", 1024 * 11 + 3, 32),
               ("f64", 256 * 35, 8), ("f64", 256 * 35 + 101, 8)]
SWEEP_COINS = {"hadamard_class": inputs.su2(np.pi / 4), "real": inputs.su2(0.3),
               "complex": inputs.su2(0.3, 0.2, -0.5)}


def _sweep_against_oracle(qw, prec, N, tile, k, coin, shift, adj):
    C = SWEEP_COINS[coin]
    T = 3 * k + 5
    psi0 = inputs.random_state((2, N), seed=17)
    want = oracle.evolve(psi0, C, T, shift=shift, adjoint=adj)
    w = qw.Walk((N,), prec=prec, shift=shift).set_coin(C)
    w.set_plan_ex(k, tile, 1)
    assert w.plan_ex() == (k, tile, 1) and w.describe()["path"] == "k_step1d_sweep"
    w.set_state(psi0)
    (w.step_adjoint if adj else w.step)(T)
    assert maxabs(w.state(), want) < amp_tol(prec, T, k)
    w.close()


@pytest.mark.parametrize("prec,N,tile", SWEEP_CASES)
@pytest.mark.parametrize("k", [2, 3, 17, 64, 127])
@pytest.mark.parametrize("coin", list(SWEEP_COINS))
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("adj", [False, True])
def test_sweep_kernel(qw, prec, N, tile, k, coin, shift, adj):
    """The time-skewed sweep (variant 1) against the oracle: several segments, a
    short last segment, one-chunk cycles, odd and large depths, all coin classes."""
    _sweep_against_oracle(qw, prec, N, tile, k, coin, shift, adj)


@pytest.mark.parametrize("prec,N,tile", [c for c in SWEEP_CASES if c[2] >= 16])
@pytest.mark.parametrize("k", [160, 255, 256, 400, 511])
@pytest.mark.parametrize("coin", ["hadamard_class", "complex"])
@pytest.mark.parametrize("adj", [False, True])
def test_sweep_kernel_deep(qw, prec, N, tile, k, coin, adj):
    """Depths up to the largest each tile takes (k < chunk / 2): the warm-up
    chunk's error front and the edge buffer at their limits."""
    if k > 16 * tile - 1:
        pytest.skip("deeper than this tile takes")
    _sweep_against_oracle(qw, prec, N, tile, k, coin, 0, adj)


def test_sweep_default_tile_follows_the_cycle_length(qw):
    for N, tile in ((1024 * 5, 32), (2048, 32), (2047, 16), (700, 16)):
        w = qw.Walk((N,), prec="f32").set_coin(inputs.hadamard())
        w.set_plan_ex(64, 0, 1)
        assert w.plan_ex() == (64, tile, 1)
        w.close()


def test_sweep_rejected_where_it_cannot_run(qw):
    w = qw.Walk((500,), prec="f32").set_coin(inputs.hadamard())
    with pytest.raises(qw.QWError):
        w.set_plan_ex(16, 0, 1)          # 500 sites are less than one 512-site chunk
    w.close()
    w = qw.Walk((1000,), prec="f32").set_coin(inputs.hadamard())
    with pytest.raises(qw.QWError):
        w.set_plan_ex(16, 32, 1)         # ... or one 1024-site chunk
    with pytest.raises(qw.QWError):
        w.set_plan_ex(256, 16, 1)        # k must stay below half the 512-site chunk
    w.close()
    w = qw.Walk((1024 * 3,), prec="f32").set_coin(inputs.hadamard())
    with pytest.raises(qw.QWError):
        w.set_plan_ex(512, 32, 1)        # k must stay below half the 1024-site chunk
    w.close()
    w = qw.Walk((1024,), prec="comp").set_coin(inputs.hadamard())
    with pytest.raises(qw.QWError):
        w.set_plan_ex(16, 0, 1)          # no sweep kernel for the double-float form
    w.close()


@pytest.mark.parametrize("prec", ["f64"])
def test_near_hadamard_coin_runs_as_given_in_double(qw, prec):
    """A coin a few double ulps away from 1/sqrt2 * [[1, 1], [1, -1]] is applied
    as given in the double form (not replaced by the exact Hadamard-class
    kernel): at T = 4096 the result follows the oracle of the
    perturbed coin, whose distance to the unperturbed walk is far above the
    rounding error."""
    N, T = 2048, 4096
    C = inputs.hadamard().copy()
    C[0, 0] += 5e-15
    psi0 = inputs.random_state((2, N), seed=61)
    want = oracle.evolve(psi0, C, T)
    exact = oracle.evolve(psi0, inputs.hadamard(), T)
    gap = maxabs(want, exact)
    w = qw.Walk((N,), prec=prec).set_coin(C)
    assert w.describe()["coin_kind"] == "real"
    w.set_state(psi0).step(T)
    got = w.state()
    P, _ = w.probabilities()
    w.close()
    assert maxabs(got, want) < gap / 8, (maxabs(got, want), gap)
    if prec == "f64":
        assert l1(P, oracle.probabilities(want)[0]) < 1e-12
    # the exact coin still takes the addition-only kernel
    w = qw.Walk((N,), prec=prec).set_coin(inputs.hadamard())
    assert w.describe()["coin_kind"] == "hadamard_class"
    w.close()
