"""Light-cone clipping of localised states (the growing computation window of
the paper's line walk, Sec. 3): the clipped steps give every amplitude of the
full-lattice steps with the same plan, bit for bit, and match the FP64 oracle;
the support box the library tracks is the light cone."""
import numpy as np
import pytest

import oracle
from paper_1003_3779_gb300 import inputs
from tests.helpers import amp_tol, maxabs

pytestmark = pytest.mark.gpu

PRECS = ["f64", "f32", "bf16", "comp"]


@pytest.fixture(scope="module")
def qw():
    import paper_1003_3779_gb300.qw as qw
    qw.lib()
    return qw


def run(qw, dims, psi0, T, clip, prec="f32", shift=0, coin=None, plan=None, adjoint=False, per_site=None,
        phases=None, chunks=None):
    """State and P after T steps (in `chunks` calls of qw_step when given)."""
    w = qw.Walk(dims, prec=prec, shift=shift).set_clipping(clip)
    if phases is not None:
        w.set_coin_phases(coin, phases)
    elif per_site is not None:
        w.set_coin(per_site, per_site=True)
    else:
        w.set_coin(coin)
    if plan is not None:
        w.set_plan_ex(*plan) if len(dims) == 1 else w.set_plan(plan)
    w.set_state(psi0)
    for Tc in (chunks or [T]):
        (w.step_adjoint if adjoint else w.step)(Tc)
    desc = w.describe()
    out = w.state()
    P, _ = w.probabilities()
    w.close()
    return out, P, desc


def same(a, b):
    """Equal values (a zero may carry either sign)."""
    return np.array_equal(a, b)


# ---------------------------------------------------------------- 1D
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("k", [1, 7, 32])
def test_hadamard_cycle_2001_from_site_0(qw, prec, k):
    """The small configuration (Hadamard, N = 2001, x0 = 0, T = 1000): the
    window wraps round site 0 at once and covers the cycle at T = 1000."""
    N, T = 2001, 1000
    psi0 = inputs.localized_1d(N)
    tile = 8 if prec in ("f64", "comp") else 16
    on = run(qw, (N,), psi0, T, True, prec, coin=inputs.hadamard(), plan=(k, tile, 0))
    off = run(qw, (N,), psi0, T, False, prec, coin=inputs.hadamard(), plan=(k, tile, 0))
    assert same(on[0], off[0]) and same(on[1], off[1])
    assert off[2]["support"] == "full"
    want = oracle.evolve(psi0, inputs.hadamard(), T)
    assert maxabs(on[0], want) < amp_tol(prec, T, k)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("adjoint", [False, True])
def test_cycle_window_grows_then_covers(qw, prec, shift, adjoint):
    """A complex coin from x0 = 4000 on N = 5003, in calls of 40, 300 and 2400
    steps: the support box after the second call is [x0 - 340, x0 + 340]; after
    the third (2 * 2740 + 1 > N) it covers the cycle."""
    N, x0 = 5003, 4000
    C = inputs.su2(0.3, 0.4, -0.7)
    psi0 = inputs.localized_1d(N, x0, (0.6, 0.8j))
    plan = (24, 8 if prec in ("f64", "comp") else 16, 0)
    kw = dict(coin=C, plan=plan, shift=shift, adjoint=adjoint)
    on = run(qw, (N,), psi0, 0, True, prec, chunks=[40, 300], **kw)
    off = run(qw, (N,), psi0, 0, False, prec, chunks=[40, 300], **kw)
    assert same(on[0], off[0]) and same(on[1], off[1])
    assert on[2]["support"] == [x0 - 340, 681, 0, 1]
    want = oracle.evolve(psi0, C, 340, shift=shift, adjoint=adjoint)
    assert maxabs(on[0], want) < amp_tol(prec, 340, 24)
    on = run(qw, (N,), psi0, 0, True, prec, chunks=[40, 300, 2400], **kw)
    off = run(qw, (N,), psi0, 0, False, prec, chunks=[40, 300, 2400], **kw)
    assert same(on[0], off[0]) and on[2]["support"] == "full"


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_cycle_per_site_coins_clipped(qw, prec):
    N, T, x0 = 3000, 700, 1500
    rng = np.random.default_rng(31)
    coins = np.stack([inputs.random_unitary(2, rng) for _ in range(N)])
    psi0 = inputs.localized_1d(N, x0)
    on = run(qw, (N,), psi0, T, True, prec, per_site=coins, plan=(16, 16 if prec == "f32" else 8, 0))
    off = run(qw, (N,), psi0, T, False, prec, per_site=coins, plan=(16, 16 if prec == "f32" else 8, 0))
    assert same(on[0], off[0])
    assert maxabs(on[0], oracle.evolve(psi0, coins, T)) < amp_tol(prec, T)


def test_cycle_default_plan_matches_the_full_sweep(qw):
    """With the default plan the full walk runs the sweep kernel and the clipped
    one the warp tiles; the two agree to rounding, and both match the oracle."""
    N, T, x0 = 40000, 1500, 100
    C = inputs.su2(0.3)
    psi0 = inputs.localized_1d(N, x0)
    on = run(qw, (N,), psi0, T, True, "f32", coin=C)
    off = run(qw, (N,), psi0, T, False, "f32", coin=C)
    want = oracle.evolve(psi0, C, T)
    assert maxabs(on[0], want) < amp_tol("f32", T) and maxabs(off[0], want) < amp_tol("f32", T)
    assert on[2]["support"] == [N - (T - x0), 2 * T + 1, 0, 1]


def test_dense_and_wrapped_states_step_in_full(qw):
    N = 4096
    w = qw.Walk((N,), prec="f32").set_coin(inputs.hadamard())
    w.set_state(inputs.random_state((2, N), seed=3)).step(5)
    assert w.describe()["support"] == "full"
    psi = np.zeros((2, N), dtype=complex)
    psi[0, 2] = 0.6
    psi[1, N - 3] = 0.8
    w.set_state(psi).step(5)          # support {2, N-3}: its bounding box is the cycle
    assert w.describe()["support"] == "full"
    assert maxabs(w.state(), oracle.evolve(psi, inputs.hadamard(), 5)) < amp_tol("f32", 5)
    w.set_state(np.zeros((2, N), dtype=complex)).step(9)
    assert np.all(w.state() == 0)
    w.close()


def test_second_set_state_replaces_the_window(qw):
    N = 5000
    w = qw.Walk((N,), prec="f32").set_coin(inputs.hadamard()).set_plan_ex(8, 16, 0)
    w.set_state(inputs.localized_1d(N, 100))
    w.set_state(inputs.localized_1d(N, 3000)).step(20)
    assert w.describe()["support"] == [2980, 41, 0, 1]
    assert maxabs(w.state(), oracle.evolve(inputs.localized_1d(N, 3000), inputs.hadamard(), 20)) < 1e-5
    w.close()


# ---------------------------------------------------------------- 2D
COINS2 = {"grover": inputs.grover(), "hh": inputs.hadamard2(),
          "complex": inputs.random_unitary(4, np.random.default_rng(77))}


@pytest.mark.parametrize("k", [1, 4, 8])
@pytest.mark.parametrize("coin", list(COINS2))
@pytest.mark.parametrize("shift", [0, 1, 2])
@pytest.mark.parametrize("start", [(0, 0), (150, 70)])
def test_torus_clipped_bitwise(qw, k, coin, shift, start):
    """A 200 x 130 torus (rows and columns not multiples of the tiles), from a
    corner (the window wraps at once) or an interior site, T = 45 (the box stays
    inside the torus) and T = 120 (it covers both axes), the fused step (k = 1)
    and the streaming kernel (k = 4, 8); moving, flip-flop and diagonal."""
    Lx, Ly = 200, 130
    C = COINS2[coin]
    psi0 = inputs.localized_2d(Lx, start[0], start[1], (0.5, -0.5j, 0.5, 0.5j), Ly=Ly)
    for T in (45, 120):
        on = run(qw, (Lx, Ly), psi0, T, True, "f32", shift=shift, coin=C, plan=k)
        off = run(qw, (Lx, Ly), psi0, T, False, "f32", shift=shift, coin=C, plan=k)
        assert same(on[0], off[0]) and same(on[1], off[1]), T
        want = oracle.evolve(psi0, C, T, shift=shift)
        assert maxabs(on[0], want) < amp_tol("f32", T), T
        if T == 45:
            assert on[2]["support"] == [(start[0] - 45) % Lx, 91, (start[1] - 45) % Ly, 91]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("adjoint", [False, True])
def test_torus_clipped_precisions_and_adjoint(qw, prec, adjoint):
    L, T = 256, 77
    psi0 = inputs.localized_2d(L, 30, 200)
    on = run(qw, (L, L), psi0, T, True, prec, coin=inputs.grover(), adjoint=adjoint)
    off = run(qw, (L, L), psi0, T, False, prec, coin=inputs.grover(), adjoint=adjoint)
    assert same(on[0], off[0]) and same(on[1], off[1])
    want = oracle.evolve(psi0, inputs.grover(), T, adjoint=adjoint)
    assert maxabs(on[0], want) < amp_tol(prec, T, 1)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_torus_phase_coins_clipped(qw, prec):
    L, T = 128, 50
    phi = inputs.region_grad_phases(L, seed=8).reshape(-1, 4).astype(np.float32)
    psi0 = inputs.localized_2d(L, 64, 64)
    on = run(qw, (L, L), psi0, T, True, prec, coin=inputs.grover(), phases=phi)
    off = run(qw, (L, L), psi0, T, False, prec, coin=inputs.grover(), phases=phi)
    assert same(on[0], off[0])


def test_region_gradient_with_clipping(qw):
    """The region-mass gradient (forward with checkpoints on the clipped steps,
    then the adjoint sweep) equals the one with clipping off."""
    import torch
    L, T, K = 64, 40, 8
    phi = inputs.region_grad_phases(L, seed=9).reshape(-1, 4).astype(np.float32)
    psi0 = inputs.localized_2d(L, 20, 20)
    rect = (16, 16, 8, 8)
    out = []
    for clip in (True, False):
        w = qw.Walk((L, L), prec="f32").set_clipping(clip).set_coin_phases(inputs.grover(), phi).set_state(psi0)
        g = torch.empty((L * L, 4), dtype=torch.float64, device="cuda")
        loss = qw.qw_backward(w.h, rect, T, K, g)
        out.append((loss, g.cpu().numpy(), w.state()))
        w.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


def test_torus_8192_localized_sampled(qw):
    """The torus of the benchmark (8192^2, Grover, k = 8) from the centre for
    T = 256: the window never covers the lattice; the whole light cone against
    the oracle (on a torus of 2T + 1 sites a side, which the walk from its
    centre does not wrap in T steps), zeros outside."""
    import torch
    L, T = 8192, 256
    c = L // 2
    w = qw.Walk((L, L), prec="f32").set_coin(inputs.grover()).set_plan(8)
    full = torch.zeros((4, L, L), dtype=torch.complex64, device="cuda")
    for k in range(4):
        full[k, c, c] = inputs.GROVER_SPREAD_STATE[k]
    w.set_state(full).step(T)
    assert w.describe()["support"] == [c - T, 2 * T + 1, c - T, 2 * T + 1]
    got = w.state(dtype=np.complex64)
    assert np.all(got[:, : c - T, :] == 0) and np.all(got[:, c + T + 1:, :] == 0)
    assert np.all(got[:, :, : c - T] == 0) and np.all(got[:, :, c + T + 1:] == 0)
    M = 2 * T + 1
    win0 = inputs.localized_2d(M, T, T)
    want = oracle.evolve(win0, inputs.grover(), T)      # the walk never reaches the window's edge
    sub = got[:, c - T: c + T + 1, c - T: c + T + 1].astype(np.complex128)
    assert maxabs(sub, want) < amp_tol("f32", T)
    w.close()


def test_steps_captured_in_a_cuda_graph_run_in_full(qw):
    """While the walk's stream is captured into a CUDA graph nothing may wait for
    it: qw_set_state skips the support search and the captured steps run on the
    whole lattice.  The replayed graph matches the oracle."""
    import ctypes
    import torch
    N, T = 4096, 64
    C = inputs.su2(0.3)
    s = torch.cuda.Stream()
    psi0 = inputs.localized_1d(N, 100)
    psi = torch.from_numpy(psi0.astype(np.complex64)).cuda()
    w = qw.Walk((N,), prec="f32", stream=ctypes.c_void_p(s.cuda_stream)).set_coin(C)
    w.set_state(psi).step(T)          # outside a capture: clipped, kernels loaded
    assert w.describe()["support"] != "full"
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        qw.qw_set_state(w.h, psi)
        qw.qw_step(w.h, T)
    g.replay()
    torch.cuda.synchronize()
    assert w.describe()["support"] == "full"
    assert maxabs(w.state(), oracle.evolve(psi0, C, T)) < amp_tol("f32", T)
    w.close()


# ---------------------------------------------------------------- boundaries and links
def _generic_run(qw, dims, psi0, T, clip, bc, shift, C, p=0.0, seed=0, fixed=None, adjoint=False, prec="f32"):
    w = qw.Walk(dims, prec=prec, shift=shift, bc=bc).set_clipping(clip).set_coin(C)
    if fixed is not None:
        w.set_links(fixed)
    if p:
        w.set_link_noise(p, seed)
    w.set_state(psi0)
    (w.step_adjoint if adjoint else w.step)(T)
    out, desc = w.state(), w.describe()
    w.close()
    return out, desc


@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("links", ["none", "fixed", "random"])
@pytest.mark.parametrize("x0", [6, 1500, 2996])
def test_line_and_segment_window_1d(qw, bc, shift, links, x0):
    """The generic tiled kernel on the cycle, the segment (reflecting ends) and
    the line (absorbing ends, the paper's line walk) with fixed or per-step
    random broken links: clipped and full steps agree bit for bit and match the
    oracle; on the segment and the line the window stops at the ends."""
    N, T = 3000, 120
    rng = np.random.default_rng(400 + bc + 3 * shift)
    C = inputs.random_unitary(2, rng)
    psi0 = inputs.localized_1d(N, x0, (0.6, 0.8j))
    fixed = (rng.uniform(size=(1, N)) < 0.1).astype(np.uint8) if links == "fixed" else None
    p, seed = (0.1, 91) if links == "random" else (0.0, 0)
    kw = dict(bc=bc, shift=shift, C=C, p=p, seed=seed, fixed=fixed)
    on, desc = _generic_run(qw, (N,), psi0, T, True, **kw)
    off, _ = _generic_run(qw, (N,), psi0, T, False, **kw)
    assert same(on, off)
    # the cycle with links: the generic tiles; the segment and the line: the window CTA
    want_path = ("k_step1d" if links == "none" else "generic") if bc == 0 else "k_step1d_window"
    assert desc["path"] == want_path
    lo, hi = x0 - T, x0 + T + 1
    if bc == 0:
        assert desc["support"] == [lo % N, 2 * T + 1, 0, 1]
    else:
        assert desc["support"] == [max(0, lo), min(N, hi) - max(0, lo), 0, 1]
    closed = fixed
    if links == "random":
        closed = oracle.link_masks((N,), seed, p, 0, T)
    want = oracle.evolve(psi0, C, T, shift=shift, bc=bc, closed=closed, closed_per_step=links == "random")
    assert maxabs(on, want) < amp_tol("f32", T)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("bc", [1, 2])
@pytest.mark.parametrize("links", ["none", "random"])
def test_window_kernel_launches_ends_and_capacity(qw, prec, bc, links):
    """The window CTA (segment and line, clipped) runs up to 256 steps per
    launch.  Calls of 40, 300, 2000 and 7000 steps from x0 = 700 on N = 12000:
    several launches per call, the box stopping at the left end, random-link
    steps carried from call to call, and a box that outgrows the CTA's window
    (about 6200 sites in FP32, 8190 with bfloat16 storage, 3150 in FP64 and
    double-float), after which the steps go back to the tiled kernel.  Bit for
    bit against the unclipped steps, and the oracle."""
    N, x0 = 12000, 700
    chunks = [40, 300, 2000, 7000]
    rng = np.random.default_rng(600 + bc)
    C = inputs.random_unitary(2, rng)
    psi0 = inputs.localized_1d(N, x0, (0.6, 0.8j))
    p, seed = (0.05, 93) if links == "random" else (0.0, 0)

    def go(clip):
        w = qw.Walk((N,), prec=prec, bc=bc).set_clipping(clip).set_coin(C)
        if p:
            w.set_link_noise(p, seed)
        w.set_state(psi0)
        paths = []
        for c in chunks:
            w.step(c)
            paths.append(w.describe()["path"])
        out = w.state()
        w.close()
        return out, paths

    on, paths = go(True)
    off, _ = go(False)
    assert same(on, off)
    assert paths[0] == "k_step1d_window" and paths[-1] == "generic"
    T = sum(chunks)
    closed = oracle.link_masks((N,), seed, p, 0, T) if p else None
    want = oracle.evolve(psi0, C, T, bc=bc, closed=closed, closed_per_step=bool(p))
    assert maxabs(on, want) < amp_tol(prec, T)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("kind", ["per_site", "phase"])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("bc", [1, 2])
def test_window_kernel_per_site_and_phase_coins(qw, prec, kind, shift, bc):
    """Per-site coin matrices and phase coins in the window CTA, from the
    middle of a 4000-site line or segment (T = 600) and from next to its right
    end (T = 300, the box stops there): clipped and unclipped bit for bit, and
    the oracle with the same coins."""
    N = 4000
    rng = np.random.default_rng(700 + 2 * shift + bc)
    base = inputs.random_unitary(2, rng)
    coins = np.stack([inputs.random_unitary(2, rng) for _ in range(N)])
    phi = rng.uniform(-1, 1, size=(N, 2)).astype(np.float32)
    for x0, T in ((2000, 600), (3990, 300)):
        psi0 = inputs.localized_1d(N, x0, (0.6, 0.8j))
        got = []
        for clip in (True, False):
            w = qw.Walk((N,), prec=prec, shift=shift, bc=bc).set_clipping(clip)
            if kind == "per_site":
                w.set_coin(coins, per_site=True)
            else:
                w.set_coin_phases(base, phi)
            w.set_state(psi0).step(T)
            got.append((w.state(), w.describe()["path"]))
            w.close()
        assert same(got[0][0], got[1][0]), x0
        assert got[0][1] == "k_step1d_window"
        if kind == "per_site":
            want = oracle.evolve(psi0, coins, T, shift=shift, bc=bc)
            extra = 0.0
        else:
            want = oracle.evolve(psi0, base, T, shift=shift, bc=bc, phi=phi.astype(np.float64))
            extra = T * 1e-7    # the phases are float inputs
        assert maxabs(got[0][0], want) < amp_tol(prec, T) + extra, x0


@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("links", ["none", "fixed", "random"])
@pytest.mark.parametrize("start", [(1, 2), (100, 60), (198, 128)])
def test_line_and_segment_window_2d(qw, bc, shift, links, start):
    """The same on a 200 x 130 lattice (the generic 64 x 8 tiles; rows and
    columns not multiples of the tile), from next to a corner, the interior and
    the far corner, T = 40."""
    Lx, Ly, T = 200, 130, 40
    rng = np.random.default_rng(500 + bc + 3 * shift)
    C = inputs.grover() if links == "none" else inputs.random_unitary(4, rng)
    psi0 = inputs.localized_2d(Lx, start[0], start[1], (0.5, -0.5j, 0.5, 0.5j), Ly=Ly)
    fixed = (rng.uniform(size=(2, Lx * Ly)) < 0.1).astype(np.uint8) if links == "fixed" else None
    p, seed = (0.1, 92) if links == "random" else (0.0, 0)
    kw = dict(bc=bc, shift=shift, C=C, p=p, seed=seed, fixed=fixed)
    on, desc = _generic_run(qw, (Lx, Ly), psi0, T, True, **kw)
    off, _ = _generic_run(qw, (Lx, Ly), psi0, T, False, **kw)
    assert same(on, off)
    closed = fixed
    if links == "random":
        closed = oracle.link_masks((Ly, Lx), seed, p, 0, T)
    want = oracle.evolve(psi0, C, T, shift=shift, bc=bc, closed=closed, closed_per_step=links == "random")
    assert maxabs(on, want) < amp_tol("f32", T)
    if bc != 0:
        x0, y0 = start
        assert desc["support"] == [max(0, x0 - T), min(Lx, x0 + T + 1) - max(0, x0 - T),
                                   max(0, y0 - T), min(Ly, y0 + T + 1) - max(0, y0 - T)]


@pytest.mark.parametrize("bc", [1, 2])
def test_line_window_adjoint_steps_in_full(qw, bc):
    """The adjoint with a boundary runs the per-site generic kernel over the
    whole lattice; the tracked window still widens with it, and clipped and
    full runs agree."""
    N, T, x0 = 2000, 90, 40
    C = inputs.su2(0.3, 0.2, -0.1)
    psi0 = inputs.localized_1d(N, x0)
    on, desc = _generic_run(qw, (N,), psi0, T, True, bc=bc, shift=0, C=C, adjoint=True)
    off, _ = _generic_run(qw, (N,), psi0, T, False, bc=bc, shift=0, C=C, adjoint=True)
    assert same(on, off) and desc["support"] == [0, x0 + T + 1, 0, 1]
    assert maxabs(on, oracle.evolve(psi0, C, T, bc=bc, adjoint=True)) < amp_tol("f32", T)
