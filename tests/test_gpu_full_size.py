"""Full-size parity in the configurations the benchmark times, on sampled sites.

A site's amplitudes after T steps depend only on the initial state within T
sites of it (the light cone), so the FP64 oracle run on the window of 2T + 1
sites around a sampled site, with an absorbing edge, gives that site's exact
value; the values outside the window reach the edge after T steps at the
earliest and never the centre.  The tolerance is the derived T * 4u per
amplitude (u = 2^-24), relative to the 2-norm of the window's initial state,
which bounds every amplitude the unitary walk can produce inside it.
"""
import numpy as np
import pytest

import oracle
from paper_1003_3779_gb300 import inputs

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def qw():
    import paper_1003_3779_gb300.qw as qw
    qw.lib()
    return qw


# the benchmark's coin classes: SU(2) theta = pi/4 (the Hadamard class, four
# additions per site-step), a real rotation theta = 0.3 and a complex SU(2) coin
FULL_COINS = {"hadamard_class": inputs.su2(np.pi / 4), "real": inputs.su2(0.3),
              "complex": inputs.su2(np.pi / 4, 0.3, -0.2)}


@pytest.mark.parametrize("coin", list(FULL_COINS))
def test_cycle_2e27_T4096_sweep_sampled(qw, coin):
    """N = 2^27, T = 4096, FP32, the random complex64 state of the benchmark,
    swept at k = 384 with 32 sites per lane (as the benchmark's autotuner picks
    for the headline coin): eight sampled sites against the oracle, plus the
    norm, for each coin class the benchmark times."""
    import torch
    N, T = 1 << 27, 4096
    C = FULL_COINS[coin]
    psi0 = inputs.random_state((2, N), seed=1, dtype=np.complex64)
    w = qw.Walk((N,), prec="f32").set_coin(C).set_plan_ex(384, 32, 1)
    assert w.describe()["coin_kind"] == coin
    w.set_state(torch.from_numpy(psi0).cuda())
    w.step(T)
    assert abs(w.norm() - 1) < T * 4 * U32
    got = w.state(dtype=np.complex64)
    rng = np.random.default_rng(7)
    sample = [0, N - 1, N // 2, 12345] + list(rng.integers(0, N, size=4))
    for x in sample:
        idx = (x - T + np.arange(2 * T + 1)) % N
        win = psi0[:, idx].astype(np.complex128)
        want = oracle.evolve(win, C, T, bc=oracle.BC_LINE)[:, T]
        scale = float(np.sqrt((np.abs(win) ** 2).sum()))
        err = float(np.abs(got[:, x].astype(np.complex128) - want).max())
        assert err <= T * 4 * U32 * scale, (x, err, scale)
    w.close()


@pytest.mark.parametrize("coin,shift", [("grover", 0), ("hh", 0), ("grover", 1), ("hh", 2)])
def test_torus_8192_streaming_sampled(qw, coin, shift):
    """8192 x 8192 torus, FP32, the streaming kernel at k = 8 as the benchmark
    times it, T = 64 (eight launches), a random state: sampled sites (corners,
    edges, interior) against the oracle on their (2T + 1)^2 windows (an
    absorbing edge on the axis lattice; on the diagonal lattice, where the
    oracle takes only the periodic edge, the window as a torus of its own: a
    path of T steps to the centre starts within T of it and wraps nowhere)."""
    import torch
    L, T = 8192, 64
    C = {"grover": inputs.grover(), "hh": inputs.hadamard2()}[coin]
    psi0 = inputs.random_state((4, L, L), seed=2, dtype=np.complex64)
    w = qw.Walk((L, L), prec="f32", shift=shift).set_coin(C).set_plan(8)
    assert w.describe()["path"] == "k_step2d_tb"
    w.set_state(torch.from_numpy(psi0).cuda())
    w.step(T)
    got = w.state(dtype=np.complex64)
    rng = np.random.default_rng(8)
    sample = [(0, 0), (L - 1, L - 1), (0, L - 1), (L // 2, 47)] + [tuple(p) for p in rng.integers(0, L, size=(3, 2))]
    M = 2 * T + 1
    for (x, y) in sample:
        ix = (x - T + np.arange(M)) % L
        iy = (y - T + np.arange(M)) % L
        win = psi0[:, iy][:, :, ix].astype(np.complex128)
        bc = oracle.BC_PERIODIC if shift == 2 else oracle.BC_LINE
        want = oracle.evolve(win, C, T, shift=shift, bc=bc)[:, T, T]
        scale = float(np.sqrt((np.abs(win) ** 2).sum()))
        err = float(np.abs(got[:, y, x].astype(np.complex128) - want).max())
        assert err <= T * 4 * U32 * scale, (x, y, err, scale)
    w.close()


def test_graph_random_regular_2e26_sampled(qw):
    """The random 4-regular graph with 2^26 vertices (2^28 arcs), FP32, Grover, in
    the autotuned form the benchmark times, T = 6 steps: the arcs of sampled
    vertices against the FP64 oracle run on the ball of radius T + 1 around each
    (arcs whose edge leaves the ball are made fixed points there; a value at the
    centre after T steps depends only on arcs within distance T, so the cut never
    reaches it).  Plus the norm, and the pull form bitwise against the chosen one."""
    import torch
    nv, T = 1 << 26, 6
    off, partner = inputs.random_regular_arcs(nv, 4, seed=5)
    A = int(off[-1])
    psi0 = inputs.random_state((A,), seed=6, dtype=np.complex64)
    w = qw.GraphWalk(off, partner, prec="f32").set_state(torch.from_numpy(psi0).cuda())
    w.autotune()
    w.step(T)
    _, norm = w.probabilities()
    assert abs(norm - 1) < T * 8 * U32
    got = w.state(dtype=np.complex64)
    chosen = w.variant()
    w.set_variant(1 if chosen != 1 else 0).set_state(torch.from_numpy(psi0).cuda())
    w.step(T)
    assert np.array_equal(w.state(dtype=np.complex64), got)
    w.close()
    rng = np.random.default_rng(9)
    for c in [0, nv - 1] + list(rng.integers(0, nv, size=4)):
        ball, frontier = {int(c)}, [int(c)]
        for _ in range(T + 1):
            nxt = []
            for v in frontier:
                for u in (partner[4 * v: 4 * v + 4] // 4).tolist():
                    if u not in ball:
                        ball.add(u)
                        nxt.append(u)
            frontier = nxt
        verts = np.array(sorted(ball), dtype=np.int64)
        local = {int(v): i for i, v in enumerate(verts)}
        arcs = (4 * verts[:, None] + np.arange(4)).ravel()
        lpart = np.empty(len(arcs), dtype=np.int64)
        for i, a in enumerate(arcs.tolist()):
            p = int(partner[a])
            lpart[i] = 4 * local[p // 4] + p % 4 if p // 4 in local else i
        loff = np.arange(0, len(arcs) + 1, 4, dtype=np.int64)
        want = oracle.graph_evolve(loff, lpart, psi0[arcs].astype(np.complex128), T)
        i0 = 4 * local[int(c)]
        err = float(np.abs(got[4 * c: 4 * c + 4].astype(np.complex128) - want[i0: i0 + 4]).max())
        scale = float(np.sqrt((np.abs(psi0[arcs].astype(np.complex128)) ** 2).sum()))
        assert err <= T * 8 * U32 * scale, (c, err, scale)
