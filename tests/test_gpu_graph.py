"""GPU parity of the walk on a general graph (Sec. 2.1) through the C ABI
(qw_gwalk_*) against the FP64 oracle's graph walk, on lattices, random regular
graphs, skewed-degree graphs with heavy vertices, loops, parallel edges and
isolated vertices; forward (both forms) and adjoint; every coin mode.

Tolerance: one step forms each amplitude from a chain of d(v) products over a
unit coin row (or, for Grover, a d-term sum scaled by 2/d), so its rounding
error is at most about (d + 4) u per step for unit-norm data; after T steps the
bound is T (dmax + 4) u."""
import numpy as np
import pytest

import oracle
from paper_1003_3779_gb300 import inputs
from tests.helpers import U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qw():
    import paper_1003_3779_gb300.qw as qw
    qw.lib()
    return qw


def tol(prec, T, dmax):
    return max(T, 1) * (dmax + 4) * U[prec] + 1e-15


def graph(name):
    """(off, partner) of the named test graph."""
    if name == "cycle":
        return inputs.lattice_graph_arcs(301)
    if name == "torus":
        return inputs.lattice_graph_arcs(23, 9)
    if name == "regular3":
        return inputs.random_regular_arcs(1000, 3, seed=11)
    if name == "regular4":
        return inputs.random_regular_arcs(1500, 4, seed=12)
    if name == "chung_lu":     # skewed degrees: vertices above degree 32, isolated vertices, loops
        return oracle.graph_arcs(3000, inputs.chung_lu_edges(3000, 6, 2.2, seed=13))
    if name == "small":        # loops, parallel edges, an isolated vertex
        return oracle.graph_arcs(6, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 3), (1, 2), (4, 2), (0, 4)])
    raise KeyError(name)


GRAPHS = ["cycle", "torus", "regular3", "regular4", "chung_lu", "small"]


def coins_for(kind, off, rng):
    deg = np.diff(off)
    if kind == "grover":
        return None
    if kind == "uniform":
        return inputs.random_unitary(int(deg[0]), rng)
    return [inputs.random_unitary(int(d), rng) if d else np.zeros((0, 0), complex) for d in deg]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", GRAPHS)
@pytest.mark.parametrize("coin", ["grover", "uniform", "per_vertex"])
@pytest.mark.parametrize("form", ["push", "pull", "scatter2", "gather2", "adjoint"])
def test_graph_walk_against_oracle(qw, prec, name, coin, form):
    off, partner = graph(name)
    deg = np.diff(off)
    if coin == "uniform" and np.any(deg != deg[0]):
        pytest.skip("a uniform coin needs a regular graph")
    rng = np.random.default_rng(GRAPHS.index(name) * 7 + len(coin))
    C = coins_for(coin, off, rng)
    psi0 = inputs.random_state((int(off[-1]),), seed=41)
    T = 13
    want = oracle.graph_evolve(off, partner, psi0, T, coins=C, adjoint=form == "adjoint")
    w = qw.GraphWalk(off, partner, prec=prec).set_coin(C).set_state(psi0)
    if form != "adjoint":
        # the two-pass forms with windows of 40 amplitudes: many buckets, ragged ones
        w.set_window(40 * (16 if prec == "f64" else 8))
        w.set_variant(["push", "pull", "scatter2", "gather2"].index(form))
        w.step(T)
    else:
        w.step_adjoint(T)
    got = w.state()
    assert np.abs(got - want).max() < tol(prec, T, int(deg.max()))
    P, norm = w.probabilities()
    Pw, normw = oracle.graph_probabilities(off, want)
    assert np.abs(P - Pw).sum() < (1e-12 if prec == "f64" else 1e-4)
    assert abs(norm - 1) < (1e-12 if prec == "f64" else 1e-5)
    w.close()


@pytest.mark.parametrize("name", ["regular4", "chung_lu", "torus"])
@pytest.mark.parametrize("window", [8 * 1000, 8 * 4096, 1 << 25])
def test_all_forms_agree_bitwise(qw, name, window):
    """Every forward form evaluates the same expression per arc: identical bits,
    whatever the bucket window of the two-pass forms."""
    off, partner = graph(name)
    psi0 = inputs.random_state((int(off[-1]),), seed=42).astype(np.complex64)
    out = []
    for v in range(4):
        w = qw.GraphWalk(off, partner, prec="f32").set_state(psi0).set_window(window).set_variant(v)
        w.step(21)
        assert w.variant() == v
        out.append(w.state(dtype=np.complex64))
        w.close()
    for o in out[1:]:
        assert np.array_equal(out[0], o)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("name", ["cycle", "torus", "regular4", "big4"])
@pytest.mark.parametrize("coin", ["grover", "uniform", "per_vertex"])
def test_fused_gather_steps_match_single_steps_bitwise(qw, prec, name, coin):
    """On graphs of degree 2 or 4 the gather form runs a call of T >= 2 steps as
    one bucketing pass, T - 1 fused gather + bucketing passes and one gather;
    one step per call runs the two separate passes.  Both feed the coin the
    same values: identical bits for T = 2, 3 and 8, and the oracle's state."""
    if name == "big4":   # 3 tiles of 2048 arcs and a ragged fourth; 16 buckets
        off, partner = inputs.random_regular_arcs(1700, 4, seed=14)
    else:
        off, partner = graph(name)
    rng = np.random.default_rng(5)
    C = coins_for(coin, off, rng)
    psi0 = inputs.random_state((int(off[-1]),), seed=43)
    window = (int(off[-1]) // 16 + 1) * (16 if prec == "f64" else 8)
    for T in (2, 3, 8):
        a = qw.GraphWalk(off, partner, prec=prec).set_coin(C).set_state(psi0).set_window(window).set_variant(3)
        b = qw.GraphWalk(off, partner, prec=prec).set_coin(C).set_state(psi0).set_window(window).set_variant(3)
        a.step(T)
        for _ in range(T):
            b.step(1)
        sa, sb = a.state(), b.state()
        assert np.array_equal(sa, sb)
        want = oracle.graph_evolve(off, partner, psi0, T, coins=C)
        assert np.abs(sa - want).max() < tol(prec, T, 4)
        # and a further call continues from the right buffer
        a.step(2)
        b.step(1)
        b.step(1)
        assert np.array_equal(a.state(), b.state())
        a.close()
        b.close()


@pytest.mark.parametrize("dims", [(64,), (40, 24), (3, 5)])
def test_graph_on_lattice_matches_the_lattice_kernels(qw, dims):
    """The lattice as a graph with the lattice's coin slots runs the flip-flop
    lattice walk: the graph kernels against the lattice kernels, FP64."""
    rng = np.random.default_rng(len(dims))
    d = 2 * len(dims)
    C = inputs.random_unitary(d, rng)
    off, partner = inputs.lattice_graph_arcs(*dims)
    lat0 = inputs.random_state((d,) + tuple(reversed(dims)), seed=43)
    T = 17
    lw = qw.Walk(dims, prec="f64", shift=qw.SHIFT_FLIPFLOP).set_coin(C).set_state(lat0)
    lw.step(T)
    want = lw.state().reshape(d, -1).T.ravel()
    gw = qw.GraphWalk(off, partner, prec="f64").set_coin(C).set_state(lat0.reshape(d, -1).T.ravel())
    gw.step(T)
    assert np.abs(gw.state() - want).max() < 1e-12
    lw.close()
    gw.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_forward_then_adjoint_returns_the_state(qw, prec):
    off, partner = graph("chung_lu")
    psi0 = inputs.random_state((int(off[-1]),), seed=44)
    w = qw.GraphWalk(off, partner, prec=prec).set_state(psi0)
    T = 30
    w.step(T).step_adjoint(T)
    assert np.abs(w.state() - psi0).max() < 2 * tol(prec, T, int(np.diff(off).max()))
    w.close()


def test_grover_uniform_state_is_a_fixed_point(qw):
    """(2/d) J - I fixes each vertex's uniform vector and S permutes arcs: the
    uniform arc state stays put on any graph (heavy vertices use the pre-pass)."""
    off, partner = graph("chung_lu")
    assert np.diff(off).max() > 32
    A = int(off[-1])
    psi = np.full(A, (0.6 + 0.8j) / np.sqrt(A))
    w = qw.GraphWalk(off, partner, prec="f64").set_state(psi)
    w.step(40)
    assert np.abs(w.state() - psi).max() < 1e-14
    w.close()


def test_graph_edge_cases(qw):
    # no edges: nothing moves, P is zero
    off = np.zeros(5, dtype=np.int64)
    w = qw.GraphWalk(off, np.zeros(0, dtype=np.int64), prec="f64")
    w.step(3).step_adjoint(2)
    P, norm = w.probabilities()
    assert np.all(P == 0) and norm == 0
    assert w.state().shape == (0,)
    w.close()
    # one vertex with a loop: Grover on d=2 swaps the two arcs, S swaps them back
    off, partner = oracle.graph_arcs(1, [(0, 0)])
    psi = np.array([0.6, 0.8j])
    w = qw.GraphWalk(off, partner, prec="f64").set_state(psi)
    w.step(5)
    assert np.abs(w.state() - oracle.graph_evolve(off, partner, psi, 5)).max() < 1e-15
    # a uniform coin on an irregular graph and bad dtypes are rejected
    off, partner = graph("small")
    w = qw.GraphWalk(off, partner, prec="f32")
    with pytest.raises(qw.QWError):
        w.set_coin(np.eye(2))
    with pytest.raises(qw.QWError):
        w.set_variant(4)
    with pytest.raises(qw.QWError):
        w.set_window(4)
    w.close()


def test_autotune_keeps_the_state(qw):
    off, partner = inputs.random_regular_arcs(1 << 14, 4, seed=14)
    psi0 = inputs.random_state((int(off[-1]),), seed=45).astype(np.complex64)
    w = qw.GraphWalk(off, partner, prec="f32").set_state(psi0)
    rep = w.autotune()
    assert rep["variant"] in (0, 1, 2, 3) and rep["push_ms_per_step"] > 0
    assert rep["two_pass_gather_ms_per_step"] > 0
    assert np.array_equal(w.state(dtype=np.complex64), psi0)
    w.close()
