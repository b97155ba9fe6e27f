"""Pins of the oracle's general-graph walk (Sec. 2.1: U = S (I (x) C) with
S|v,e> = |v',e>), each against something other than the oracle itself:
hand-worked examples, the exact classical motion of the Grover walk on a path,
the lattice walks (the cycle and the torus are graphs; their walk with the
lattice's coin slots as arc slots is the flip-flop lattice walk, computed by the
oracle's separate lattice code), the invariant uniform state of the Grover coin,
and the dense unitary built column by column."""
import numpy as np
import pytest

import oracle
from paper_1003_3779_gb300 import inputs

SQ = 1 / np.sqrt(2)


def test_graph_arcs_hand_example():
    """Edges (0,1), a loop (1,1), (2,0): slots follow the order of the edge ends."""
    off, partner = oracle.graph_arcs(3, [(0, 1), (1, 1), (2, 0)])
    assert off.tolist() == [0, 2, 5, 6]
    # v0: [edge to 1, edge to 2]; v1: [edge to 0, loop end 0, loop end 1]; v2: [edge to 0]
    assert partner.tolist() == [2, 5, 0, 4, 3, 1]


def test_graph_hadamard_interference_hand_example():
    """Path 0-1-2 with coins [1], H, [1], start on vertex 0's arc: after two steps
    the amplitude splits 1/sqrt2 to each end; after four it recombines on the
    start arc (worked by hand; a wrong sign in H or a transposed coin changes it)."""
    off, partner = oracle.graph_arcs(3, [(0, 1), (1, 2)])
    coins = [np.eye(1), inputs.hadamard(), np.eye(1)]
    psi = np.zeros(4, complex)
    psi[0] = 1
    want = {1: [0, 1, 0, 0], 2: [SQ, 0, 0, SQ], 3: [0, SQ, SQ, 0], 4: [1, 0, 0, 0]}
    for T, w in want.items():
        got = oracle.graph_evolve(off, partner, psi, T, coins=coins)
        assert np.abs(got - np.array(w)).max() < 1e-15, T


@pytest.mark.parametrize("n", [2, 3, 7])
def test_graph_grover_path_moves_like_a_classical_particle(n):
    """On a path the Grover coin is [1] at the ends and the swap [[0,1],[1,0]]
    inside, so the walk is deterministic transport: a particle keeps its
    direction and turns back at the ends.  Compared exactly with a classical
    simulation of that particle for every start arc."""
    off, partner = oracle.graph_arcs(n, [(i, i + 1) for i in range(n - 1)])

    def arc(v, towards):  # slot 0 is the edge to v-1 (if v > 0), then the edge to v+1
        return off[v] + (0 if towards < v or v == 0 else 1)

    for a0 in range(int(off[-1])):
        v = int(np.searchsorted(off, a0, side="right") - 1)
        nb = [u for u in (v - 1, v + 1) if 0 <= u < n]
        pos, towards = v, nb[a0 - off[v]]
        psi = np.zeros(int(off[-1]), complex)
        psi[a0] = 1
        for T in range(1, 3 * n):
            # coin: move on past pos (or back at an end); shift: cross that edge
            nxt = [u for u in (pos - 1, pos + 1) if 0 <= u < n and u != towards] or [towards]
            pos, towards = nxt[0], pos
            got = oracle.graph_evolve(off, partner, psi, T)
            want = np.zeros_like(got)
            want[arc(pos, towards)] = 1
            assert np.array_equal(got, want), (a0, T)


@pytest.mark.parametrize("dims", [(7,), (1,), (2,), (5, 3), (1, 4), (2, 2)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_graph_walk_on_lattice_is_flipflop_lattice_walk(dims, adjoint):
    rng = np.random.default_rng(sum(dims) + 10 * adjoint)
    d = 2 * len(dims)
    C = inputs.random_unitary(d, rng)
    off, partner = inputs.lattice_graph_arcs(*dims)
    shape = (d,) + tuple(reversed(dims))
    lat = inputs.random_state(shape, seed=40)
    T = 11
    want = oracle.evolve(lat, C, T, shift=oracle.SHIFT_FLIPFLOP, adjoint=adjoint)
    arcs = lat.reshape(d, -1).T.ravel()          # arc d*v + c holds coin c of site v
    got = oracle.graph_evolve(off, partner, arcs, T, coins=C, adjoint=adjoint)
    assert np.abs(got - want.reshape(d, -1).T.ravel()).max() < 1e-13
    P, norm = oracle.graph_probabilities(off, got)
    Pl, norml = oracle.probabilities(want)
    assert np.abs(P - Pl.ravel()).max() < 1e-14 and abs(norm - norml) < 1e-14


@pytest.mark.parametrize("kind", ["regular", "chung_lu"])
def test_graph_grover_uniform_state_is_invariant(kind):
    """(2/d) J - I fixes the all-ones vector of each vertex and S permutes the
    arcs, so the uniform arc state is a fixed point on any graph (isolated
    vertices, loops and parallel edges included)."""
    if kind == "regular":
        off, partner = inputs.random_regular_arcs(500, 3, seed=5)
    else:
        off, partner = oracle.graph_arcs(400, inputs.chung_lu_edges(400, 6, 2.3, seed=6))
    A = int(off[-1])
    psi = np.full(A, (0.6 + 0.8j) / np.sqrt(A))
    got = oracle.graph_evolve(off, partner, psi, 25)
    assert np.abs(got - psi).max() < 1e-15 * 25 * np.diff(off).max()


def small_graph(rng):
    edges = [(0, 1), (1, 2), (2, 0), (2, 3), (3, 3), (1, 2), (4, 2), (0, 4)]
    off, partner = oracle.graph_arcs(6, edges)     # vertex 5 is isolated
    coins = [inputs.random_unitary(int(d), rng) if d else np.zeros((0, 0)) for d in np.diff(off)]
    return off, partner, coins


def test_graph_dense_unitary_and_adjoint():
    """U built column by column is unitary; the adjoint run's columns are U^dagger;
    with identity coins U = S and S^2 = I."""
    rng = np.random.default_rng(7)
    off, partner, coins = small_graph(rng)
    A = int(off[-1])
    E = np.eye(A, dtype=complex)
    U = np.stack([oracle.graph_evolve(off, partner, E[k], 1, coins=coins) for k in range(A)], axis=1)
    Ud = np.stack([oracle.graph_evolve(off, partner, E[k], 1, coins=coins, adjoint=True) for k in range(A)], axis=1)
    assert np.abs(U.conj().T @ U - E).max() < 1e-14
    assert np.abs(Ud - U.conj().T).max() < 1e-15
    ident = [np.eye(int(d)) for d in np.diff(off)]
    S = np.stack([oracle.graph_evolve(off, partner, E[k], 1, coins=ident) for k in range(A)], axis=1)
    assert np.array_equal(S @ S, E.real)
    assert np.array_equal(np.argmax(S, axis=0), partner)


def test_graph_oracle_rejects_bad_partner():
    off = np.array([0, 2, 4], dtype=np.int64)
    with pytest.raises(RuntimeError):
        oracle.graph_evolve(off, np.array([1, 2, 3, 0]), np.zeros(4, complex), 1)   # not an involution
    with pytest.raises(RuntimeError):
        oracle.graph_evolve(off, np.array([1, 0, 3, 4]), np.zeros(4, complex), 1)   # out of range
