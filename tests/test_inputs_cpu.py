"""The seeded input generators: shapes, invariants and reproducibility (no GPU)."""
import numpy as np
import pytest

from paper_1003_3779_gb300 import inputs


@pytest.mark.parametrize("nv,d", [(10, 3), (1000, 4), (7, 2), (1, 2)])
def test_random_regular_arcs_is_a_regular_multigraph(nv, d):
    off, partner = inputs.random_regular_arcs(nv, d, seed=4)
    A = nv * d
    assert np.array_equal(off, np.arange(0, A + 1, d))
    assert partner.shape == (A,) and np.array_equal(np.sort(partner), np.arange(A))
    assert np.array_equal(partner[partner], np.arange(A))          # an involution: S^2 = I
    assert not np.any(partner == np.arange(A))                     # every edge has two ends
    o2, p2 = inputs.random_regular_arcs(nv, d, seed=4)
    assert np.array_equal(p2, partner)                              # seeded
    with pytest.raises(ValueError):
        inputs.random_regular_arcs(3, 3, seed=1)                   # odd number of edge ends


@pytest.mark.parametrize("dims", [(5,), (1,), (4, 3), (1, 1), (2, 5)])
def test_lattice_graph_arcs_follow_the_coin_directions(dims):
    off, partner = inputs.lattice_graph_arcs(*dims)
    d = 2 * len(dims)
    ns = int(np.prod(dims))
    assert np.array_equal(off, np.arange(0, d * ns + 1, d))
    assert np.array_equal(partner[partner], np.arange(d * ns))
    Lx = dims[0]
    Ly = dims[1] if len(dims) == 2 else 1
    for v in range(ns):
        x, y = v % Lx, v // Lx
        if len(dims) == 1:
            # slot 0 is the edge to x - 1, slot 1 the edge to x + 1, arriving in the opposite slot
            assert partner[2 * v] == 2 * ((x - 1) % Lx) + 1
            assert partner[2 * v + 1] == 2 * ((x + 1) % Lx)
        else:
            assert partner[4 * v] == 4 * (y * Lx + (x + 1) % Lx) + 1
            assert partner[4 * v + 2] == 4 * (((y + 1) % Ly) * Lx + x) + 3


def test_chung_lu_edges_have_skewed_degrees():
    e = inputs.chung_lu_edges(3000, 6, 2.2, seed=13)
    assert e.shape == (9000, 2) and e.min() >= 0 and e.max() < 3000
    deg = np.bincount(e.ravel(), minlength=3000)
    assert deg.sum() == 18000
    assert deg[:10].mean() > 10 * deg[1000:].mean()                # low indices are the hubs
    assert deg.max() > 32 and (deg == 0).sum() > 0                 # heavy and isolated vertices
    assert np.array_equal(e, inputs.chung_lu_edges(3000, 6, 2.2, seed=13))
