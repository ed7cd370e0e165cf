"""Pins of the triangle-counting oracle (the masked product L*L .* L of the
paper's triangle-counting experiment) against facts fixed by mathematics,
not by the oracle: trace(A^3)/6 by dense matmul and by scipy's sparse
product, brute force over vertex triples (total and per highest-labelled
vertex), closed forms of complete, cycle, wheel and complete bipartite
graphs, and invariance under relabelling."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1804_00695_gb300 import inputs as I


def graph_from_edges(n, edges):
    """Symmetric pattern without self loops from an undirected edge list."""
    if not edges:
        return I.Csr(n, n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    e = np.array(edges, dtype=np.int64)
    r = np.concatenate([e[:, 0], e[:, 1]])
    c = np.concatenate([e[:, 1], e[:, 0]])
    return I._coo_to_csr(n, r, c)


def random_graph(n, p, seed):
    u = I.uniform01(np.arange(n * n, dtype=np.uint64), seed, 11).reshape(n, n)
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if u[i, j] < p]
    return graph_from_edges(n, edges)


def dense(g):
    d = np.zeros((g.nrows, g.nrows), dtype=np.int64)
    d[np.repeat(np.arange(g.nrows), np.diff(g.row_ptr)), g.col] = 1
    return d


def brute(g, perm):
    """Triangles by checking every vertex triple; per vertex: those whose
    vertex with the largest label under perm is it."""
    d = dense(g)
    per = np.zeros(g.nrows, dtype=np.int64)
    total = 0
    for a, b, c in itertools.combinations(range(g.nrows), 3):
        if d[a, b] and d[b, c] and d[a, c]:
            total += 1
            per[max((a, b, c), key=lambda v: perm[v])] += 1
    return total, per


@pytest.mark.parametrize("n,p,seed", [(12, 0.5, 1), (30, 0.3, 2), (40, 0.15, 3), (25, 0.9, 4)])
def test_brute_force_and_trace(n, p, seed):
    g = random_graph(n, p, seed)
    perm = oracle.degree_order(g)
    total, per = oracle.triangles(g)
    bt, bper = brute(g, perm)
    assert total == bt
    assert np.array_equal(per, bper)
    d = dense(g)
    assert total == int(np.trace(d @ d @ d)) // 6


def test_closed_forms():
    for n in (3, 4, 7, 10):   # complete graph: C(n, 3)
        g = graph_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
        assert oracle.triangles(g)[0] == math.comb(n, 3)
    for n in (4, 5, 9):       # cycles of length > 3 have none
        assert oracle.triangles(graph_from_edges(n, [(i, (i + 1) % n) for i in range(n)]))[0] == 0
    assert oracle.triangles(graph_from_edges(3, [(0, 1), (1, 2), (2, 0)]))[0] == 1
    for n in (5, 8, 13):      # wheel: a hub joined to an n-cycle has n triangles
        edges = [(i, (i + 1) % n) for i in range(n)] + [(n, i) for i in range(n)]
        assert oracle.triangles(graph_from_edges(n + 1, edges))[0] == n
    edges = [(i, 4 + j) for i in range(4) for j in range(5)]   # K_{4,5}: bipartite
    assert oracle.triangles(graph_from_edges(9, edges))[0] == 0
    assert oracle.triangles(graph_from_edges(6, []))[0] == 0     # no edges


def test_relabel_invariance_and_given_orders():
    g = random_graph(60, 0.2, 7)
    total, _ = oracle.triangles(g)
    # the same graph under a random relabelling
    q = np.argsort(I.uniform01(np.arange(g.nrows, dtype=np.uint64), 8, 12))
    rows = np.repeat(np.arange(g.nrows), np.diff(g.row_ptr))
    h = I._coo_to_csr(g.nrows, q[rows], q[g.col.astype(np.int64)])
    assert oracle.triangles(h)[0] == total
    # any order gives the same total; per-vertex counts follow the order
    for perm in (np.arange(g.nrows), np.argsort(np.argsort(-np.diff(g.row_ptr), kind="stable")),
                 np.argsort(q)):
        t, per = oracle.triangles(g, perm)
        assert t == total and per.sum() == total
        assert np.array_equal(per, brute(g, perm)[1])
    with pytest.raises(ValueError):
        oracle.triangles(g, np.zeros(g.nrows, dtype=np.int64))


def test_degree_order():
    g = random_graph(50, 0.2, 9)
    perm = oracle.degree_order(g)
    deg = np.diff(g.row_ptr)
    inv = np.argsort(perm)
    assert np.array_equal(np.sort(perm), np.arange(g.nrows))
    assert np.all(np.diff(deg[inv]) >= 0)
    # ties in index order
    for a_, b_ in zip(inv[:-1], inv[1:]):
        if deg[a_] == deg[b_]:
            assert a_ < b_


@pytest.mark.parametrize("scale", [8, 11])
def test_rmat_against_scipy(scale):
    """R-MAT graphs of the benchmark's generator: the total equals
    sum((A*A) .* A) / 6 by scipy's sparse product."""
    sp = pytest.importorskip("scipy.sparse")
    g = I.rmat_symmetric(scale, 16, seed=1)
    a = sp.csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(g.nrows, g.nrows))
    ref = int(round((a @ a).multiply(a).sum())) // 6
    total, per = oracle.triangles(g)
    assert total == ref and per.sum() == total
