"""GPU parity of triangle counting by the masked product L*L .* L
(spgemm_triangles) against the CPU oracle, through the C ABI: the count is
exact; the labels (unique up to the order of vertices of equal degree) are
checked to be a permutation with non-decreasing degrees, and the per-vertex
counts are compared exactly with the oracle run on the same labels.  Light
rows (a warp each), heavy rows (a block each, bitmap in shared memory) and a
graph too wide for the shared bitmap (bitmap in global memory)."""
import math

import numpy as np
import pytest

import oracle
import paper_1804_00695_gb300 as sg
from paper_1804_00695_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h(cuda_lib):
    return sg.Handle()


def graph_from_edges(n, edges):
    e = np.array(edges, dtype=np.int64).reshape(-1, 2)
    return I._coo_to_csr(n, np.concatenate([e[:, 0], e[:, 1]]), np.concatenate([e[:, 1], e[:, 0]]))


def check(h, g):
    G = sg.Csr.from_host(g, "cuda", np.float32)
    total, perm, vc = h.triangles(G, labels=True)
    ref_total, _ = oracle.triangles(g)
    assert total == ref_total
    perm = perm.cpu().numpy()
    assert np.array_equal(np.sort(perm), np.arange(g.nrows))
    deg = np.diff(g.row_ptr)
    assert np.all(np.diff(deg[np.argsort(perm)]) >= 0)
    t2, per = oracle.triangles(g, perm)
    assert t2 == total
    assert np.array_equal(vc.cpu().numpy(), per)
    assert h.triangles(G) == total          # without the optional outputs
    return total


@pytest.mark.parametrize("scale", [6, 10, 13, 16])
def test_rmat(h, scale):
    assert check(h, I.rmat_symmetric(scale, 16, seed=1)) > 0


def test_closed_forms_and_edge_cases(h):
    n = 300                                   # complete graph: heavy rows
    g = graph_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    assert check(h, g) == math.comb(n, 3)
    m = 40                                    # wheel: hub plus an m-cycle
    g = graph_from_edges(m + 1, [(i, (i + 1) % m) for i in range(m)] + [(m, i) for i in range(m)])
    assert check(h, g) == m
    g = graph_from_edges(30, [(i, 10 + j) for i in range(10) for j in range(20)])   # bipartite
    assert check(h, g) == 0
    z = I.Csr(7, 7, np.zeros(8, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    assert check(h, z) == 0
    # self loops are ignored
    g = I.rmat_symmetric(9, 8, seed=5)
    rows = np.repeat(np.arange(g.nrows), np.diff(g.row_ptr))
    loops = np.arange(0, g.nrows, 7)
    gl = I._coo_to_csr(g.nrows, np.concatenate([rows, loops]), np.concatenate([g.col.astype(np.int64), loops]))
    G = sg.Csr.from_host(gl, "cuda", np.float32)
    assert h.triangles(G) == oracle.triangles(g)[0]


def test_wide_graph_global_bitmap(h):
    """2^21 vertices (more columns than the shared-memory bitmap holds): a
    clique of 200 vertices spread over the ids, plus a random sparse graph."""
    n = 1 << 21
    ids = (np.arange(200, dtype=np.int64) * 10007) % n
    edges = [(int(ids[i]), int(ids[j])) for i in range(200) for j in range(i + 1, 200)]
    u = I.uniform01(np.arange(40000, dtype=np.uint64), 3, 13)
    v = I.uniform01(np.arange(40000, dtype=np.uint64), 4, 13)
    a, b = (u * n).astype(np.int64), (v * n).astype(np.int64)
    keep = a != b
    edges += list(zip(a[keep].tolist(), b[keep].tolist()))
    g = graph_from_edges(n, edges)
    total = check(h, g)
    assert total >= math.comb(200, 3)
