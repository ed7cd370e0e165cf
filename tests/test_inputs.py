"""The seeded input generators against their recipes: the counter-based
generator against the published SplitMix64 sequence, the random batch
matrices against the row-length and value distributions they are defined
by, the batch sizes against their log-uniform law, the R-MAT graph against
its structural invariants and the stencils against their closed-form sizes."""
import math

import numpy as np

from paper_1804_00695_gb300 import inputs as I


def test_splitmix64_published_sequence():
    # SplitMix64 from state 0: its first three outputs as published with the
    # generator's reference implementation
    got = I.splitmix64(np.arange(3, dtype=np.uint64), 0, 0)
    assert [int(x) for x in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform01_range_and_streams():
    c = np.arange(200000, dtype=np.uint64)
    u = I.uniform01(c, 7)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    v = I.uniform01(c, 7, 1)
    assert abs(np.corrcoef(u, v)[0, 1]) < 0.01          # streams are independent
    assert np.array_equal(u, I.uniform01(c, 7))          # reproducible


def test_random_square_rows_and_values():
    n = 3000
    m = I.random_square(n, 11)
    lens = np.diff(m.row_ptr)
    assert lens.min() >= 4 and lens.max() <= 32
    assert set(np.unique(lens).tolist()) == set(range(4, 33))       # U{4..32}
    assert abs(lens.mean() - 18.0) < 0.5
    for i in range(0, n, 97):
        row = m.col[m.row_ptr[i]:m.row_ptr[i + 1]]
        assert np.all(np.diff(row) > 0) and row.min() >= 0 and row.max() < n
    v = m.val.astype(np.float64)
    assert abs(v.mean()) < 0.02 and abs(v.std() - 1.0) < 0.02      # N(0,1)
    assert m.val.dtype == np.float32


def test_batch_sizes_log_uniform():
    s = np.array(I.batch_sizes(4096, 1024, 65536, 1), dtype=np.float64)
    assert s.min() >= 1024 and s.max() < 65536
    x = (np.log(s) - math.log(1024)) / (math.log(65536) - math.log(1024))
    assert abs(x.mean() - 0.5) < 0.02 and abs(x.var() - 1 / 12) < 0.01
    assert I.batch_sizes(8, 1024, 65536, 1) == I.batch_sizes(8, 1024, 65536, 1)


def test_rmat_structure():
    g = I.rmat_symmetric(10, 16, seed=1)
    n = 1 << 10
    assert g.nrows == g.ncols == n
    d = g.to_dense()
    assert np.array_equal(d, d.T) and np.all(np.diag(d) == 0)
    assert set(np.unique(g.val).tolist()) == {1.0}
    deg = np.diff(g.row_ptr)
    assert g.nnz <= 2 * 16 * n
    assert deg.max() > 10 * deg.mean()       # the skew of a=.57: hub vertices
    assert deg[0] == deg.max()               # vertex 0 takes the a-quadrant at every level


def test_laplace3d_closed_form_sizes():
    for n in (3, 5, 8):
        m = I.laplace3d_27pt(n)
        assert m.nrows == n ** 3 and m.nnz == (3 * n - 2) ** 3
        rows = np.repeat(np.arange(m.nrows), np.diff(m.row_ptr))
        diag = m.val[rows == m.col]
        assert np.all(diag == 26.0) and np.all(m.val[rows != m.col] == -1.0)
