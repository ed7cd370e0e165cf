"""The roofline numerator of the bench line: bench.kernel_bytes for the
Galerkin products A*P and R*(AP) against the byte counts that follow from the
closed-form sizes (CSR offsets 8 B per row, 4 B column + 8 B value per
entry; every row of P is reached), evaluated from 1D aggregate counts."""
import numpy as np

import bench
from paper_1804_00695_gb300 import inputs as I


def _aggs_reached(n, halo):
    """Sum over fine points x of the number of aggregates floor(x'/3) with
    |x' - x| <= halo, 0 <= x' < n (1D factor of the Kronecker patterns)."""
    return sum(len({x2 // 3 for x2 in range(max(0, x - halo), min(n, x + halo + 1))}) for x in range(n))


def _ap_bytes(n):
    rows = n ** 3
    nnz_a = (3 * n - 2) ** 3
    nnz_p = _aggs_reached(n, 1) ** 3
    nnz_ap = _aggs_reached(n, 2) ** 3
    return 3 * 8 * rows + 12 * (nnz_a + nnz_p + nnz_ap)


def test_closed_form_sizes_at_128():
    assert _aggs_reached(128, 1) == 212 and _aggs_reached(128, 2) == 296
    assert _ap_bytes(128) == 1144796832


def test_kernel_bytes_matches_closed_form():
    n = 24
    a, p, r = I.galerkin_problem(n)
    # row offsets of AP from its Kronecker pattern (T^2 p in each dimension)
    one_d = np.array([len({x2 // 3 for x2 in range(max(0, x - 2), min(n, x + 3))}) for x in range(n)])
    # array indexed [z, y, x] flattened in C order: row i = x + n*y + n*n*z
    lens = np.einsum("k,j,i->kji", one_d, one_d, one_d).reshape(-1)
    ap_rp = np.zeros(n ** 3 + 1, dtype=np.int64)
    np.cumsum(lens, out=ap_rp[1:])
    allr = np.ones(a.nrows, dtype=bool)
    assert bench.kernel_bytes(a, p.row_ptr, ap_rp, allr, 8) == _ap_bytes(n)


def _rap_bytes(n):
    """R*(AP): R's offsets and entries (R = P^T: one row per aggregate, nnz(P)
    entries), every row of AP (each fine point lies in an aggregate, so R
    reaches all of them), RAP's offsets and entries (tridiagonal in each
    dimension over the m = ceil(n/3) aggregates: (3m - 2)^3 entries)."""
    m = -(-n // 3)
    nnz_p = _aggs_reached(n, 1) ** 3
    nnz_ap = _aggs_reached(n, 2) ** 3
    nnz_rap = (3 * m - 2) ** 3
    return 8 * m ** 3 + 12 * nnz_p + 8 * n ** 3 + 12 * nnz_ap + 8 * m ** 3 + 12 * nnz_rap


def test_step_bytes_at_128():
    """The whole Galerkin step's roofline numerator (the bench line's
    step_algorithmic_bytes): A*P plus R*(AP) at 128^3."""
    assert _rap_bytes(128) == 468179492
    assert _ap_bytes(128) + _rap_bytes(128) == 1612976324


def test_kernel_bytes_rap_matches_closed_form():
    import oracle
    n = 24
    a, p, r = I.galerkin_problem(n)
    ap = oracle.spgemm(a, p)
    rap = oracle.spgemm(r, I.Csr(a.nrows, p.ncols, ap.row_ptr, ap.col, ap.val))
    m = -(-n // 3)
    c = np.arange(m)
    one_d = np.where((c == 0) | (c == m - 1), 2, 3)     # aggregates c-1, c, c+1 that exist
    lens = np.einsum("k,j,i->kji", one_d, one_d, one_d).reshape(-1)
    rap_rp = np.zeros(m ** 3 + 1, dtype=np.int64)
    np.cumsum(lens, out=rap_rp[1:])
    assert np.array_equal(rap_rp, rap.row_ptr)        # the closed-form pattern is the product's
    allr = np.ones(r.nrows, dtype=bool)
    assert bench.kernel_bytes(r, ap.row_ptr, rap_rp, allr, 8) == _rap_bytes(n)


def test_narrow_rows_rule():
    """bench.narrow_numeric_rows (which rows' bytes the narrow kernel's
    roofline counts): every row of both Galerkin products is narrow; a row
    whose B rows span more than 128 blocks of 32 columns, one with more than
    32 outputs and one with more than 8192 products are not."""
    import oracle
    n = 24
    a, p, r = I.galerkin_problem(n)
    ap = oracle.spgemm(a, p)
    apc = I.Csr(a.nrows, p.ncols, ap.row_ptr, ap.col, ap.val)
    rap = oracle.spgemm(r, apc)
    assert bench.narrow_numeric_rows(a, p, ap.row_ptr, bench.row_flops_np(a, p.row_ptr)).all()
    assert bench.narrow_numeric_rows(r, apc, rap.row_ptr, bench.row_flops_np(r, ap.row_ptr)).all()

    def csr(rows, ncols):
        rp = np.concatenate([[0], np.cumsum([len(x) for x in rows])]).astype(np.int64)
        col = np.array([c for x in rows for c in x], dtype=np.int32)
        return I.Csr(len(rows), ncols, rp, col, np.ones(len(col)))

    ncols = 40000
    # B: row 0 = column 0; row 1 = column 128*32 - 1 (block 127); row 2 = column 128*32 (block 128);
    # row 3 = 33 columns; row 4 = 9000 columns in blocks 0..281 (not used alone)
    b = csr([[0], [128 * 32 - 1], [128 * 32], list(range(100, 133)), list(range(9000))], ncols)
    a2 = csr([[0, 1], [0, 2], [3], [0]], 5)
    res = oracle.spgemm(a2, b)
    got = bench.narrow_numeric_rows(a2, b, res.row_ptr, bench.row_flops_np(a2, b.row_ptr))
    assert got.tolist() == [True, False, False, True]
    # products above 8192 alone: three entries of A on a B row of 4000 columns
    # (blocks 0..124: inside the window, 375 pairs), the output count given as 32
    b3 = csr([list(range(4000))], ncols)
    a3 = csr([[0, 0, 0]], 1)     # repeated column only for the count's sake (the oracle is not run)
    fl = bench.row_flops_np(a3, b3.row_ptr)
    assert fl.tolist() == [12000]
    assert not bench.narrow_numeric_rows(a3, b3, np.array([0, 32]), fl)[0]
    assert bench.narrow_numeric_rows(a3, b3, np.array([0, 32]), np.array([8192]))[0]
