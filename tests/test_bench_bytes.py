"""The roofline numerator of the bench line: bench.kernel_bytes for the
Galerkin A*P product against the byte count that follows from the
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
