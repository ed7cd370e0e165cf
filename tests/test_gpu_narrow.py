"""GPU parity of the narrow-row kernels (rows of C inside a window of 128
blocks of 32 columns, counted and multiplied over a dense window of the
compressed column sets) against the CPU oracle, through the C ABI: pattern
bit-exact, values within the stated tolerance; with the window at its limit
and one block past it, unsorted rows, long rows of A, rows with more than 32
outputs or more than 8192 products (which leave the narrow numeric kernel),
every lanes option, and the path switched off."""
import numpy as np
import pytest

import oracle
import paper_1804_00695_gb300 as sg
from paper_1804_00695_gb300 import inputs as I
from gpu_helpers import assert_matches, host_csr, oracle_product, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h(cuda_lib):
    return sg.Handle()


def run(h, a, b, dtype=np.float64):
    c = h.spgemm(to_dev(a, dtype), to_dev(b, dtype))
    h.check()
    return c


def _csr(nrows, ncols, rows, cols, seed, shuffle=False):
    """CSR from (row, col) lists (deduplicated), values uniform in [-0.5, 0.5)."""
    key = np.unique(np.asarray(rows, dtype=np.int64) * ncols + np.asarray(cols, dtype=np.int64))
    r, c = key // ncols, (key % ncols).astype(np.int32)
    rp = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=nrows), out=rp[1:])
    if shuffle:
        for i in range(nrows):
            s0, s1 = int(rp[i]), int(rp[i + 1])
            perm = np.argsort(I.splitmix64(np.arange(s1 - s0, dtype=np.uint64), seed + i))
            c[s0:s1] = c[s0:s1][perm]
    return I.Csr(nrows, ncols, rp, c, I.uniform01(np.arange(len(key), dtype=np.uint64), seed) - 0.5)


@pytest.mark.parametrize("n", [9, 16, 29])
@pytest.mark.parametrize("narrow", [1, 0])
def test_galerkin_narrow_on_off(h, n, narrow):
    """Both Galerkin products with the narrow path on (every row narrow) and
    off (hash kernels only); R*(AP) against the oracle on the device AP."""
    a, p, r = I.galerkin_problem(n)
    h.set_option(sg.OPT_NARROW, narrow)
    try:
        ap = run(h, a, p)
        sym, num = h.bin_counts()
        assert_matches(ap, oracle.spgemm(a, p), "f64")
        if narrow:
            assert sym[sg.BIN_NARROW] == a.nrows and num[sg.BIN_NARROW] == a.nrows, (sym, num)
        else:
            assert sym[sg.BIN_NARROW] == 0 and num[sg.BIN_NARROW] == 0
        rap = h.spgemm(to_dev(r), ap)
        h.check()
        sym, num = h.bin_counts()
        assert_matches(rap, oracle.spgemm(r, host_csr(ap)), "f64")
        if narrow:
            assert num[sg.BIN_NARROW] == r.nrows, num
    finally:
        h.set_option(sg.OPT_NARROW, 1)


def test_window_limit(h):
    """Row i of C holds the columns 32*k1 and 32*k2 + 31: a window of k2-k1+1
    blocks.  127 and 128 blocks apart end at the limit (narrow) and one block
    past it (hash kernels); windows at the first and last blocks of B."""
    nblk = 600
    ncols = 32 * nblk
    b = _csr(nblk, ncols, list(range(nblk)) * 2, [32 * k for k in range(nblk)] + [32 * k + 31 for k in range(nblk)], 3)
    rows, cols = [], []
    gaps = [0, 1, 126, 127, 128, 300]
    starts = [0, 5, 200, nblk - 128, nblk - 129, 17]
    for i, (s, gp) in enumerate(zip(starts, gaps * 1)):
        rows += [i, i]
        cols += [s, min(s + gp, nblk - 1)]
    a = _csr(len(gaps), nblk, rows, cols, 4)
    for dt, tag in ((np.float64, "f64"), (np.float32, "f32")):
        c = run(h, a, b, dt)
        assert_matches(c, oracle_product(a, b, dt), tag)
        sym, num = h.bin_counts()
        narrow_rows = sum(1 for s, gp in zip(starts, gaps) if min(s + gp, nblk - 1) - s + 1 <= 128)
        assert sym[sg.BIN_NARROW] == narrow_rows and num[sg.BIN_NARROW] == narrow_rows, (sym, num)


def _banded(nrows, ncols, width, per_row, seed, shuffle):
    """Row i: per_row distinct columns within [c0, c0 + width), c0 following i."""
    rows, cols = [], []
    for i in range(nrows):
        c0 = (i * (ncols - width)) // max(1, nrows - 1)
        pick = I.splitmix64(np.arange(per_row, dtype=np.uint64), seed * 1000 + i) % np.uint64(width)
        rows += [i] * per_row
        cols += (c0 + pick.astype(np.int64)).tolist()
    return _csr(nrows, ncols, rows, cols, seed, shuffle)


@pytest.mark.parametrize("shuffle", [False, True])
@pytest.mark.parametrize("lanes", [(0, 0), (4, 4), (8, 8), (16, 16), (32, 4)])
def test_banded_lanes_and_unsorted(h, shuffle, lanes):
    """Banded operands: rows of A with 3..70 entries (longer than a lane
    group's share and, for some, than 32), rows of B with 1..12 entries,
    unsorted rows, every lanes option of both narrow kernels, FP64 and FP32."""
    ls, ln = lanes
    rows, cols = [], []
    for i in range(700):
        k = 3 + (i * 37) % 68
        c0 = (i * 780) // 699
        pick = I.splitmix64(np.arange(k, dtype=np.uint64), 7000 + i) % np.uint64(120)
        rows += [i] * k
        cols += (c0 + pick.astype(np.int64)).tolist()
    a = _csr(700, 900, rows, cols, 5, shuffle)
    rows, cols = [], []
    for k in range(900):
        m = 1 + (k * 5) % 12
        c0 = (k * 2800) // 899
        pick = I.splitmix64(np.arange(m, dtype=np.uint64), 9000 + k) % np.uint64(60)
        rows += [k] * m
        cols += (c0 + pick.astype(np.int64)).tolist()
    b = _csr(900, 2900, rows, cols, 6, shuffle)
    h.set_option(sg.OPT_LANES_NARROW_SYMBOLIC, ls)
    h.set_option(sg.OPT_LANES_NARROW_NUMERIC, ln)
    try:
        for dt, tag in ((np.float64, "f64"), (np.float32, "f32")):
            c = run(h, a, b, dt)
            assert_matches(c, oracle_product(a, b, dt), tag)
            sym, num = h.bin_counts()
            assert sym[sg.BIN_NARROW] > 0 and num[sg.BIN_NARROW] > 0, (sym, num)
    finally:
        h.set_option(sg.OPT_LANES_NARROW_SYMBOLIC, 0)
        h.set_option(sg.OPT_LANES_NARROW_NUMERIC, 0)


def test_narrow_rows_leaving_the_numeric_kernel(h):
    """Rows narrow in the symbolic phase but with more than 32 outputs, or
    more than 8192 products, are multiplied by the other kernels; rows with
    at most 32 outputs and 8192 products stay; all against the oracle."""
    ncols, nb = 3000, 6000
    rows, cols = [], []
    # B: row k holds the 30 columns [100*(k%20), +30): 300 rows share them
    for k in range(nb):
        c0 = 100 * (k % 20)
        rows += [k] * 30
        cols += list(range(c0, c0 + 30))
    b = _csr(nb, ncols, rows, cols, 8)
    rows, cols = [], []
    for i in range(300):
        g = i % 19
        if i % 3 == 0:          # 300 rows of B of one group: 9000 products, 30 outputs
            ks = list(range(g, nb, 20))
        elif i % 3 == 1:        # rows of two neighbouring groups: 60 outputs
            ks = [g, g + 1, g + 20, g + 21]
        else:                   # rows of one group: 30 outputs
            ks = [g, g + 20, g + 40]
        rows += [i] * len(ks)
        cols += ks
    a = _csr(300, nb, rows, cols, 9)
    fl = oracle.row_flops(a, b)
    c = run(h, a, b)
    assert_matches(c, oracle.spgemm(a, b), "f64")
    sym, num = h.bin_counts()
    assert sym[sg.BIN_NARROW] == 300, sym
    lens = np.diff(c.row_ptr.cpu().numpy())
    expect_num = int(np.sum((lens <= 32) & (fl <= 8192)))
    assert num[sg.BIN_NARROW] == expect_num == 100, (num, expect_num)


def test_narrow_edge_values(h):
    """Explicit zeros stay in the pattern, empty rows of A and B, A*I = A
    exactly, and the double-word option (narrow rows accumulate natively)."""
    a = _banded(200, 400, 50, 7, 11, True)
    keep = np.ones(a.nnz, dtype=bool)
    for i in range(0, 200, 9):                 # some empty rows of A
        keep[a.row_ptr[i]:a.row_ptr[i + 1]] = False
    rows = np.repeat(np.arange(a.nrows), np.diff(a.row_ptr))[keep]
    a = _csr(200, 400, rows, a.col[keep], 12, True)
    b = _banded(400, 800, 40, 5, 13, True)
    bz = I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, np.where(np.arange(b.nnz) % 4 == 0, 0.0, b.val))
    c = run(h, a, bz)
    assert_matches(c, oracle.spgemm(a, bz), "f64")
    eye = I.Csr(400, 400, np.arange(401, dtype=np.int64), np.arange(400, dtype=np.int32), np.ones(400))
    c = run(h, a, eye)
    ref = oracle.spgemm(a, eye)
    assert np.array_equal(c.col.cpu().numpy(), ref.col) and np.array_equal(c.val.cpu().numpy(), ref.val)
    h.set_option(sg.OPT_F64_NATIVE, 0)
    try:
        c = run(h, a, b)
    finally:
        h.set_option(sg.OPT_F64_NATIVE, 1)
    assert_matches(c, oracle.spgemm(a, b), "f64")
