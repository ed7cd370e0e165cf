"""GPU parity of the two-phase SpGEMM (symbolic + numeric) against the CPU
oracle, through the C ABI: pattern bit-exact, values within the stated
tolerance, on the workloads' generators at several sizes and on edge cases."""
import numpy as np
import pytest

import oracle
import paper_1804_00695_gb300 as sg
from paper_1804_00695_gb300 import inputs as I
from gpu_helpers import assert_matches, host_csr, oracle_product, to_dev

pytestmark = pytest.mark.gpu


def run(h, a, b, dtype=np.float64):
    A, B = to_dev(a, dtype), to_dev(b, dtype)
    c = h.spgemm(A, B)
    h.check()
    return c


@pytest.fixture(scope="module")
def h(cuda_lib):
    return sg.Handle()


def test_laplace2d_64_squared(h):
    a = I.laplace2d_5pt(64)
    c = run(h, a, a)
    ref = oracle.spgemm(a, a)
    assert c.nnz == 51972
    assert_matches(c, ref, "f64")
    # closed form: exact integers
    assert np.array_equal(c.val.cpu().numpy(), ref.val)


@pytest.mark.parametrize("n", [9, 16, 29])
def test_galerkin_small(h, n):
    a, p, r = I.galerkin_problem(n)
    ap = run(h, a, p)
    ref_ap = oracle.spgemm(a, p)
    assert_matches(ap, ref_ap, "f64")
    R = to_dev(r)
    rap = h.spgemm(R, ap)
    h.check()
    # the second product consumes the device AP: the oracle takes the same
    # values as its input, so the stated bound holds with nothing added
    assert_matches(rap, oracle.spgemm(r, host_csr(ap)), "f64")


def test_galerkin_128_full(h):
    """The 128^3 Galerkin product at full size, every entry."""
    a, p, r = I.galerkin_problem(128)
    A, P, R = to_dev(a), to_dev(p), to_dev(r)
    ap = h.spgemm(A, P)
    h.check()
    ref_ap = oracle.spgemm(a, p)
    assert ap.nnz == 25934336
    assert_matches(ap, ref_ap, "f64")
    rap = h.spgemm(R, ap)
    h.check()
    assert rap.nnz == 2048383
    assert_matches(rap, oracle.spgemm(r, host_csr(ap)), "f64")


@pytest.mark.parametrize("scale", [8, 11])
def test_rmat_f32(h, scale):
    g = I.rmat_symmetric(scale, 16, seed=1)
    c = run(h, g, g, np.float32)
    ref = oracle_product(g, g, np.float32)
    assert_matches(c, ref, "f32")
    assert np.array_equal(c.val.double().cpu().numpy(), ref.val)  # integer counts: exact


@pytest.mark.parametrize("dtype,tag", [(np.float64, "f64"), (np.float32, "f32")])
@pytest.mark.parametrize("shape,dens,seed", [((50, 70, 40), 0.1, 1), ((300, 200, 500), 0.03, 2),
                                             ((1, 1000, 1), 0.9, 3), ((257, 64, 3000), 0.02, 4)])
def test_random_unsorted(h, dtype, tag, shape, dens, seed):
    m, k, n = shape
    a = I.random_csr(m, k, dens, seed, shuffle_cols=True)
    b = I.random_csr(k, n, dens, seed + 50, shuffle_cols=True)
    c = run(h, a, b, dtype)
    assert_matches(c, oracle_product(a, b, dtype), tag)


def _spread_rows(widths, ncols, seed):
    rows, cols = [], []
    for i, w in enumerate(widths):
        stride = max(1, ncols // w)
        cols.extend(((np.arange(w) * stride + i * 13) % ncols).tolist())
        rows.extend([i] * w)
    key = np.unique(np.array(rows, dtype=np.int64) * ncols + np.array(cols))
    rp = np.zeros(len(widths) + 1, dtype=np.int64)
    np.cumsum(np.bincount(key // ncols, minlength=len(widths)), out=rp[1:])
    return I.Csr(len(widths), ncols, rp, (key % ncols).astype(np.int32),
                 I.uniform01(np.arange(len(key), dtype=np.uint64), seed) - 0.5)


def _eye(n):
    return I.Csr(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n))


@pytest.mark.parametrize("ncols", [300000, 2000000])
def test_every_bin_both_phases(h, ncols):
    """Rows sized to land in every bin (1..6) of both phases: the shared-memory
    maps, the global second-level map, and the shared (300k columns) or global
    (2M columns) symbolic bitmap."""
    widths = [3, 12, 25, 40, 150, 600, 2500, 9000, 30000]
    a = _spread_rows(widths, ncols, 5)
    eye = _eye(ncols)
    c = run(h, a, eye)
    assert_matches(c, oracle.spgemm(a, eye), "f64")
    sym, num = h.bin_counts()
    assert all(num[b] > 0 for b in range(1, 7)), num
    assert all(sym[b] > 0 for b in range(1, 7)), sym
    c = run(h, a, eye, np.float32)
    assert_matches(c, oracle_product(a, eye, np.float32), "f32")
    h.set_option(sg.OPT_F64_NATIVE, 0)   # double-word accumulation
    c = run(h, a, eye)
    h.set_option(sg.OPT_F64_NATIVE, 1)
    assert_matches(c, oracle.spgemm(a, eye), "f64")


@pytest.mark.parametrize("native", [0, 1])
@pytest.mark.parametrize("lanes", [0, 4, 8, 16, 32])
def test_lane_options_galerkin(h, native, lanes):
    """Every lanes-per-row choice and both FP64 accumulation modes."""
    a, p, r = I.galerkin_problem(12)
    h.set_option(sg.OPT_F64_NATIVE, native)
    h.set_option(sg.OPT_LANES_NUMERIC, lanes)
    h.set_option(sg.OPT_LANES_SYMBOLIC, lanes)
    try:
        for x, y in ((a, p), (r, a)):
            c = run(h, x, y)
            assert_matches(c, oracle.spgemm(x, y), "f64")
    finally:
        h.set_option(sg.OPT_F64_NATIVE, 1)
        h.set_option(sg.OPT_LANES_NUMERIC, 0)
        h.set_option(sg.OPT_LANES_SYMBOLIC, 0)


@pytest.mark.parametrize("shape", [(60, 50, 70, 0.2), (40, 200, 30, 0.3)])
def test_double_word_range_fallback(h, shape):
    """Values outside the double-word range (tiny, huge) take the native
    path and still meet the FP64 tolerance; zeros are exact.  Rows of A
    shorter and longer than one staging batch (32 entries)."""
    m, k, n, dens = shape
    a = I.random_csr(m, k, dens, 31)
    b = I.random_csr(k, n, dens, 32)
    av = a.val.copy()
    av[::7] *= 1e-30      # below 2^-32: those rows go native
    bv = b.val.copy()
    h.set_option(sg.OPT_F64_NATIVE, 0)   # double-word accumulation
    try:
        for scale_b in (1.0, 1e25):   # 1e25 > 2^32: the whole call goes native
            a2 = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, av)
            b2 = I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, bv * scale_b)
            c = run(h, a2, b2)
            assert_matches(c, oracle.spgemm(a2, b2), "f64")
    finally:
        h.set_option(sg.OPT_F64_NATIVE, 1)


@pytest.mark.parametrize("shuffle", [False, True])
def test_huge_rows_window_and_hash(h, shuffle):
    """Rows with more than 4096 outputs: sorted rows of B take the windowed
    dense accumulator, unsorted ones the two-level hash map."""
    a = _spread_rows([3, 9000, 700, 15000], 20000, 17)
    b = I.random_csr(20000, 70000, 0.0003, 18, shuffle_cols=shuffle)
    for dt, tag in ((np.float64, "f64"), (np.float32, "f32")):
        c = run(h, a, b, dt)
        assert_matches(c, oracle_product(a, b, dt), tag)
    sym, num = h.bin_counts()
    assert num[6] > 0


def _strided_rows(nrows, ncols, widths, mult, step, seed):
    """Row i holds widths[i % len(widths)] columns (i*mult + t*step) mod ncols."""
    rows, cols = [], []
    for i in range(nrows):
        w = widths[i % len(widths)]
        cols.extend(((i * mult + np.arange(w, dtype=np.int64) * step) % ncols).tolist())
        rows.extend([i] * w)
    key = np.unique(np.array(rows, dtype=np.int64) * ncols + np.array(cols, dtype=np.int64))
    rp = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(np.bincount(key // ncols, minlength=nrows), out=rp[1:])
    return I.Csr(nrows, ncols, rp, (key % ncols).astype(np.int32),
                 I.uniform01(np.arange(len(key), dtype=np.uint64), seed) - 0.5)


@pytest.mark.parametrize("small_cap", [32, 16])
@pytest.mark.parametrize("ncols", [9000, 25000, 50000, 300000])
def test_medium_rows_every_span(h, ncols, small_cap):
    """Rows of 17..1024 outputs whose columns span at most 512 blocks of 32
    (first dense rank accumulator), 512..1024 blocks with at most 512 outputs
    (second), up to 2048 blocks (third), or more (hash maps), in FP32,
    double-word FP64 and native FP64."""
    nb = 3000
    a = _strided_rows(1200, nb, [1, 2, 5, 9, 17, 30, 44], 7, 11, 41)
    b = _strided_rows(nb, ncols, [20, 23], 37, ncols // 23 + 1, 42)
    h.set_option(sg.OPT_SMALL_CAP, small_cap)
    h.set_timing(True)
    h.reset_timings()
    try:
        for dt, tag, native in ((np.float64, "f64", 0), (np.float64, "f64", 1), (np.float32, "f32", 0)):
            h.set_option(sg.OPT_F64_NATIVE, native)
            c = run(h, a, b, dt)
            assert_matches(c, oracle_product(a, b, dt), tag)
        labels = set(h.timings())
    finally:
        h.set_option(sg.OPT_F64_NATIVE, 1)
        h.set_option(sg.OPT_SMALL_CAP, 32)
        h.set_timing(False)
    sym, num = h.bin_counts()
    assert num[2] > 0 and num[3] > 0 and num[4] > 0, num
    want = {9000: "numeric.rank512", 25000: "numeric.rank1024", 50000: "numeric.rank2048",
            300000: "numeric.wide"}[ncols]
    assert any(l.startswith(want) for l in labels), labels


def test_timing_modes(h):
    """Timing mode 2 brackets only the numeric-phase launches with events,
    mode 1 every launch; the product is the same either way."""
    a, p, _ = I.galerkin_problem(10)
    ref = oracle_product(a, p, np.float64)
    got = {}
    try:
        for mode in (1, 2):
            h.set_timing(mode)
            h.reset_timings()
            c = run(h, a, p)
            assert_matches(c, ref, "f64")
            got[mode] = set(h.timings())
    finally:
        h.set_timing(False)
    assert all(l.startswith("numeric") for l in got[2]) and "numeric.narrow" in got[2], got[2]
    assert got[2] < got[1] and any(l.startswith("symbolic") for l in got[1]), got[1]
    with pytest.raises(sg.SpgemmError):
        h.set_timing(3)


def test_window_long_and_short_b_rows(h):
    """Rows with more than 4096 outputs over sorted B whose rows are short
    (walked by one thread per a_ik, a few entries per window) or long (more
    than 256 entries, walked by whole warps), in FP32 and FP64."""
    a = _strided_rows(40, 3000, [60, 97, 130], 13, 29, 71)
    b = _strided_rows(3000, 200000, [3, 20, 400, 3000, 17], 101, 61, 72)
    for dt, tag in ((np.float64, "f64"), (np.float32, "f32")):
        c = run(h, a, b, dt)
        assert_matches(c, oracle_product(a, b, dt), tag)
    sym, num = h.bin_counts()
    assert num[6] > 0, num


def test_heavy_rows_random(h):
    """Rows whose products overlap heavily (many insertions per key)."""
    a = _spread_rows([5, 50, 500, 5000], 6000, 7)
    b = I.random_csr(6000, 3000, 0.01, 8)
    for dt, tag in ((np.float64, "f64"), (np.float32, "f32")):
        c = run(h, a, b, dt)
        assert_matches(c, oracle_product(a, b, dt), tag)


def test_edge_cases(h):
    # empty A (no rows)
    e = I.Csr(0, 5, np.zeros(1, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0))
    b = I.random_csr(5, 7, 0.5, 9)
    c = run(h, e, b)
    assert c.nnz == 0 and c.row_ptr.cpu().tolist() == [0]
    # all rows empty
    z = I.Csr(6, 5, np.zeros(7, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0))
    c = run(h, z, b)
    assert c.nnz == 0 and c.row_ptr.cpu().tolist() == [0] * 7
    # B with a single column, ncols = 1
    a = I.random_csr(40, 30, 0.3, 10)
    b1 = I.random_csr(30, 1, 0.6, 11)
    c = run(h, a, b1)
    assert_matches(c, oracle.spgemm(a, b1), "f64")
    # A * I = A (sorted): exact in native FP64, within tolerance as double-words
    eye = I.Csr(30, 30, np.arange(31, dtype=np.int64), np.arange(30, dtype=np.int32), np.ones(30))
    h.set_option(sg.OPT_F64_NATIVE, 0)
    c = run(h, a, eye)
    h.set_option(sg.OPT_F64_NATIVE, 1)
    assert np.array_equal(c.col.cpu().numpy(), a.col)
    assert np.all(np.abs(c.val.cpu().numpy() - a.val) <= 1e-12 * np.abs(a.val))
    c = run(h, a, eye)
    assert np.array_equal(c.col.cpu().numpy(), a.col) and np.array_equal(c.val.cpu().numpy(), a.val)
    # explicit zeros stay in the pattern
    az = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, np.zeros(a.nnz))
    c = run(h, az, eye)
    assert c.nnz == a.nnz and not c.val.any()


def test_errors(h):
    a = I.random_csr(10, 8, 0.3, 12)
    b = I.random_csr(9, 8, 0.3, 13)
    with pytest.raises(sg.SpgemmError) as ei:
        h.symbolic(to_dev(a), to_dev(b))
    assert ei.value.status == 2  # dimension mismatch
    bad = I.Csr(10, 8, a.row_ptr, a.col.copy(), a.val)
    bad.col[3] = 8 if bad.nnz > 3 else 0
    b8 = I.random_csr(8, 8, 0.3, 14)
    with pytest.raises(sg.SpgemmError) as ei:
        h.symbolic(to_dev(bad), to_dev(b8))
    assert ei.value.status == 3  # index out of range
    A, B = to_dev(a), to_dev(b8)
    rp, nnz = h.symbolic(A, B)
    A2 = to_dev(a)
    with pytest.raises(sg.SpgemmError) as ei:
        h.numeric(A2, B, rp, nnz)
    assert ei.value.status == 8  # numeric without matching symbolic
    h.numeric(A, B, rp, nnz)
    h.check()


def test_row_flops_and_compression(h):
    a = I.random_csr(200, 300, 0.05, 15, shuffle_cols=True)
    b = I.laplace2d_5pt(int(np.sqrt(300)) + 1)
    b = I.random_csr(300, 900, 0.05, 16)
    A, B = to_dev(a), to_dev(b)
    assert np.array_equal(h.row_flops(A, B).cpu().numpy(), oracle.row_flops(a, b))
    cnt, pairs = h.compress(B)
    rp, blk, mask = oracle.compress_rows(b)          # sorted input: canonical form
    cnt = cnt.cpu().numpy()
    pairs = pairs.cpu().numpy().view(np.uint32)
    assert np.array_equal(cnt, np.diff(rp))
    for k in range(b.nrows):
        got = pairs[b.row_ptr[k]:b.row_ptr[k] + cnt[k]]
        assert np.array_equal(got[:, 0], blk[rp[k]:rp[k + 1]].astype(np.uint32))
        assert np.array_equal(got[:, 1], mask[rp[k]:rp[k + 1]])
    # unsorted rows: the decoded sets still equal the column sets
    cnt2, pairs2 = h.compress(A)
    cnt2 = cnt2.cpu().numpy(); pairs2 = pairs2.cpu().numpy().view(np.uint32)
    for i in range(a.nrows):
        s = set(a.col[a.row_ptr[i]:a.row_ptr[i + 1]].tolist())
        dec = set()
        for kb, mk in pairs2[a.row_ptr[i]:a.row_ptr[i] + cnt2[i]]:
            dec.update(32 * int(kb) + t for t in range(32) if (int(mk) >> t) & 1)
        assert dec == s


def test_compression_long_rows(h):
    """Rows longer than 128 entries (compressed by a warp each): sorted rows
    with dense runs crossing the 32-entry steps (blocks full of columns) and
    sparse stretches, against the canonical compression; unsorted long rows,
    against the runs of equal blocks in storage order."""
    rows, cols = [], []
    for i in range(60):
        w = 129 + 37 * i
        dense = np.arange(w // 2) + 64 * (i % 5)                 # runs of 32 columns per block
        sparse = 5000 + np.arange(w - w // 2) * (7 + i % 3)
        c = np.unique(np.concatenate([dense, sparse]))
        rows += [i] * len(c)
        cols += c.tolist()
    key = np.array(rows, dtype=np.int64) * 100000 + np.array(cols, dtype=np.int64)
    b = I.Csr(60, 100000, np.concatenate([[0], np.cumsum(np.bincount(key // 100000, minlength=60))]).astype(np.int64),
              (key % 100000).astype(np.int32), np.ones(len(key)))
    cnt, pairs = h.compress(to_dev(b))
    rp, blk, mask = oracle.compress_rows(b)
    cnt = cnt.cpu().numpy()
    pairs = pairs.cpu().numpy().view(np.uint32)
    assert np.array_equal(cnt, np.diff(rp))
    for k in range(b.nrows):
        got = pairs[b.row_ptr[k]:b.row_ptr[k] + cnt[k]]
        assert np.array_equal(got[:, 0], blk[rp[k]:rp[k + 1]].astype(np.uint32))
        assert np.array_equal(got[:, 1], mask[rp[k]:rp[k + 1]])
    # the same rows with their entries permuted: runs of equal blocks in
    # storage order, each run one pair
    order = np.lexsort((I.uniform01(np.arange(b.nnz, dtype=np.uint64), 19), np.repeat(np.arange(60), np.diff(b.row_ptr))))
    bu = I.Csr(60, 100000, b.row_ptr, b.col[order], b.val)
    cnt2, pairs2 = h.compress(to_dev(bu))
    cnt2 = cnt2.cpu().numpy(); pairs2 = pairs2.cpu().numpy().view(np.uint32)
    for k in range(bu.nrows):
        c = bu.col[bu.row_ptr[k]:bu.row_ptr[k + 1]].astype(np.int64)
        bl = c >> 5
        runs = np.concatenate([[0], np.nonzero(bl[1:] != bl[:-1])[0] + 1])
        assert cnt2[k] == len(runs)
        got = pairs2[bu.row_ptr[k]:bu.row_ptr[k] + cnt2[k]]
        for t, r0 in enumerate(runs):
            r1 = runs[t + 1] if t + 1 < len(runs) else len(c)
            assert got[t, 0] == bl[r0]
            assert got[t, 1] == np.bitwise_or.reduce((np.uint64(1) << (c[r0:r1] % 32).astype(np.uint64))).astype(np.uint32)


@pytest.mark.parametrize("mean_len", [8, 40])
def test_compression_row_lengths(h, mean_len):
    """Matrices whose rows average a dozen or more entries: sorted rows of
    lengths around the four-column load steps and the 32-entry steps of the
    long-row kernel (empty, 1, 15, 16, 17, 31, 32, 33, 65, 128, and rows
    longer than 128 left to the warp-per-row kernel) with dense runs across
    block edges, against the canonical compression; the same rows permuted,
    against the runs of equal blocks in storage order; then a product
    through these descriptors."""
    rng = np.random.default_rng(mean_len)
    lens = [0, 1, 15, 16, 17, 31, 32, 33, 65, 128, 129, 300]
    nrow = 400
    row_len = np.array([lens[(i // 8) % len(lens)] if i % 8 == 0 else int(rng.integers(mean_len - 4, mean_len + 5))
                        for i in range(nrow)])
    ncols = 20000
    rows, cols = [], []
    for i, L in enumerate(row_len):
        if L == 0:
            continue
        dense = np.arange(L // 2) + 40 * (i % 7) + 3          # runs spanning block edges
        sparse = 3000 + rng.choice(ncols - 3000, size=L - L // 2, replace=False)
        c = np.unique(np.concatenate([dense, sparse]))
        rows += [i] * len(c)
        cols += c.tolist()
    key = np.array(rows, dtype=np.int64) * ncols + np.array(cols, dtype=np.int64)
    b = I.Csr(nrow, ncols, np.concatenate([[0], np.cumsum(np.bincount(key // ncols, minlength=nrow))]).astype(np.int64),
              (key % ncols).astype(np.int32), np.ones(len(key)))
    cnt, pairs = h.compress(to_dev(b))
    rp, blk, mask = oracle.compress_rows(b)
    cnt = cnt.cpu().numpy()
    pairs = pairs.cpu().numpy().view(np.uint32)
    assert np.array_equal(cnt, np.diff(rp))
    for k in range(b.nrows):
        got = pairs[b.row_ptr[k]:b.row_ptr[k] + cnt[k]]
        assert np.array_equal(got[:, 0], blk[rp[k]:rp[k + 1]].astype(np.uint32))
        assert np.array_equal(got[:, 1], mask[rp[k]:rp[k + 1]])
    order = np.lexsort((I.uniform01(np.arange(b.nnz, dtype=np.uint64), 23),
                        np.repeat(np.arange(nrow), np.diff(b.row_ptr))))
    bu = I.Csr(nrow, ncols, b.row_ptr, b.col[order], b.val)
    cnt2, pairs2 = h.compress(to_dev(bu))
    cnt2 = cnt2.cpu().numpy(); pairs2 = pairs2.cpu().numpy().view(np.uint32)
    for k in range(bu.nrows):
        c = bu.col[bu.row_ptr[k]:bu.row_ptr[k + 1]].astype(np.int64)
        if len(c) == 0:
            assert cnt2[k] == 0
            continue
        bl = c >> 5
        runs = np.concatenate([[0], np.nonzero(bl[1:] != bl[:-1])[0] + 1])
        assert cnt2[k] == len(runs)
        got = pairs2[bu.row_ptr[k]:bu.row_ptr[k] + cnt2[k]]
        for t, r0 in enumerate(runs):
            r1 = runs[t + 1] if t + 1 < len(runs) else len(c)
            assert got[t, 0] == bl[r0]
            assert got[t, 1] == np.bitwise_or.reduce((np.uint64(1) << (c[r0:r1] % 32).astype(np.uint64))).astype(np.uint32)
    # and the product through these descriptors
    a = I.random_csr(150, nrow, 0.03, 29, shuffle_cols=True)
    assert_matches(h.spgemm(to_dev(a), to_dev(bu)), oracle.spgemm(a, bu), "f64")
