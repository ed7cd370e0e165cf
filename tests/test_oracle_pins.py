"""Pins of the CPU oracle against facts fixed by mathematics, not by itself:
dense brute force, identities, explicit set unions, closed-form stencil
products (Kronecker factorisation) and graph invariants."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1804_00695_gb300 import inputs as I


def dense_pattern(m):
    d = np.zeros((m.nrows, m.ncols), dtype=bool)
    rows = np.repeat(np.arange(m.nrows), np.diff(m.row_ptr))
    d[rows, m.col] = True
    return d


def csr_to_dense(rp, col, val, nrows, ncols):
    d = np.zeros((nrows, ncols))
    rows = np.repeat(np.arange(nrows), np.diff(rp))
    d[rows, col] = val
    return d


@pytest.mark.parametrize("seed,shape,dens,shuffle", [
    (1, (7, 9, 5), 0.3, False), (2, (31, 17, 40), 0.2, True), (3, (48, 48, 48), 0.1, True),
    (4, (1, 30, 1), 0.9, False), (5, (20, 1, 33), 0.5, True), (6, (33, 33, 33), 0.0, False)])
def test_brute_force_dense(seed, shape, dens, shuffle):
    m, k, n = shape
    a = I.random_csr(m, k, dens, seed, shuffle_cols=shuffle)
    b = I.random_csr(k, n, dens, seed + 100, shuffle_cols=shuffle)
    c = oracle.spgemm(a, b)
    # Pattern: boolean product of stored masks (structural, no cancellation).
    pat = (dense_pattern(a).astype(np.int64) @ dense_pattern(b).astype(np.int64)) > 0
    got = csr_to_dense(c.row_ptr, c.col, np.ones(c.nnz), m, n) > 0
    assert np.array_equal(pat, got)
    assert c.nnz == pat.sum()
    for i in range(m):  # ascending columns
        assert np.all(np.diff(c.col[c.row_ptr[i]:c.row_ptr[i + 1]]) > 0)
    ref = a.to_dense() @ b.to_dense()
    absref = np.abs(a.to_dense()) @ np.abs(b.to_dense())
    cv = csr_to_dense(c.row_ptr, c.col, c.val, m, n)
    cb = csr_to_dense(c.row_ptr, c.col, c.bound, m, n)
    assert np.all(np.abs(cv - ref) <= 1e-13 * absref + 1e-300)
    assert np.allclose(cb, absref, rtol=1e-13, atol=0)
    assert c.mults.sum() == sum(np.diff(b.row_ptr)[a.col].tolist())


def test_identity_and_permutation():
    a = I.random_csr(40, 40, 0.15, 11, shuffle_cols=True)
    eye = I.Csr(40, 40, np.arange(41, dtype=np.int64), np.arange(40, dtype=np.int32), np.ones(40))
    for c in (oracle.spgemm(a, eye), oracle.spgemm(eye, a)):
        for i in range(40):
            s = slice(a.row_ptr[i], a.row_ptr[i + 1])
            order = np.argsort(a.col[s])
            assert np.array_equal(c.col[c.row_ptr[i]:c.row_ptr[i + 1]], a.col[s][order])
            assert np.array_equal(c.val[c.row_ptr[i]:c.row_ptr[i + 1]], a.val[s][order])
    perm = np.array(I.splitmix64(np.arange(40), 5) % np.uint64(1 << 30)).argsort()
    pm = I.Csr(40, 40, np.arange(41, dtype=np.int64), perm.astype(np.int32), np.ones(40))
    c = oracle.spgemm(pm, a)  # row i of P*A = row perm[i] of A
    for i in range(40):
        r = perm[i]
        s = slice(a.row_ptr[r], a.row_ptr[r + 1])
        order = np.argsort(a.col[s])
        assert np.array_equal(c.col[c.row_ptr[i]:c.row_ptr[i + 1]], a.col[s][order])
        assert np.array_equal(c.val[c.row_ptr[i]:c.row_ptr[i + 1]], a.val[s][order])


def test_counts_from_set_unions():
    a = I.random_csr(300, 500, 0.02, 21, shuffle_cols=True)
    b = I.random_csr(500, 700, 0.03, 22, shuffle_cols=True)
    cnt, mults = oracle.symbolic(a, b)
    for i in range(a.nrows):
        s = set()
        m = 0
        for k in a.col[a.row_ptr[i]:a.row_ptr[i + 1]]:
            cols = b.col[b.row_ptr[k]:b.row_ptr[k + 1]]
            s.update(cols.tolist())
            m += len(cols)
        assert cnt[i] == len(s)
        assert mults[i] == m
    # row range call agrees with the full call
    c_full = oracle.spgemm(a, b)
    c_part = oracle.spgemm(a, b, 100, 200)
    p0 = c_full.row_ptr[100]
    assert np.array_equal(c_part.col, c_full.col[p0:c_full.row_ptr[200]])
    assert np.array_equal(c_part.val, c_full.val[p0:c_full.row_ptr[200]])


def test_laplace2d_squared_closed_form():
    """(4I - N)^2 = 16I - 8N + N^2 on the 64x64 grid: diagonal 16 + degree,
    grid neighbours -8, diagonal neighbours +2, distance-2 straight +1."""
    n = 64
    a = I.laplace2d_5pt(n)
    c = oracle.spgemm(a, a)
    assert c.nnz == 51972 and c.mults.sum() == 100104
    for i in range(n * n):
        x, y = i % n, i // n
        deg = (x > 0) + (x < n - 1) + (y > 0) + (y < n - 1)
        exp = {}
        for dx in range(-2, 3):
            for dy in range(-2, 3):
                xx, yy = x + dx, y + dy
                if not (0 <= xx < n and 0 <= yy < n):
                    continue
                d = abs(dx) + abs(dy)
                if d == 0:
                    exp[xx + n * yy] = 16.0 + deg
                elif d == 1:
                    exp[xx + n * yy] = -8.0
                elif d == 2 and dx != 0 and dy != 0:
                    exp[xx + n * yy] = 2.0
                elif d == 2:
                    exp[xx + n * yy] = 1.0
        cols = c.col[c.row_ptr[i]:c.row_ptr[i + 1]]
        vals = c.val[c.row_ptr[i]:c.row_ptr[i + 1]]
        assert cols.tolist() == sorted(exp)
        assert vals.tolist() == [exp[j] for j in sorted(exp)]


def _t1(n):
    t = np.zeros((n, n))
    for x in range(n):
        for y in range(max(0, x - 1), min(n, x + 2)):
            t[x, y] = 1
    return t


def _kron3(m):
    return np.kron(np.kron(m, m), m)


@pytest.mark.parametrize("n", [5, 7, 8])
def test_laplace3d_squared_closed_form(n):
    """A = 27I - K with K = T(x)T(x)T, so A^2 = 729I - 54K + (T^2)(x)(T^2)(x)(T^2);
    nnz(A^2) = (5n-6)^3 and mults = (sum of squared 1D row lengths)^3."""
    a = I.laplace3d_27pt(n)
    assert a.nnz == (3 * n - 2) ** 3
    c = oracle.spgemm(a, a)
    t = _t1(n)
    exp = 729 * np.eye(n ** 3) - 54 * _kron3(t) + _kron3(t @ t)
    got = csr_to_dense(c.row_ptr, c.col, c.val, n ** 3, n ** 3)
    assert np.array_equal(got, exp)  # integers: exact
    assert c.nnz == (5 * n - 6) ** 3
    rl = t.sum(1)
    assert c.mults.sum() == int((rl ** 2).sum()) ** 3


def _agg1d(n):
    nc = (n + 2) // 3
    p = np.zeros((n, nc))
    p[np.arange(n), np.arange(n) // 3] = 1
    return p


@pytest.mark.parametrize("n", [6, 10, 11])
def test_galerkin_prolongator_definition(n):
    """The generator's P equals (I - (2/3) D^-1 A) P_tent computed by the oracle."""
    a = I.laplace3d_27pt(n)
    pt = I.tentative_prolongator(n)
    # S = I - (2/3) D^-1 A with D = 26 I: S = A * (-(2/3)/26) + I on A's pattern.
    rows = np.repeat(np.arange(a.nrows), np.diff(a.row_ptr))
    sval = -(2.0 / 3.0) / 26.0 * a.val + (rows == a.col)
    s = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, sval)
    ref = oracle.spgemm(s, pt)
    p = I.galerkin_prolongator(n)
    assert np.array_equal(ref.row_ptr, p.row_ptr) and np.array_equal(ref.col, p.col)
    assert np.allclose(ref.val, p.val, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("n", [6, 10, 11])
def test_galerkin_products_closed_form(n):
    """AP = (108/13) P_t + (5/13) Q - (1/39) Q2 and RAP = P^T AP, with
    Q = (Tp)^(x)3, Q2 = (T^2 p)^(x)3 built from 1D factors."""
    a, p, r = I.galerkin_problem(n)
    ap = oracle.spgemm(a, p)
    t = _t1(n)
    p1 = _agg1d(n)
    tp, t2p = t @ p1, t @ t @ p1
    pt, q, q2 = _kron3(p1), _kron3(tp), _kron3(t2p)
    ap_exp = (108 / 13) * pt + (5 / 13) * q - (1 / 39) * q2
    got = csr_to_dense(ap.row_ptr, ap.col, ap.val, a.nrows, p.ncols)
    assert np.allclose(got, ap_exp, rtol=0, atol=1e-13 * 100)
    assert ap.nnz == (np.count_nonzero(t2p)) ** 3
    apm = I.Csr(a.nrows, p.ncols, ap.row_ptr, ap.col, ap.val)
    rap = oracle.spgemm(r, apm)
    terms = [((4 / 13) * (108 / 13), p1, p1), ((4 / 13) * (5 / 13), p1, tp), (-(4 / 13) / 39, p1, t2p),
             ((108 / 13) / 39, tp, p1), ((5 / 13) / 39, tp, tp), (-1 / 39 / 39, tp, t2p)]
    rap_exp = sum(cf * _kron3(x.T @ y) for cf, x, y in terms)
    got = csr_to_dense(rap.row_ptr, rap.col, rap.val, r.nrows, p.ncols)
    assert np.allclose(got, rap_exp, rtol=0, atol=1e-11)
    pat = _kron3((tp.T @ t2p) > 0) > 0
    assert np.array_equal(csr_to_dense(rap.row_ptr, rap.col, np.ones(rap.nnz), r.nrows, p.ncols) > 0, pat)


def test_galerkin_128_sizes():
    """Pattern sizes of the 128^3 problem from the 1D factors alone."""
    n = 128
    t = _t1(n)
    p1 = _agg1d(n)
    tp, t2p = t @ p1, t @ t @ p1
    assert np.count_nonzero(tp) ** 3 == 9528128
    assert np.count_nonzero(t2p) ** 3 == 25934336
    assert np.count_nonzero(tp.T @ t2p) ** 3 == 2048383
    # mults of A*P: sum over rows of A of sum over its columns k of nnz(P_k)
    assert int((t @ (tp != 0).sum(1)).sum()) ** 3 == 254840104
    rl_ap = (t2p != 0).sum(1)          # nnz of AP rows per 1D index
    assert int(((tp != 0).T @ rl_ap).sum()) ** 3 == 99897344


def test_rmat_square_invariants():
    g = I.rmat_symmetric(10, 16, seed=1)
    assert oracle.validate(g) == 0
    d = g.to_dense()
    assert np.array_equal(d, d.T) and np.all(np.diag(d) == 0)
    c = oracle.spgemm(g, g)
    deg = np.diff(g.row_ptr)
    cd = csr_to_dense(c.row_ptr, c.col, c.val, g.nrows, g.ncols)
    assert np.array_equal(np.diag(cd), deg.astype(float))
    assert cd.sum() == float((deg ** 2).sum())
    assert np.array_equal(cd, cd.T)
    assert np.array_equal(cd, d @ d)


def test_backward_definition():
    a = I.random_csr(23, 31, 0.2, 41, shuffle_cols=True)
    b = I.random_csr(31, 19, 0.25, 42, shuffle_cols=True)
    c = oracle.spgemm(a, b)
    dc = I.uniform01(np.arange(c.nnz, dtype=np.uint64), 43) * 2 - 1
    da, db = oracle.backward(a, b, c.row_ptr, c.col, dc)
    dcd = csr_to_dense(c.row_ptr, c.col, dc, a.nrows, b.ncols)
    ad, bd = a.to_dense(), b.to_dense()
    gA = dcd @ bd.T
    gB = ad.T @ dcd
    ra = np.repeat(np.arange(a.nrows), np.diff(a.row_ptr))
    rb = np.repeat(np.arange(b.nrows), np.diff(b.row_ptr))
    assert np.allclose(da, gA[ra, a.col], rtol=1e-13, atol=1e-14)
    assert np.allclose(db, gB[rb, b.col], rtol=1e-13, atol=1e-14)
    # Euler identity for the bilinear form: <dA,A> = <dC,C> = <dB,B>
    lc = float(dc @ c.val)
    assert np.isclose(da @ a.val, lc, rtol=1e-12) and np.isclose(db @ b.val, lc, rtol=1e-12)
    # central differences (exact for a bilinear map up to rounding)
    h = 1e-3
    for p in (0, a.nnz // 2, a.nnz - 1):
        ap_, am_ = a.val.copy(), a.val.copy()
        ap_[p] += h; am_[p] -= h
        lp = float(dc @ oracle.spgemm(I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, ap_), b).val)
        lm = float(dc @ oracle.spgemm(I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, am_), b).val)
        assert np.isclose((lp - lm) / (2 * h), da[p], rtol=1e-9, atol=1e-11)


def test_fma_range_composes_to_product():
    """Section 3.2.2: C2 = A2*B2 + C1 over consecutive B row ranges gives A*B."""
    a = I.random_csr(60, 80, 0.08, 51, shuffle_cols=True)
    b = I.random_csr(80, 70, 0.1, 52, shuffle_cols=True)
    full = oracle.spgemm(a, b)
    cur = None
    for lo, hi in ((0, 13), (13, 14), (14, 50), (50, 80)):
        cur = oracle.fma_range(a, b, lo, hi, cur)
    rp, col, val = cur
    assert np.array_equal(rp, full.row_ptr) and np.array_equal(col, full.col)
    assert np.all(np.abs(val - full.val) <= 1e-13 * full.bound)


def test_compress_rows_decodes():
    m = I.random_csr(50, 300, 0.1, 61, shuffle_cols=True)
    rp, blk, mask = oracle.compress_rows(m)
    for i in range(m.nrows):
        s = set(m.col[m.row_ptr[i]:m.row_ptr[i + 1]].tolist())
        dec = set()
        bl = blk[rp[i]:rp[i + 1]]
        assert np.all(np.diff(bl) > 0)
        for kb, mk in zip(bl, mask[rp[i]:rp[i + 1]]):
            assert mk != 0
            dec.update(32 * int(kb) + t for t in range(32) if (int(mk) >> t) & 1)
        assert dec == s


def test_validate_errors():
    good = I.random_csr(10, 10, 0.3, 71)
    assert oracle.validate(good) == 0
    bad = I.Csr(2, 5, np.array([0, 2, 3]), np.array([1, 1, 4], dtype=np.int32), np.ones(3))
    assert oracle.validate(bad) == 3
    oor = I.Csr(2, 5, np.array([0, 1, 2]), np.array([1, 5], dtype=np.int32), np.ones(2))
    assert oracle.validate(oor) == 2


def _row_flops_loops(a, b):
    """Multiplications of each row of A*B counted with explicit loops: for
    every stored a_ik, one per stored entry of row k of B (Section 3.1)."""
    out = []
    for i in range(a.nrows):
        f = 0
        for p in range(int(a.row_ptr[i]), int(a.row_ptr[i + 1])):
            k = int(a.col[p])
            f += int(b.row_ptr[k + 1]) - int(b.row_ptr[k])
        out.append(f)
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("seed,shape,dens", [(81, (40, 60, 30), 0.1), (82, (200, 150, 90), 0.05),
                                             (83, (1, 50, 20), 0.8), (84, (64, 1, 5), 0.5)])
def test_row_flops_per_row(seed, shape, dens):
    """oracle.row_flops row by row against the loop count and against the
    multiplications the C oracle's symbolic pass counts, on unsorted rows
    (rows of A with no entries and rows of B with none included)."""
    m, k, n = shape
    a = I.random_csr(m, k, dens, seed, shuffle_cols=True)
    b = I.random_csr(k, n, dens, seed + 7, shuffle_cols=True)
    got = oracle.row_flops(a, b)
    assert np.array_equal(got, _row_flops_loops(a, b))
    _, mults = oracle.symbolic(a, b)
    assert np.array_equal(got, mults)


@pytest.mark.parametrize("n", [6, 11])
def test_row_flops_galerkin_closed_form(n):
    """Per-row multiplications of A*P and R*(AP) from 1D factors: the patterns
    are Kronecker cubes, so row x + n*y + n^2*z of A*P does f(x) f(y) f(z)
    multiplications with f = T times the row lengths of Tp, and row J of
    R*(AP) does g(j1) g(j2) g(j3) with g = pattern(Tp)^T times the row
    lengths of T^2 p (at n = 128 the totals are 634^3 and 464^3, the sizes
    test_galerkin_128_sizes checks)."""
    a, p, r = I.galerkin_problem(n)
    t = _t1(n)
    p1 = _agg1d(n)
    tp, t2p = t @ p1, t @ t @ p1
    f1 = (t != 0).astype(np.int64) @ (tp != 0).sum(1).astype(np.int64)
    np.testing.assert_array_equal(oracle.row_flops(a, p), np.kron(np.kron(f1, f1), f1))
    ap = oracle.spgemm(a, p)
    apm = I.Csr(a.nrows, p.ncols, ap.row_ptr, ap.col, ap.val)
    g1 = (tp != 0).T.astype(np.int64) @ (t2p != 0).sum(1).astype(np.int64)
    np.testing.assert_array_equal(oracle.row_flops(r, apm), np.kron(np.kron(g1, g1), g1))
    assert int(f1.sum()) ** 3 == int(oracle.row_flops(a, p).sum())
