"""Pins of the multigrid family generators (Section 4's Laplace3D, BigStar2D,
Brick3D and Elasticity operators with smoothed-aggregation prolongators)
against constructions written out independently here: operators by a loop
over grid points and stencil offsets, prolongators by dense matrix algebra
P = (I - omega D^-1 A) P_tent; plus the closed-form 27-point generators,
interior row counts, zero row sums of the operators and the partition of
unity of P away from the boundary.  Also the oracle's product on these
families against the dense product."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1804_00695_gb300 import inputs as I

FAMILIES = {"laplace3d_7pt": (3, 7, 1), "bigstar2d_13pt": (2, 13, 1), "brick3d_27pt": (3, 27, 1),
            "elasticity3d_81": (3, 81, 3)}


def stencil_by_loops(name, n):
    """Dense operator: for every grid point and every stencil offset inside
    the grid, the offset's weight (Kronecker the block for elasticity)."""
    base = "brick3d_27pt" if name == "elasticity3d_81" else name
    d, off, w = I._stencil_weights(base)
    N = n ** d
    a = np.zeros((N, N))
    for pt in itertools.product(range(n), repeat=d):
        i = sum(pt[k] * n ** k for k in range(d))
        for o, wo in zip(off, w):
            q = [pt[k] + o[k] for k in range(d)]
            if all(0 <= x < n for x in q):
                a[i, sum(q[k] * n ** k for k in range(d))] += wo
    return np.kron(a, I.ELASTICITY_BLOCK) if name == "elasticity3d_81" else a


def tentative(name, n):
    d, _, b = FAMILIES[name]
    N, nc = n ** d, (n + 2) // 3
    pt = np.zeros((N, nc ** d))
    for i in range(N):
        x = [(i // n ** k) % n for k in range(d)]
        pt[i, sum((x[k] // 3) * nc ** k for k in range(d))] = 1.0
    return np.kron(pt, np.eye(b))


@pytest.mark.parametrize("name", list(FAMILIES))
@pytest.mark.parametrize("n", [4, 7])
def test_against_dense_construction(name, n):
    a, p, r = I.family_problem(name, n)
    ad = stencil_by_loops(name, n)
    assert np.array_equal(a.to_dense(), ad)
    pd = (np.eye(len(ad)) - (2.0 / 3.0) * np.diag(1.0 / np.diag(ad)) @ ad) @ tentative(name, n)
    got = p.to_dense()
    assert np.all(np.abs(got - pd) <= 1e-15)
    # stored entries are the nonzeros of the exact P (dense rounding leaves
    # only residues below 1e-15 elsewhere)
    assert np.all(p.val != 0.0)
    assert np.all(np.abs(pd[got == 0.0]) < 1e-15)
    assert np.array_equal(r.to_dense(), got.T)
    for m in (a, p, r):   # columns ascending, no duplicates
        assert oracle.validate(m) == 0
        for i in range(m.nrows):
            c = m.col[m.row_ptr[i]:m.row_ptr[i + 1]]
            assert np.all(np.diff(c) > 0)


def test_brick_matches_closed_form():
    for n in (5, 9, 13):
        a = I.stencil_matrix("brick3d_27pt", n)
        b = I.laplace3d_27pt(n)
        assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
        assert np.array_equal(a.val, b.val)
        p = I.smoothed_prolongator("brick3d_27pt", n)
        q = I.galerkin_prolongator(n)
        assert np.array_equal(p.row_ptr, q.row_ptr) and np.array_equal(p.col, q.col)
        assert np.max(np.abs(p.val - q.val)) <= 2e-16


@pytest.mark.parametrize("name", list(FAMILIES))
def test_interior_rows_and_unity(name):
    d, per_row, b = FAMILIES[name]
    n = 11
    a, p, _ = I.family_problem(name, n)
    reach = 2 if name == "bigstar2d_13pt" else 1
    lens = np.diff(a.row_ptr)
    rows = np.arange(a.nrows)
    pts = rows // b
    inner = np.ones(a.nrows, dtype=bool)
    for k in range(d):
        x = (pts // n ** k) % n
        inner &= (x >= reach) & (x < n - reach)
    assert np.all(lens[inner] == per_row)
    assert lens.max() == per_row
    assert np.all(lens[~inner] < per_row)
    # zero row sums of the operator away from the boundary
    ones = np.ones(a.ncols)
    rs = np.add.reduceat(a.val * ones[a.col], a.row_ptr[:-1]) if a.nnz else np.zeros(a.nrows)
    assert np.all(np.abs(rs[inner]) < 1e-12)
    # P 1 = (I - omega D^-1 A) 1 = 1 where A 1 = 0
    pv = np.add.reduceat(p.val, p.row_ptr[:-1])
    if b == 1:
        assert np.all(np.abs(pv[inner] - 1.0) < 1e-14)
    else:   # block rows: P (1 per unknown) sums to 1 over the unknown's own column too
        pm = p.to_dense() @ np.kron(np.ones((p.ncols // b, 1)), np.eye(b))
        assert np.all(np.abs(pm[inner] - np.eye(b)[rows[inner] % b]) < 1e-14)


@pytest.mark.parametrize("name", list(FAMILIES))
def test_oracle_products_dense(name):
    """R*A, A*P and R*(A*P) by the oracle against dense products."""
    a, p, r = I.family_problem(name, 6)
    ad, pd, rd = a.to_dense(), p.to_dense(), r.to_dense()
    for x, y, ref in ((r, a, rd @ ad), (a, p, ad @ pd)):
        c = oracle.spgemm(x, y)
        cd = I.Csr(c.nrows, c.ncols, c.row_ptr, c.col, c.val).to_dense()
        assert np.all(np.abs(cd - ref) <= 1e-12 * (np.abs(x.to_dense()) @ np.abs(y.to_dense())) + 0.0)
    ap = oracle.spgemm(a, p)
    rap = oracle.spgemm(r, I.Csr(ap.nrows, ap.ncols, ap.row_ptr, ap.col, ap.val))
    cd = I.Csr(rap.nrows, rap.ncols, rap.row_ptr, rap.col, rap.val).to_dense()
    assert np.allclose(cd, rd @ ad @ pd, rtol=0, atol=1e-11)
    # the coarse operator of a symmetric A is symmetric
    assert np.allclose(cd, cd.T, rtol=0, atol=1e-11)


@pytest.mark.parametrize("delta", [1, 4, 16, 64, 256])
def test_random_rhs_rows(delta):
    """Right-hand sides of the density experiment (Table 2): every row holds
    exactly min(delta, ncols) distinct columns, ascending and in range; the
    columns are spread evenly over the matrix and the values are N(0,1)."""
    nrows, ncols = 700, 3000
    m = I.random_rhs(nrows, ncols, delta, seed=11)
    assert (m.nrows, m.ncols) == (nrows, ncols)
    lens = np.diff(m.row_ptr)
    assert np.all(lens == min(delta, ncols))
    for i in range(0, nrows, 37):
        c = m.col[m.row_ptr[i]:m.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0) and c.min() >= 0 and c.max() < ncols
    # columns: each tenth of the range receives about a tenth of the entries
    hist = np.bincount(m.col.astype(np.int64) * 10 // ncols, minlength=10) / m.nnz
    assert np.all(np.abs(hist - 0.1) < 0.1 * (0.5 if m.nnz >= 10000 else 1.0))
    if m.nnz >= 10000:
        assert abs(m.val.mean()) < 0.05 and abs(m.val.std() - 1.0) < 0.05


def test_random_rhs_more_than_ncols():
    """delta above the number of columns gives full rows."""
    m = I.random_rhs(40, 30, 64, seed=3)
    assert np.all(np.diff(m.row_ptr) == 30)
    for i in range(m.nrows):
        assert np.array_equal(m.col[m.row_ptr[i]:m.row_ptr[i + 1]], np.arange(30))
