"""Seeded synthetic inputs for the SpGEMM workloads.

This module only builds input matrices (CSR with int64 row pointers and int32
column indices).  It contains none of the multiplication's arithmetic and
serves the CUDA library, the CPU oracle and the benchmark alike.

Workloads (stand-ins for the paper's multigrid and graph matrices, Section
3.2 and Section 4.1.2 of Deveci et al.):

* ``laplace2d_5pt(n)``: 2D 5-point Laplacian on an n x n grid, lexicographic
  ordering i = x + n*y, diagonal 4, neighbours -1.
* ``laplace3d_27pt(n)``: 3D 27-point Laplacian on an n^3 grid, lexicographic
  ordering i = x + n*y + n^2*z, diagonal 26, every neighbour -1, boundary rows
  truncated.
* ``galerkin_prolongator(n)``: smoothed-aggregation prolongator
  P = (I - (2/3) D^-1 A) P_tent for the 27-point A above, with aggregates
  agg(x) = floor(x/3) in each dimension and P_tent piecewise constant (1.0).
  Because A = 27 I - T(x)T(x)T with T the tridiagonal all-ones matrix, and
  D = 26 I, P = (4/13) P_tent + (1/39) (Tp)(x)(Tp)(x)(Tp), so every entry is
  written directly from one-dimensional factors.  The restriction is R = P^T.
* ``stencil_matrix(name, n)``, ``smoothed_prolongator(name, n)``,
  ``family_problem(name, n)``: the multigrid families of Section 4 - 7-point
  3D Laplacian, 13-point 2D biharmonic star ("BigStar2D"), 27-point 3D
  brick, and 3D elasticity (27-point stencil Kronecker a 3x3 SPD block, 81
  entries per row) - with smoothed-aggregation prolongators (aggregates of 3
  points per dimension, omega 2/3) written per stencil offset.
* ``rmat_symmetric(scale, edge_factor, abcd, seed)``: R-MAT graph with a
  counter-based generator (SplitMix64 finaliser over a counter), self-loops
  dropped, symmetrised, duplicates removed, values 1.0 (float32).
* ``random_batch(...)``: square n_i x n_i matrices with n_i log-uniform in
  [lo, hi], each row holding a uniform 4..32 distinct random columns, N(0,1)
  float32 values.

The counter-based generator: u64 word number c of stream (seed, s) is
SplitMix64's output function applied to seed*0xD1B54A32D192ED03 +
s*0xC2B2AE3D27D4EB4F + (c+1)*0x9E3779B97F4A7C15 (mod 2^64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_U64 = np.uint64
_M = (1 << 64) - 1


@dataclass
class Csr:
    """CSR matrix held in host memory: int64 row_ptr, int32 col, values."""
    nrows: int
    ncols: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def astype(self, dtype) -> "Csr":
        return Csr(self.nrows, self.ncols, self.row_ptr, self.col, self.val.astype(dtype))

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.nrows, self.ncols), dtype=np.float64)
        rows = np.repeat(np.arange(self.nrows), np.diff(self.row_ptr))
        np.add.at(d, (rows, self.col.astype(np.int64)), self.val.astype(np.float64))
        return d


def splitmix64(counter: np.ndarray, seed: int, stream: int = 0) -> np.ndarray:
    """SplitMix64 finaliser applied to a counter (vectorised, uint64 wrap)."""
    c = np.asarray(counter, dtype=_U64)
    base = (seed * 0xD1B54A32D192ED03 + stream * 0xC2B2AE3D27D4EB4F) & _M
    with np.errstate(over="ignore"):
        z = _U64(base) + (c + _U64(1)) * _U64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> _U64(30))) * _U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> _U64(27))) * _U64(0x94D049BB133111EB)
        z = z ^ (z >> _U64(31))
    return z


def uniform01(counter: np.ndarray, seed: int, stream: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the counter-based words."""
    return (splitmix64(counter, seed, stream) >> _U64(11)).astype(np.float64) * (1.0 / (1 << 53))


def _csr_from_1d(rows: list[list[int]], vals: list[list[float]], ncols: int) -> Csr:
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([c for r in rows for c in r], dtype=np.int32)
    val = np.array([v for r in vals for v in r], dtype=np.float64)
    return Csr(len(rows), ncols, rp, col, val)


def kron_lex(slow: Csr, fast: Csr, vals: tuple[np.ndarray, ...] | None = None,
             fvals: tuple[np.ndarray, ...] | None = None):
    """Kronecker product with lexicographic ordering: row = f + nf*s,
    col = cf + mf*cs, value = vs*vf.  Columns stay ascending when both
    factors have ascending columns.  Optional extra value arrays are carried
    through the same pattern (products taken entry by entry)."""
    ns, nf = slow.nrows, fast.nrows
    lens_s = np.diff(slow.row_ptr)
    lens_f = np.diff(fast.row_ptr)
    # Row (s, f) has lens_s[s]*lens_f[f] entries.
    row_len = (lens_s[:, None] * lens_f[None, :]).reshape(-1)
    rp = np.zeros(ns * nf + 1, dtype=np.int64)
    np.cumsum(row_len, out=rp[1:])
    nnz = int(rp[-1])
    # For every output row, enumerate slow entries (outer) x fast entries (inner).
    s_idx = np.repeat(np.arange(ns), nf)
    f_idx = np.tile(np.arange(nf), ns)
    out_rows = np.repeat(np.arange(ns * nf), row_len)
    pos_in_row = np.arange(nnz, dtype=np.int64) - rp[out_rows]
    lf = lens_f[f_idx][out_rows]
    ps = slow.row_ptr[s_idx[out_rows]] + pos_in_row // lf
    pf = fast.row_ptr[f_idx[out_rows]] + pos_in_row % lf
    col = (fast.col[pf].astype(np.int64) + fast.ncols * slow.col[ps].astype(np.int64))
    val = slow.val[ps] * fast.val[pf]
    extra = []
    if vals is not None:
        for vs, vf in zip(vals, fvals):
            extra.append(vs[ps] * vf[pf])
    m = Csr(ns * nf, slow.ncols * fast.ncols, rp, col.astype(np.int32), val)
    return (m, extra) if vals is not None else m


def tridiag_ones(n: int) -> Csr:
    rows = [[j for j in (i - 1, i, i + 1) if 0 <= j < n] for i in range(n)]
    return _csr_from_1d(rows, [[1.0] * len(r) for r in rows], n)


def laplace2d_5pt(n: int) -> Csr:
    """2D 5-point Laplacian, i = x + n*y, diagonal 4, neighbours -1."""
    rows, vals = [], []
    for y in range(n):
        for x in range(n):
            r, v = [], []
            for dx, dy in ((0, -1), (-1, 0), (0, 0), (1, 0), (0, 1)):
                xx, yy = x + dx, y + dy
                if 0 <= xx < n and 0 <= yy < n:
                    r.append(xx + n * yy)
                    v.append(4.0 if (dx, dy) == (0, 0) else -1.0)
            rows.append(r); vals.append(v)
    return _csr_from_1d(rows, vals, n * n)


def laplace3d_27pt(n: int) -> Csr:
    """3D 27-point Laplacian A = 27 I - T(x)T(x)T on an n^3 grid, built as a
    Kronecker product of 1D tridiagonal all-ones patterns."""
    t = tridiag_ones(n)
    k = kron_lex(kron_lex(t, t), t)
    diag = np.repeat(np.arange(k.nrows, dtype=np.int64), np.diff(k.row_ptr)) == k.col
    val = np.where(diag, 26.0, -1.0)
    return Csr(k.nrows, k.ncols, k.row_ptr, k.col, val)


def _agg_1d(n: int):
    """1D factors of the prolongator: Tp pattern with (Tp) counts and the
    indicator of the own aggregate, nc = ceil(n/3) aggregates."""
    nc = (n + 2) // 3
    rows, cnt, ind = [], [], []
    for x in range(n):
        c = {}
        for xx in (x - 1, x, x + 1):
            if 0 <= xx < n:
                c[xx // 3] = c.get(xx // 3, 0) + 1
        keys = sorted(c)
        rows.append(keys)
        cnt.append([float(c[k]) for k in keys])
        ind.append([1.0 if k == x // 3 else 0.0 for k in keys])
    tp = _csr_from_1d(rows, cnt, nc)
    ind_arr = np.array([v for r in ind for v in r], dtype=np.float64)
    return tp, ind_arr


def galerkin_prolongator(n: int) -> Csr:
    """P = (I - (2/3) D^-1 A) P_tent for the 27-point A on an n^3 grid."""
    tp, ind = _agg_1d(n)
    two, ex = kron_lex(tp, tp, (ind,), (ind,))
    three, ex3 = kron_lex(two, tp, (ex[0],), (ind,))
    # three.val = product of Tp counts; ex3[0] = product of own-aggregate indicators.
    val = (4.0 / 13.0) * ex3[0] + (1.0 / 39.0) * three.val
    return Csr(three.nrows, three.ncols, three.row_ptr, three.col, val)


def tentative_prolongator(n: int) -> Csr:
    """P_tent: fine point (x,y,z) -> aggregate (x//3, y//3, z//3), value 1."""
    nc = (n + 2) // 3
    x = np.arange(n ** 3, dtype=np.int64)
    cx, cy, cz = (x % n) // 3, ((x // n) % n) // 3, (x // (n * n)) // 3
    col = (cx + nc * cy + nc * nc * cz).astype(np.int32)
    rp = np.arange(n ** 3 + 1, dtype=np.int64)
    return Csr(n ** 3, nc ** 3, rp, col, np.ones(n ** 3))


def transpose(m: Csr) -> Csr:
    """Structural transpose (stable counting sort by column)."""
    rows = np.repeat(np.arange(m.nrows, dtype=np.int64), np.diff(m.row_ptr))
    order = np.argsort(m.col, kind="stable")
    cnt = np.bincount(m.col, minlength=m.ncols).astype(np.int64)
    rp = np.zeros(m.ncols + 1, dtype=np.int64)
    np.cumsum(cnt, out=rp[1:])
    return Csr(m.ncols, m.nrows, rp, rows[order].astype(np.int32), m.val[order])


def galerkin_problem(n: int):
    """(A, P, R) of the Galerkin triple product R*(A*P) on an n^3 grid."""
    a = laplace3d_27pt(n)
    p = galerkin_prolongator(n)
    return a, p, transpose(p)


# ---------------------------------------------------------------- multigrid families
# Stencil operators on a lexicographic grid (i = x0 + n0*(x1 + n1*x2), x0
# fastest), boundary rows truncated, and their smoothed-aggregation
# prolongators P = (I - omega D^-1 A) P_tent with aggregates of 3 points per
# dimension (agg(x) = x // 3 in each dimension, coarse points ordered the same
# way).  Block operators (several unknowns per grid point) are the scalar
# stencil Kronecker a small dense block K, unknown fastest; their P_tent is
# the scalar one Kronecker the identity of K's order.

def _offsets(d: int, reach: int):
    """All offsets of a d-dimensional box of half-width reach, as a (k, d) array."""
    r = np.arange(-reach, reach + 1)
    g = np.stack(np.meshgrid(*([r] * d), indexing="ij"), axis=-1).reshape(-1, d)
    return g[:, ::-1].copy()   # column 0 is x0


STENCILS = {
    # name: (dimension, offsets, weights); weights of the 7-point and 27-point
    # Laplacians (diagonal = number of neighbours, neighbours -1) and of the
    # 13-point biharmonic star (20 at the centre, -8 at the 4 nearest, 2 at the
    # 4 diagonal, 1 at the 4 second-nearest points)
    "laplace3d_7pt": (3, np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]),
                      np.array([6.0, -1, -1, -1, -1, -1, -1])),
    "bigstar2d_13pt": (2, np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1], [1, 1], [1, -1], [-1, 1], [-1, -1],
                                    [2, 0], [-2, 0], [0, 2], [0, -2]]),
                       np.array([20.0, -8, -8, -8, -8, 2, 2, 2, 2, 1, 1, 1, 1])),
    "brick3d_27pt": (3, _offsets(3, 1), None),
}
# 3 unknowns per point (displacements), coupled by an SPD block
ELASTICITY_BLOCK = np.array([[3.0, 1.0, 1.0], [1.0, 3.0, 1.0], [1.0, 1.0, 3.0]])


def _stencil_weights(name: str):
    d, off, w = STENCILS[name]
    if w is None:   # 27-point: 26 at the centre, -1 elsewhere
        w = np.where(np.all(off == 0, axis=1), 26.0, -1.0)
    return d, off, w


def _stencil_block(dims, off, r0: int, r1: int):
    """Offsets sorted by linear displacement (so that columns ascend within a
    row), their displacements, the grid coordinates of rows [r0, r1) and the
    (rows x offsets) mask of in-grid neighbours."""
    dims = np.asarray(dims, dtype=np.int64)
    stride = np.concatenate([[1], np.cumprod(dims)[:-1]])
    lin = off @ stride
    order = np.argsort(lin, kind="stable")
    rows = np.arange(r0, r1, dtype=np.int64)
    x = [(rows // stride[k]) % dims[k] for k in range(len(dims))]
    ok = np.ones((r1 - r0, len(off)), dtype=bool)
    for k in range(len(dims)):
        xx = x[k][:, None] + off[order][None, :, k]
        ok &= (xx >= 0) & (xx < dims[k])
    return order, lin[order], rows, x, ok


def _grid_csr(n, rows, cols, vals, ncols, r0=0):
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows - r0, minlength=n), out=rp[1:])
    return Csr(n, ncols, rp, cols.astype(np.int32), vals)


def _block_kron(m: Csr, block: np.ndarray, zero_drop: bool = False, extra=None):
    """m Kronecker a dense block (unknown fastest); with extra = (m2_val,
    block2) the result's values are m.val*block + m2_val*block2 on the same
    pattern; zero_drop removes entries that are exactly 0."""
    b = block.shape[0]
    bc = Csr(b, b, np.arange(0, b * b + 1, b, dtype=np.int64), np.tile(np.arange(b, dtype=np.int32), b),
             block.reshape(-1).astype(np.float64))
    if extra is None:
        out = kron_lex(m, bc)
    else:
        out, ex = kron_lex(m, bc, (extra[0],), (extra[1].reshape(-1).astype(np.float64),))
        out = Csr(out.nrows, out.ncols, out.row_ptr, out.col, out.val + ex[0])
    if zero_drop:
        keep = out.val != 0.0
        rows = np.repeat(np.arange(out.nrows, dtype=np.int64), np.diff(out.row_ptr))[keep]
        out = _grid_csr(out.nrows, rows, out.col[keep], out.val[keep], out.ncols)
    return out


_ROW_BLOCK = 1 << 20   # rows generated at a time (bounds the temporaries)


def stencil_matrix(name: str, n: int) -> Csr:
    """Operator of a family on an n^d grid: "laplace3d_7pt", "bigstar2d_13pt",
    "brick3d_27pt" or "elasticity3d_81" (the 27-point stencil Kronecker
    ELASTICITY_BLOCK: 81 entries per interior row)."""
    base = "brick3d_27pt" if name == "elasticity3d_81" else name
    d, off, w = _stencil_weights(base)
    dims, N = [n] * d, n ** d
    lens, cols, vals = [], [], []
    for r0 in range(0, N, _ROW_BLOCK):
        r1 = min(N, r0 + _ROW_BLOCK)
        order, lin, rows, _, ok = _stencil_block(dims, off, r0, r1)
        lens.append(ok.sum(axis=1))
        cols.append((rows[:, None] + lin[None, :])[ok].astype(np.int32))
        vals.append(np.broadcast_to(w[order][None, :], ok.shape)[ok])
    rp = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.concatenate(lens), out=rp[1:])
    m = Csr(N, N, rp, np.concatenate(cols), np.concatenate(vals))
    return _block_kron(m, ELASTICITY_BLOCK) if name == "elasticity3d_81" else m


def smoothed_prolongator(name: str, n: int, omega: float = 2.0 / 3.0) -> Csr:
    """P = (I - omega D^-1 A) P_tent of a family (aggregates of 3 points per
    dimension), written per stencil offset: row i takes, for every in-grid
    offset o, [o = 0] - omega w_o / d at column agg(i + o) (d the diagonal),
    duplicates of a column summed and exact zeros dropped.  For the block
    family: P_tent Kronecker I - (omega / d) (A_scalar P_tent) Kronecker K
    with d = 26 * K's diagonal."""
    base = "brick3d_27pt" if name == "elasticity3d_81" else name
    dd, off, w = _stencil_weights(base)
    dims = [n] * dd
    nc = (n + 2) // 3
    N, NC = n ** dd, nc ** dd
    diag = float(w[np.all(off == 0, axis=1)][0])
    block = name == "elasticity3d_81"
    scale = omega / (diag * ELASTICITY_BLOCK[0, 0]) if block else omega / diag
    # the aggregates a row reaches lie within one of its own in every
    # dimension (stencil reach <= 2 < 3 + 1): slot = sum_k (agg_k(col) -
    # agg_k(row) + 1) 3^k indexes a dense accumulator of 3^d slots per row,
    # and ascending slots are ascending coarse columns.  agg_k(col) -
    # agg_k(row) = (x_k mod 3 + o_k) // 3 depends on x_k mod 3 and o_k only.
    S = 3 ** dd
    slot_col = np.zeros(S, dtype=np.int64)
    for k in range(dd):
        slot_col += ((np.arange(S) // 3 ** k) % 3) * nc ** k
    lens, cols, es, qs = [], [], [], []
    for r0 in range(0, N, _ROW_BLOCK):
        r1 = min(N, r0 + _ROW_BLOCK)
        order, _, rows, x, ok = _stencil_block(dims, off, r0, r1)
        o = off[order]
        slot = np.zeros(ok.shape, dtype=np.int64)
        base_col = np.zeros(r1 - r0, dtype=np.int64)
        for k in range(dd):
            slot += ((x[k] % 3)[:, None] + o[None, :, k]) // 3 * 3 ** k + 3 ** k
            base_col += (x[k] // 3 - 1) * nc ** k
        key = (np.arange(r1 - r0, dtype=np.int64)[:, None] * S + slot)[ok]
        size = (r1 - r0) * S
        wo = np.broadcast_to(w[order][None, :], ok.shape)[ok]
        centre = np.broadcast_to(np.all(o == 0, axis=1)[None, :], ok.shape)[ok].astype(np.float64)
        used = np.bincount(key, minlength=size) > 0
        e = np.bincount(key, weights=centre, minlength=size)[used]    # P_tent part
        q = np.bincount(key, weights=wo, minlength=size)[used]        # (A P_tent) part
        idx = np.nonzero(used)[0]
        urow, sl = idx // S, idx % S
        ucol = (base_col[urow] + slot_col[sl]).astype(np.int32)
        if not block:
            val = e - scale * q
            keep = val != 0.0
            urow, ucol, e, q = urow[keep], ucol[keep], val[keep], None
        lens.append(np.bincount(urow, minlength=r1 - r0))
        cols.append(ucol)
        es.append(e)
        qs.append(q)
    rp = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(np.concatenate(lens), out=rp[1:])
    s = Csr(N, NC, rp, np.concatenate(cols), np.concatenate(es))
    if not block:
        return s
    kb = ELASTICITY_BLOCK
    return _block_kron(s, np.eye(kb.shape[0]), zero_drop=True, extra=(-scale * np.concatenate(qs), kb))


def family_problem(name: str, n: int):
    """(A, P, R = P^T) of a multigrid family on an n^d grid."""
    a = stencil_matrix(name, n)
    p = smoothed_prolongator(name, n)
    return a, p, transpose(p)


def _coo_to_csr(n: int, rows: np.ndarray, cols: np.ndarray, val_dtype=np.float32) -> Csr:
    key = np.unique(rows.astype(np.int64) * n + cols.astype(np.int64))
    r = key // n
    c = (key % n).astype(np.int32)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rp[1:])
    return Csr(n, n, rp, c, np.ones(len(c), dtype=val_dtype))


def rmat_symmetric(scale: int, edge_factor: int = 16, abcd=(0.57, 0.19, 0.19, 0.05),
                   seed: int = 1, chunk: int = 1 << 21) -> Csr:
    """Symmetrised R-MAT graph, values 1.0 (float32).  Edge e, level l draws
    one uniform from counter e*scale + l and picks a quadrant: [0,a) top-left,
    [a,a+b) top-right, [a+b,a+b+c) bottom-left, else bottom-right; level 0
    decides the most significant bit."""
    n = 1 << scale
    m = edge_factor * n
    a, b, c, _ = abcd
    rs, cs = [], []
    for e0 in range(0, m, chunk):
        e = np.arange(e0, min(m, e0 + chunk), dtype=np.uint64)
        r = np.zeros(len(e), dtype=np.int64)
        cc = np.zeros(len(e), dtype=np.int64)
        for lvl in range(scale):
            u = uniform01(e * _U64(scale) + _U64(lvl), seed)
            rbit = (u >= a + b).astype(np.int64)
            cbit = (((u >= a) & (u < a + b)) | (u >= a + b + c)).astype(np.int64)
            bit = scale - 1 - lvl
            r |= rbit << bit
            cc |= cbit << bit
        keep = r != cc
        rs.append(r[keep]); cs.append(cc[keep])
    r = np.concatenate(rs); cc = np.concatenate(cs)
    return _coo_to_csr(n, np.concatenate([r, cc]), np.concatenate([cc, r]))


def random_square(n: int, seed: int, rmin: int = 4, rmax: int = 32, dtype=np.float32) -> Csr:
    """n x n matrix, each row holding a uniform rmin..rmax distinct random
    columns (uniform without replacement: the first distinct ones of a row's
    candidate draws), N(0,1) values (Box-Muller), columns ascending."""
    return random_rows(n, n, seed, rmin, rmax, dtype)


def random_rhs(nrows: int, ncols: int, delta: int, seed: int, dtype=np.float64) -> Csr:
    """Random right-hand side of the density experiment (Section 4, Table 2):
    nrows x ncols, every row holding min(delta, ncols) distinct uniform
    random columns, N(0,1) values."""
    return random_rows(nrows, ncols, seed, delta, delta, dtype)


def random_rows(nrows: int, ncols: int, seed: int, rmin: int, rmax: int, dtype=np.float32) -> Csr:
    """nrows x ncols matrix, each row holding a uniform rmin..rmax distinct
    random columns (at most ncols; uniform without replacement: the first
    distinct ones of the row's candidate draws), N(0,1) values (Box-Muller),
    columns ascending."""
    n = nrows
    ncand = rmax + 16
    rows = np.arange(n, dtype=np.uint64)
    rlen = rmin + (uniform01(rows, seed, 1) * (rmax - rmin + 1)).astype(np.int64)
    rlen = np.minimum(rlen, min(rmax, ncols))
    cand_ctr = rows[:, None] * _U64(ncand) + np.arange(ncand, dtype=np.uint64)[None, :]
    cand = (uniform01(cand_ctr, seed, 2) * ncols).astype(np.int64)
    # position of each candidate's first occurrence in its row
    order = np.argsort(cand, axis=1, kind="stable")
    sc = np.take_along_axis(cand, order, axis=1)
    first = np.ones_like(sc, dtype=bool)
    first[:, 1:] = sc[:, 1:] != sc[:, :-1]
    keep = np.zeros_like(first)
    np.put_along_axis(keep, order, first, axis=1)          # True at first occurrences
    rank = np.cumsum(keep, axis=1) - 1                      # index among distinct draws
    take = keep & (rank < rlen[:, None])
    lens = take.sum(axis=1).astype(np.int64)
    short = np.nonzero(lens < rlen)[0]
    rows_sel, cols_sel = np.nonzero(take)
    vals = cand[rows_sel, cols_sel]
    extra_r, extra_c = [], []
    for i in short:   # extremely rare: draw more from a further stream
        seen = set(cand[i][keep[i]].tolist())
        k = 0
        while len(seen) < rlen[i]:
            v = int(uniform01(np.array([int(i) * 1024 + k], dtype=np.uint64), seed, 3)[0] * ncols)
            k += 1
            if v not in seen:
                seen.add(v); extra_r.append(i); extra_c.append(v)
    r_all = np.concatenate([rows_sel.astype(np.int64), np.array(extra_r, dtype=np.int64)])
    c_all = np.concatenate([vals, np.array(extra_c, dtype=np.int64)])
    o = np.lexsort((c_all, r_all))
    r_all, c_all = r_all[o], c_all[o]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r_all, minlength=n), out=rp[1:])
    col = c_all.astype(np.int32)
    nnz = int(rp[-1])
    ctr = np.arange(nnz, dtype=np.uint64)
    u1 = uniform01(ctr, seed, 4)
    u2 = uniform01(ctr, seed, 5)
    val = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
    return Csr(n, ncols, rp, col, val.astype(dtype))


def batch_sizes(count: int, lo: int, hi: int, seed: int = 1) -> list[int]:
    """n_i = floor(exp(U[ln lo, ln hi])) for i < count."""
    u = uniform01(np.arange(count, dtype=np.uint64), seed, 6)
    return [int(math.floor(math.exp(math.log(lo) + x * (math.log(hi) - math.log(lo))))) for x in u]


def random_batch(count: int = 256, lo: int = 1024, hi: int = 65536, seed: int = 1,
                 dtype=np.float32):
    """List of (A_i, B_i) pairs; instance i uses seeds 2*(seed+i) and 2*(seed+i)+1."""
    out = []
    for i, n in enumerate(batch_sizes(count, lo, hi, seed)):
        s = seed + i
        out.append((random_square(n, 2 * s, dtype=dtype), random_square(n, 2 * s + 1, dtype=dtype)))
    return out


def random_csr(nrows: int, ncols: int, density: float, seed: int, dtype=np.float64,
               shuffle_cols: bool = False) -> Csr:
    """Small random test matrix: each (i,j) stored with probability density,
    values uniform in [-1, 1).  shuffle_cols permutes columns within each row
    (unsorted input)."""
    ctr = np.arange(nrows * ncols, dtype=np.uint64)
    keep = uniform01(ctr, seed, 7) < density
    mask = keep.reshape(nrows, ncols)
    rows, cols = np.nonzero(mask)
    vals = uniform01(ctr, seed, 8)[mask.reshape(-1)] * 2.0 - 1.0
    rp = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=nrows), out=rp[1:])
    col = cols.astype(np.int32)
    if shuffle_cols:
        key = uniform01(np.arange(len(col), dtype=np.uint64), seed, 9)
        order = np.lexsort((key, rows))
        col = col[order]; vals = vals[order]
    return Csr(nrows, ncols, rp, col, vals.astype(dtype))
