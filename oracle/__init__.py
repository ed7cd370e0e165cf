"""CPU oracle for C = A*B (Gustavson, dense accumulator, IEEE double).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU baseline import this package; the CUDA library never does, and
this package imports nothing from it.

Functions follow Deveci et al., "Sparse Matrix-Matrix Multiplication on
Multilevel Memory Architectures":
  * ``spgemm``            - Section 2.1 (row-wise two-phase product), with the
                            dense accumulator of Section 3.1;
  * ``fma_range``         - Section 3.2.2 (fused multiply-add over a row range
                            of B, the subprocedure of Algorithms 1-3);
  * ``backward``          - exact gradients of <dC, A*B> on the stored patterns;
  * ``compress_rows``     - Section 2.1 column compression (block index, bit mask);
  * ``row_flops``         - Section 3.1: insertions per row = multiplications;
  * ``partition`` & co.   - Algorithm 4 and the copy costs of Algorithms 2 and 3
                            (see ``oracle.chunking``);
  * ``triangles``         - triangle counting by the masked product L*L .* L
                            of Section 4.1's triangle-counting experiment
                            (degree-ordered lower triangle, sorted-row merges).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        i64, p = C.c_int64, C.c_void_p
        _lib.oracle_validate_csr.argtypes = [i64, i64, p, p]
        _lib.oracle_symbolic_rows.argtypes = [i64, i64, i64, p, p, p, p, p, p]
        _lib.oracle_numeric_rows.argtypes = [i64, i64, i64, p, p, p, p, p, p, p, p, p, p]
        _lib.oracle_fma_range_rows.argtypes = [i64, i64, i64, i64, i64] + [p] * 13
        _lib.oracle_backward.argtypes = [i64, i64] + [p] * 11
        _lib.oracle_set_num_threads.argtypes = [C.c_int]
        _lib.oracle_degree_order.argtypes = [i64, p, p]
        _lib.oracle_triangles.argtypes = [i64, p, p, p, p]
        _lib.oracle_triangles.restype = i64
    return _lib


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(n: int) -> None:
    lib().oracle_set_num_threads(int(n))


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _cf(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Result:
    """Oracle product: CSR arrays plus the per-entry bound sum |a_ik||b_kj|."""

    def __init__(self, nrows, ncols, row_ptr, col, val, bound, mults):
        self.nrows, self.ncols = nrows, ncols
        self.row_ptr, self.col, self.val, self.bound, self.mults = row_ptr, col, val, bound, mults

    @property
    def nnz(self):
        return int(self.row_ptr[-1])


def validate(m) -> int:
    """0 if well formed; 1 bad row_ptr, 2 column out of range, 3 duplicate column."""
    return int(lib().oracle_validate_csr(m.nrows, m.ncols, _p(_c64(m.row_ptr)), _p(_c32(m.col))))


def symbolic(a, b, r0: int = 0, r1: int | None = None):
    """(cnt, mults) per row of C for rows [r0, r1)."""
    r1 = a.nrows if r1 is None else r1
    cnt = np.zeros(r1 - r0, dtype=np.int64)
    mults = np.zeros(r1 - r0, dtype=np.int64)
    arp, acol, brp, bcol = _c64(a.row_ptr), _c32(a.col), _c64(b.row_ptr), _c32(b.col)
    rc = lib().oracle_symbolic_rows(r0, r1, b.ncols, _p(arp), _p(acol), _p(brp), _p(bcol),
                                    _p(cnt), _p(mults))
    if rc != 0:
        raise MemoryError("oracle symbolic failed")
    return cnt, mults


def spgemm(a, b, r0: int = 0, r1: int | None = None) -> Result:
    """C[r0:r1] = A[r0:r1] * B in IEEE double, columns ascending per row."""
    if a.ncols != b.nrows:
        raise ValueError("dimension mismatch")
    r1 = a.nrows if r1 is None else r1
    cnt, mults = symbolic(a, b, r0, r1)
    rp = np.zeros(r1 - r0 + 1, dtype=np.int64)
    np.cumsum(cnt, out=rp[1:])
    nnz = int(rp[-1])
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz, dtype=np.float64)
    bound = np.zeros(nnz, dtype=np.float64)
    arp, acol, aval = _c64(a.row_ptr), _c32(a.col), _cf(a.val)
    brp, bcol, bval = _c64(b.row_ptr), _c32(b.col), _cf(b.val)
    rc = lib().oracle_numeric_rows(r0, r1, b.ncols, _p(arp), _p(acol), _p(aval),
                                   _p(brp), _p(bcol), _p(bval), _p(rp), _p(col), _p(val), _p(bound))
    if rc != 0:
        raise RuntimeError(f"oracle numeric failed ({rc})")
    return Result(r1 - r0, b.ncols, rp, col, val, bound, mults)


def fma_range(a, b, lo: int, hi: int, partial=None):
    """C2 = A[:, lo:hi] * B[lo:hi, :] + C1 (Section 3.2.2); partial = C1 as
    (row_ptr, col, val) or None for an empty C1.  Returns (row_ptr, col, val)."""
    n = a.nrows
    arp, acol, aval = _c64(a.row_ptr), _c32(a.col), _cf(a.val)
    brp, bcol, bval = _c64(b.row_ptr), _c32(b.col), _cf(b.val)
    if partial is not None:
        prp, pcol, pval = _c64(partial[0]), _c32(partial[1]), _cf(partial[2])
    else:
        prp = pcol = pval = None
    cnt = np.zeros(n, dtype=np.int64)
    L = lib()
    rc = L.oracle_fma_range_rows(0, n, b.ncols, lo, hi, _p(arp), _p(acol), _p(aval), _p(brp), _p(bcol),
                                 _p(bval), _p(prp), _p(pcol), _p(pval), _p(cnt), None, None, None)
    if rc != 0:
        raise MemoryError
    orp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt, out=orp[1:])
    ocol = np.zeros(int(orp[-1]), dtype=np.int32)
    oval = np.zeros(int(orp[-1]), dtype=np.float64)
    rc = L.oracle_fma_range_rows(0, n, b.ncols, lo, hi, _p(arp), _p(acol), _p(aval), _p(brp), _p(bcol),
                                 _p(bval), _p(prp), _p(pcol), _p(pval), _p(cnt), _p(orp), _p(ocol), _p(oval))
    if rc != 0:
        raise MemoryError
    return orp, ocol, oval


def backward(a, b, c_row_ptr, c_col, dc_val):
    """(dA values on pattern(A), dB values on pattern(B)) of L = <dC, A*B>."""
    da = np.zeros(a.nnz, dtype=np.float64)
    db = np.zeros(b.nnz, dtype=np.float64)
    arp, acol, aval = _c64(a.row_ptr), _c32(a.col), _cf(a.val)
    brp, bcol, bval = _c64(b.row_ptr), _c32(b.col), _cf(b.val)
    crp, ccol, dcv = _c64(c_row_ptr), _c32(c_col), _cf(dc_val)
    rc = lib().oracle_backward(a.nrows, b.ncols, _p(arp), _p(acol), _p(aval), _p(brp), _p(bcol), _p(bval),
                               _p(crp), _p(ccol), _p(dcv), _p(da), _p(db))
    if rc != 0:
        raise RuntimeError(f"oracle backward failed ({rc})")
    return da, db


def row_flops(a, b) -> np.ndarray:
    """Multiplications per row of C: sum over stored a_ik of nnz(B_k)."""
    blen = np.diff(b.row_ptr)
    per_entry = blen[a.col.astype(np.int64)]
    out = np.zeros(a.nrows, dtype=np.int64)
    rows = np.repeat(np.arange(a.nrows), np.diff(a.row_ptr))
    np.add.at(out, rows, per_entry)
    return out


def compress_rows(m):
    """Section 2.1 column compression: each row's column set as ascending
    (block = col // 32, mask with bit col % 32 set) pairs, one per block.
    Returns (row_ptr, block, mask) with mask as uint32."""
    rows = np.repeat(np.arange(m.nrows, dtype=np.int64), np.diff(m.row_ptr))
    blk = m.col.astype(np.int64) // 32
    bit = (np.uint64(1) << (m.col.astype(np.uint64) % np.uint64(32))).astype(np.uint64)
    key = rows * (1 << 26) + blk
    uniq, inv = np.unique(key, return_inverse=True)
    mask = np.zeros(len(uniq), dtype=np.uint64)
    np.bitwise_or.at(mask, inv, bit)
    urow = uniq // (1 << 26)
    rp = np.zeros(m.nrows + 1, dtype=np.int64)
    np.cumsum(np.bincount(urow, minlength=m.nrows), out=rp[1:])
    return rp, (uniq % (1 << 26)).astype(np.int32), mask.astype(np.uint32)


def _sub_rows(m, r0: int, r1: int):
    """Rows [r0, r1) of a CSR matrix as a new matrix (offsets rebased)."""
    from types import SimpleNamespace
    p0, p1 = int(m.row_ptr[r0]), int(m.row_ptr[r1])
    return SimpleNamespace(nrows=r1 - r0, ncols=m.ncols, row_ptr=m.row_ptr[r0:r1 + 1] - p0,
                           col=m.col[p0:p1], val=m.val[p0:p1], nnz=p1 - p0)


def _cat_rows(parts):
    """Concatenate (row_ptr, col, val) row blocks in order."""
    rps, cols, vals, off = [np.zeros(1, dtype=np.int64)], [], [], 0
    for rp, col, val in parts:
        rps.append(rp[1:] + off)
        off += int(rp[-1])
        cols.append(col); vals.append(val)
    return (np.concatenate(rps), np.concatenate(cols) if cols else np.zeros(0, np.int32),
            np.concatenate(vals) if vals else np.zeros(0))


def degree_order(g) -> np.ndarray:
    """New label of every vertex: position of (degree, vertex) in ascending
    order (ties by vertex index)."""
    perm = np.zeros(g.nrows, dtype=np.int64)
    if lib().oracle_degree_order(g.nrows, _p(_c64(g.row_ptr)), _p(perm)) != 0:
        raise MemoryError("oracle degree order failed")
    return perm


def triangles(g, perm=None):
    """(total, per-vertex counts) of triangles of the undirected graph with
    the symmetric pattern g (no self loops), by the masked product L*L .* L:
    L the strictly lower triangle after relabelling by `perm` (default: the
    degree order); the count of vertex u is the number of triangles whose
    highest-labelled vertex is u."""
    rc = np.zeros(g.nrows, dtype=np.int64)
    pp = None if perm is None else _c64(perm)
    total = lib().oracle_triangles(g.nrows, _p(_c64(g.row_ptr)), _p(_c32(g.col)), _p(pp), _p(rc))
    if total == -1:
        raise MemoryError("oracle triangles failed")
    if total == -2:
        raise ValueError("perm is not a permutation")
    return int(total), rc
