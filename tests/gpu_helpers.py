"""Shared helpers of the GPU parity tests: move inputs to the device and
compare the library's product with the CPU oracle element by element."""
import numpy as np

import oracle
import paper_1804_00695_gb300 as sg

TOL = {"f64": 1e-12, "f32": 1e-5}


def to_dev(m, dtype=np.float64):
    return sg.Csr.from_host(m, "cuda", dtype)


def assert_matches(c, ref, dtype: str):
    """c: sg.Csr on the device; ref: oracle.Result.  Pattern bit-exact,
    values within tol * sum |a_ik||b_kj| (exact where that sum is 0)."""
    rp = c.row_ptr.cpu().numpy()
    col = c.col.cpu().numpy()
    val = c.val.double().cpu().numpy()
    assert rp.shape == ref.row_ptr.shape
    assert np.array_equal(rp, ref.row_ptr), "row_ptr differs"
    assert np.array_equal(col, ref.col), "columns differ"
    err = np.abs(val - ref.val)
    lim = TOL[dtype] * ref.bound
    bad = err > lim
    if bad.any():
        k = int(np.argmax(bad))
        raise AssertionError(f"{int(bad.sum())} values out of tolerance; first at {k}: "
                             f"got {val[k]!r} want {ref.val[k]!r} bound {ref.bound[k]!r}")


def oracle_product(a, b, dtype=np.float64):
    """Oracle on inputs rounded to the device dtype first (promotion is exact)."""
    from paper_1804_00695_gb300 import inputs as I
    a2 = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, a.val.astype(dtype).astype(np.float64))
    b2 = I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, b.val.astype(dtype).astype(np.float64))
    return oracle.spgemm(a2, b2)
