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


def host_csr(c):
    """A device product copied back as an inputs.Csr (FP64 values), so that
    the oracle can take exactly the values a later device product consumed."""
    from paper_1804_00695_gb300 import inputs as I
    return I.Csr(c.nrows, c.ncols, c.row_ptr.cpu().numpy(), c.col.cpu().numpy(),
                 c.val.double().cpu().numpy())


def oracle_product(a, b, dtype=np.float64):
    """Oracle on inputs rounded to the device dtype first (promotion is exact)."""
    from paper_1804_00695_gb300 import inputs as I
    a2 = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, a.val.astype(dtype).astype(np.float64))
    b2 = I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, b.val.astype(dtype).astype(np.float64))
    return oracle.spgemm(a2, b2)


def grad_bounds(a, b, c_row_ptr, c_col, dc):
    """Per-entry error scales of the backward: sum_j |dC_ij||b_kj| for every
    stored a_ik and sum_i |a_ik||dC_ij| for every stored b_kj (the terms each
    gradient entry sums), from the oracle gradient of |.| inputs."""
    from paper_1804_00695_gb300 import inputs as I
    absdc = np.abs(np.asarray(dc, dtype=np.float64))
    ones_a = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, np.ones(a.nnz))
    ones_b = I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, np.ones(b.nnz))
    abs_a = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, np.abs(a.val.astype(np.float64)))
    abs_b = I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, np.abs(b.val.astype(np.float64)))
    ba, _ = oracle.backward(ones_a, abs_b, c_row_ptr, c_col, absdc)
    _, bb = oracle.backward(abs_a, ones_b, c_row_ptr, c_col, absdc)
    return ba, bb


def assert_grads_match(a, b, c_row_ptr, c_col, dc, da, db, tol):
    """dA and dB (host arrays) against the oracle gradient of <dC, A*B>,
    each entry within tol times the sum of the absolute terms it adds."""
    ra, rb = oracle.backward(a, b, c_row_ptr, c_col, np.asarray(dc, dtype=np.float64))
    ba, bb = grad_bounds(a, b, c_row_ptr, c_col, dc)
    assert np.all(np.abs(np.asarray(da, dtype=np.float64) - ra) <= tol * ba), "dA out of tolerance"
    assert np.all(np.abs(np.asarray(db, dtype=np.float64) - rb) <= tol * bb), "dB out of tolerance"
