"""GPU parity of the backward kernel and the autograd Function: dA and dB
against the oracle gradient, the bilinear identity <dA,A> = <dC,C> = <dB,B>,
and torch.autograd through the library."""
import numpy as np
import pytest

import oracle
import paper_1804_00695_gb300 as sg
from paper_1804_00695_gb300 import inputs as I
from gpu_helpers import assert_grads_match, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h(cuda_lib):
    return sg.Handle()


def grads(h, a, b, dtype, seed):
    import torch
    A, B = to_dev(a, dtype), to_dev(b, dtype)
    C = h.spgemm(A, B)
    dc = (I.uniform01(np.arange(C.nnz, dtype=np.uint64), seed) * 2 - 1).astype(dtype)
    da, db = h.backward(A, B, C, torch.from_numpy(dc).cuda())
    h.check()
    ref = oracle.spgemm(I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, a.val.astype(dtype).astype(np.float64)),
                        I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, b.val.astype(dtype).astype(np.float64)))
    ra, rb = oracle.backward(I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, a.val.astype(dtype).astype(np.float64)),
                             I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, b.val.astype(dtype).astype(np.float64)),
                             ref.row_ptr, ref.col, dc.astype(np.float64))
    return da.double().cpu().numpy(), db.double().cpu().numpy(), ra, rb, dc, ref


def bound_a(a, b, ref, dc):
    """sum over terms of |dC_ij||b_kj| per entry of A (tolerance scale)."""
    absd = I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, np.abs(b.val.astype(np.float64)))
    dct = I.Csr(ref.nrows, ref.ncols, ref.row_ptr, ref.col, np.abs(dc.astype(np.float64)))
    ba, _ = oracle.backward(I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, np.ones(a.nnz)), absd,
                            ref.row_ptr, ref.col, dct.val)
    return ba


def _wide_case():
    """Rows of C spanning more than 2048 blocks of 32 columns (binary-search
    path) next to narrow rows (shared-memory map path)."""
    nb, ncols, per = 1500, 150000, 12
    k = np.repeat(np.arange(nb), per)
    t = np.tile(np.arange(per), nb)
    wide = (k * 7919 + t * (ncols // per + 3)) % ncols       # rows of B spread over all columns
    narrow = (k * 37 + t * 5) % 2000                          # rows of B within 2000 columns
    cols = np.where(k < nb // 2, wide, narrow)
    key = np.unique(k * ncols + cols)
    rp = np.zeros(nb + 1, dtype=np.int64)
    np.cumsum(np.bincount(key // ncols, minlength=nb), out=rp[1:])
    b = I.Csr(nb, ncols, rp, (key % ncols).astype(np.int32),
              I.uniform01(np.arange(len(key), dtype=np.uint64), 17) - 0.5)
    d = I.random_csr(200, nb, 0.01, 16).to_dense() != 0
    d[:100, : nb // 2] = False          # rows 0..99 reach only the narrow rows of B
    d[np.arange(200), nb // 2 + np.arange(200)] = True
    r, cidx = np.nonzero(d)
    arp = np.zeros(201, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=200), out=arp[1:])
    a = I.Csr(200, nb, arp, cidx.astype(np.int32), I.uniform01(np.arange(len(cidx), dtype=np.uint64), 18) - 0.5)
    return a, b


def _long_rows_case():
    """Rows of C with more than 1024 entries (searched in global memory) next
    to short rows (searched in a shared-memory copy of their columns)."""
    a = I.random_csr(120, 2000, 0.05, 31)
    b = I.random_csr(2000, 5000, 0.02, 32)
    keep = np.ones(a.nnz, dtype=bool)
    rows = np.repeat(np.arange(a.nrows), np.diff(a.row_ptr))
    for i in range(60):                       # rows 0..59 keep two entries each
        keep[a.row_ptr[i] + 2:a.row_ptr[i + 1]] = False
    rp = np.zeros(a.nrows + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows[keep], minlength=a.nrows), out=rp[1:])
    return I.Csr(a.nrows, a.ncols, rp, a.col[keep], a.val[keep]), b


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 1e-5)])
@pytest.mark.parametrize("case", ["random", "batch_like", "galerkin", "wide", "long_rows"])
def test_backward_matches_oracle(h, dtype, tol, case):
    if case == "long_rows":
        a, b = _long_rows_case()
        lens = np.diff(oracle.spgemm(a, b).row_ptr)
        assert lens.max() > 1024 and lens.min() <= 1024
    elif case == "wide":
        a, b = _wide_case()
    elif case == "random":
        a = I.random_csr(300, 200, 0.04, 11, shuffle_cols=True)
        b = I.random_csr(200, 250, 0.05, 12, shuffle_cols=True)
    elif case == "batch_like":
        a = I.random_square(3000, 21, dtype=np.float64)
        b = I.random_square(3000, 22, dtype=np.float64)
    else:
        a, b, _ = I.galerkin_problem(10)
    da, db, ra, rb, dc, ref = grads(h, a, b, dtype, 13)
    ba = bound_a(a, b, ref, dc)
    assert np.all(np.abs(da - ra) <= tol * ba + 1e-300)
    # dB: each entry sums |a_ik||dC_ij| terms; scale by the same kind of bound
    absa = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, np.abs(a.val.astype(dtype).astype(np.float64)))
    _, bb = oracle.backward(absa, I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, np.ones(b.nnz)),
                            ref.row_ptr, ref.col, np.abs(dc.astype(np.float64)))
    assert np.all(np.abs(db - rb) <= tol * bb + 1e-300)
    # Euler identity of the bilinear form on the device results
    lc = float(dc.astype(np.float64) @ ref.val)
    scale = float(np.abs(dc.astype(np.float64)) @ ref.bound)
    assert abs(da @ a.val.astype(dtype).astype(np.float64) - lc) <= 10 * tol * scale
    assert abs(db @ b.val.astype(dtype).astype(np.float64) - lc) <= 10 * tol * scale


def test_autograd_function(h):
    import torch
    a = I.random_csr(120, 90, 0.05, 21)
    b = I.random_csr(90, 80, 0.06, 22)
    A, B = to_dev(a), to_dev(b)
    A.val.requires_grad_(True)
    B.val.requires_grad_(True)
    C = sg.spgemm_autograd(A, B, h)
    w = torch.linspace(-1, 1, C.nnz, dtype=torch.float64, device="cuda")
    loss = (C.val * w).sum()
    loss.backward()
    assert_grads_match(a, b, C.row_ptr.cpu().numpy(), C.col.cpu().numpy(), w.cpu().numpy(),
                       A.val.grad.cpu().numpy(), B.val.grad.cpu().numpy(), 1e-12)
