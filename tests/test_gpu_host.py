"""GPU parity of spgemm_host (operands in host memory, copied in by the
library, both phases on the device, C copied out or kept on the device)
against the CPU oracle, through the C ABI: the Galerkin chain with the
intermediate product kept on the device, FP32 with unsorted rows, empty
results, and a failing allocator."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1804_00695_gb300 as sg
from paper_1804_00695_gb300 import inputs as I
from gpu_helpers import assert_matches, host_csr, oracle_product

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h(cuda_lib):
    return sg.Handle()


def _host_result(c):
    """A HostCsr result as an inputs.Csr (FP64 values) for the oracle checks."""
    return I.Csr(c.nrows, c.ncols, c.row_ptr.numpy(), c.col.numpy(), c.val.double().numpy())


def _matches_host(c, ref, tag):
    from gpu_helpers import TOL
    assert np.array_equal(c.row_ptr.numpy(), ref.row_ptr)
    assert np.array_equal(c.col.numpy(), ref.col)
    assert np.all(np.abs(c.val.double().numpy() - ref.val) <= TOL[tag] * ref.bound)


@pytest.mark.parametrize("n", [9, 16])
def test_host_galerkin_chain(h, n):
    """A and P on the host -> AP kept on the device -> R (host) * AP -> RAP on
    the host; each product against the oracle (R*AP on the device AP)."""
    a, p, r = I.galerkin_problem(n)
    A, P, R = (sg.HostCsr.from_numpy(m) for m in (a, p, r))
    ap = h.host_product(A, P, keep_on_device=True)
    assert ap.row_ptr.device.type == "cuda"
    assert_matches(ap, oracle.spgemm(a, p), "f64")
    rap = h.host_product(R, ap)
    assert rap.row_ptr.device.type == "cpu"
    _matches_host(rap, oracle.spgemm(r, host_csr(ap)), "f64")
    for _ in range(2):                       # repeated calls reuse the device copies
        ap2 = h.host_product(A, P)
        _matches_host(ap2, oracle.spgemm(a, p), "f64")


@pytest.mark.parametrize("shape,dens,seed", [((300, 200, 500), 0.03, 2), ((64, 900, 40), 0.2, 5)])
def test_host_random_f32_unsorted(h, shape, dens, seed):
    m, k, n = shape
    a = I.random_csr(m, k, dens, seed, shuffle_cols=True)
    b = I.random_csr(k, n, dens, seed + 50, shuffle_cols=True)
    c = h.host_product(sg.HostCsr.from_numpy(a, np.float32), sg.HostCsr.from_numpy(b, np.float32))
    _matches_host(c, oracle_product(a, b, np.float32), "f32")


def test_host_empty_and_allocator_failure(h):
    z = I.Csr(6, 5, np.zeros(7, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0))
    b = I.random_csr(5, 7, 0.5, 9)
    c = h.host_product(sg.HostCsr.from_numpy(z), sg.HostCsr.from_numpy(b))
    assert c.nnz == 0 and c.row_ptr.tolist() == [0] * 7
    import torch
    a = I.random_csr(40, 30, 0.3, 10)
    A, B = sg.HostCsr.from_numpy(a), sg.HostCsr.from_numpy(I.random_csr(30, 20, 0.3, 11))
    lib = sg.load()
    fail = sg.ALLOC_FN(lambda user, nnz, col_p, val_p: 1)
    rp = torch.empty(a.nrows + 1, dtype=torch.int64).pin_memory()
    dc = sg.CsrDesc(a.nrows, 20, 0, rp.data_ptr(), None, None)
    da, db = A.desc(), B.desc()
    st = lib.spgemm_host(h._h, sg.F64, ctypes.byref(da), ctypes.byref(db), ctypes.byref(dc), fail, None, 0,
                         torch.cuda.current_stream().cuda_stream)
    assert st == 4
    # the handle stays usable
    c = h.host_product(A, B)
    _matches_host(c, oracle.spgemm(a, _host_result(B)), "f64")
