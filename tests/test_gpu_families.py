"""GPU parity of the products of every multigrid family of Section 4
(Laplace3D 7-point, BigStar2D 13-point, Brick3D 27-point, Elasticity 81 per
row) against the CPU oracle, through the C ABI: R*A and A*P separately (as
the paper reports them) and R*(AP) with the oracle's AP as B, at sizes that
span many row blocks with a ragged last one; FP64 and FP32."""
import numpy as np
import pytest

import oracle
import paper_1804_00695_gb300 as sg
from paper_1804_00695_gb300 import inputs as I
from gpu_helpers import assert_matches, oracle_product, to_dev

pytestmark = pytest.mark.gpu

SIZES = {"laplace3d_7pt": (23, 41), "bigstar2d_13pt": (97, 301), "brick3d_27pt": (19, 35),
         "elasticity3d_81": (11, 22)}


@pytest.fixture(scope="module")
def h(cuda_lib):
    return sg.Handle()


@pytest.mark.parametrize("name", list(SIZES))
@pytest.mark.parametrize("which", [0, 1])
def test_family_products(h, name, which):
    n = SIZES[name][which]
    a, p, r = I.family_problem(name, n)
    A, P, R = to_dev(a), to_dev(p), to_dev(r)
    assert_matches(h.spgemm(R, A), oracle.spgemm(r, a), "f64")
    ap_o = oracle.spgemm(a, p)
    assert_matches(h.spgemm(A, P), ap_o, "f64")
    ap = I.Csr(ap_o.nrows, ap_o.ncols, ap_o.row_ptr, ap_o.col, ap_o.val)
    assert_matches(h.spgemm(R, to_dev(ap)), oracle.spgemm(r, ap), "f64")


@pytest.mark.parametrize("name", list(SIZES))
def test_family_products_f32(h, name):
    n = SIZES[name][0]
    a, p, r = I.family_problem(name, n)
    assert_matches(h.spgemm(to_dev(a, np.float32), to_dev(p, np.float32)), oracle_product(a, p, np.float32), "f32")
    assert_matches(h.spgemm(to_dev(r, np.float32), to_dev(a, np.float32)), oracle_product(r, a, np.float32), "f32")
