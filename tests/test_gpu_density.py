"""GPU parity of the right-hand-side density experiment (Section 4, Table 2):
the Elasticity family's R and A multiplied by random right-hand sides with
delta = 1, 4, 16, 64 and 256 entries per row, against the CPU oracle through
the C ABI (pattern bit-exact, values within the FP64 bound).  The densest
right-hand sides give rows of C that fill most of their columns, the sparsest
ones rows of one entry per stored a_ik."""
import numpy as np
import pytest

import oracle
import paper_1804_00695_gb300 as sg
from paper_1804_00695_gb300 import inputs as I
from gpu_helpers import assert_matches, oracle_product, to_dev

pytestmark = pytest.mark.gpu

DELTAS = [1, 4, 16, 64, 256]


@pytest.fixture(scope="module")
def h(cuda_lib):
    return sg.Handle()


@pytest.mark.parametrize("n", [7, 10])
@pytest.mark.parametrize("delta", DELTAS)
def test_density_products(h, n, delta):
    a, _, r = I.family_problem("elasticity3d_81", n)
    rhs = I.random_rhs(a.ncols, a.ncols, delta, seed=100 + delta)
    Y = to_dev(rhs)
    assert_matches(h.spgemm(to_dev(r), Y), oracle.spgemm(r, rhs), "f64")
    assert_matches(h.spgemm(to_dev(a), Y), oracle.spgemm(a, rhs), "f64")


@pytest.mark.parametrize("delta", [4, 256])
def test_density_products_f32(h, delta):
    a, _, r = I.family_problem("elasticity3d_81", 8)
    rhs = I.random_rhs(a.ncols, a.ncols, delta, seed=7)
    for x in (r, a):
        got = h.spgemm(to_dev(x, np.float32), to_dev(rhs, np.float32))
        assert_matches(got, oracle_product(x, rhs, np.float32), "f32")
