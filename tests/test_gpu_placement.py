"""GPU parity of the device calls with their operands in each placement of
Table 3 (Section 3.3.1): all in HBM, A / B / C in pinned host memory (read
and written in place by the kernels over the host link), all pinned, and all
in managed (UVM) memory; against the CPU oracle through the C ABI.  The
placement changes where the bytes travel, never the result: pattern exact and
values within the usual bound in every case."""
import numpy as np
import pytest

import oracle
import paper_1804_00695_gb300 as sg
from paper_1804_00695_gb300 import inputs as I
from gpu_helpers import assert_matches, host_csr, oracle_product

pytestmark = pytest.mark.gpu

# (placement of A, of B, of C), named as the columns of Table 3
PLACEMENTS = {
    "HBM": ("device", "device", "device"),
    "A_Pin": ("pinned", "device", "device"),
    "B_Pin": ("device", "pinned", "device"),
    "C_Pin": ("device", "device", "pinned"),
    "HostPin": ("pinned", "pinned", "pinned"),
    "UVM": ("managed", "managed", "managed"),
}


@pytest.fixture(scope="module")
def h(cuda_lib):
    return sg.Handle()


def _where(t):
    """'device', 'pinned' or 'managed', as seen from torch."""
    if t.device.type == "cpu":
        return "pinned" if t.is_pinned() else "pageable"
    return "managed" if hasattr(t, "_managed_owner") else "device"


@pytest.mark.parametrize("name", list(PLACEMENTS))
@pytest.mark.parametrize("n", [12, 24])
def test_galerkin_placements(h, name, n):
    """R*(A*P) of the 27-point problem with each placement for both products."""
    pa, pb, pc = PLACEMENTS[name]
    a, p, r = I.galerkin_problem(n)
    A, P = sg.Csr.placed(a, pa), sg.Csr.placed(p, pb)
    assert _where(A.col) == pa and _where(P.col) == pb
    ap = h.spgemm(A, P, placement=pc)
    assert _where(ap.col) == pc and _where(ap.row_ptr) == pc
    assert_matches(ap, oracle.spgemm(a, p), "f64")
    # R*AP: R in A's placement, the AP just made as B, C in pc
    R = sg.Csr.placed(r, pa)
    rap = h.spgemm(R, ap, placement=pc)
    assert_matches(rap, oracle.spgemm(r, host_csr(ap)), "f64")


@pytest.mark.parametrize("name", ["A_Pin", "HostPin", "UVM"])
def test_random_f32_unsorted_placements(h, name):
    """FP32, unsorted input rows, ragged shapes, several bins of rows."""
    pa, pb, pc = PLACEMENTS[name]
    a = I.random_csr(700, 400, 0.03, 11, shuffle_cols=True)
    b = I.random_csr(400, 900, 0.05, 12, shuffle_cols=True)
    c = h.spgemm(sg.Csr.placed(a, pa, np.float32), sg.Csr.placed(b, pb, np.float32), placement=pc)
    assert_matches(c, oracle_product(a, b, np.float32), "f32")


def test_mixed_and_empty(h):
    """A pinned times B managed with C in HBM; an empty A in pinned memory."""
    a = I.random_csr(333, 257, 0.02, 21)
    b = I.random_csr(257, 129, 0.04, 22)
    c = h.spgemm(sg.Csr.placed(a, "pinned"), sg.Csr.placed(b, "managed"))
    assert_matches(c, oracle.spgemm(a, b), "f64")
    z = I.Csr(50, 257, np.zeros(51, dtype=np.int64), np.zeros(0, np.int32), np.zeros(0))
    c = h.spgemm(sg.Csr.placed(z, "pinned"), sg.Csr.placed(b, "pinned"), placement="pinned")
    assert c.nnz == 0 and np.array_equal(c.row_ptr.numpy(), np.zeros(51, dtype=np.int64))


def test_backward_pinned(h):
    """Gradients of <dC, A*B> with A, B, dC and the gradients' inputs pinned."""
    from gpu_helpers import assert_grads_match
    import torch
    a = I.random_csr(300, 200, 0.05, 31)
    b = I.random_csr(200, 250, 0.05, 32)
    A, B = sg.Csr.placed(a, "pinned"), sg.Csr.placed(b, "pinned")
    c = h.spgemm(A, B, placement="pinned")
    dc = I.uniform01(np.arange(c.nnz, dtype=np.uint64), 33, 1) - 0.5
    dC = torch.from_numpy(dc).pin_memory()
    da, db = h.backward(A, B, c, dC)
    assert_grads_match(a, b, c.row_ptr.numpy(), c.col.numpy(), dc, da.cpu().numpy(), db.cpu().numpy(), 1e-12)
