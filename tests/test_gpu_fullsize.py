"""Full-size parity of the workloads the benchmark measures, in the launch
configuration it uses: every output the oracle can afford is compared
(sampled row blocks, the heaviest rows, sampled batch instances), and
properties that hold at any size are checked on the whole result."""
import numpy as np
import pytest

import oracle
import paper_1804_00695_gb300 as sg
from paper_1804_00695_gb300 import inputs as I
from gpu_helpers import TOL, to_dev

pytestmark = pytest.mark.gpu


def rows_of(c, r0, r1):
    rp = c.row_ptr[r0:r1 + 1].cpu().numpy()
    p0, p1 = int(rp[0]), int(rp[-1])
    return rp - p0, c.col[p0:p1].cpu().numpy(), c.val[p0:p1].double().cpu().numpy()


def test_rmat20_full(cuda_lib):
    """R-MAT scale 20, edge factor 16, C = A*A in FP32 (values are common-neighbour
    counts, exact integers): sampled blocks and the heaviest rows against the
    oracle, the sum of all entries against sum_k deg_k^2, symmetry on samples."""
    import torch
    g = I.rmat_symmetric(20, 16, seed=1)
    h = sg.Handle()
    A = to_dev(g, np.float32)
    c = h.spgemm(A, A)
    h.check()
    deg = np.diff(g.row_ptr)
    total = 0.0
    for p0 in range(0, c.nnz, 1 << 30):     # sum in pieces: a float64 copy of all values would not fit
        total += float(torch.sum(c.val[p0:p0 + (1 << 30)], dtype=torch.float64))
    assert total == float((deg.astype(np.float64) ** 2).sum())
    rng = np.random.default_rng(7)
    blocks = [(int(r), int(r) + 200) for r in rng.integers(0, g.nrows - 200, size=8)]
    blocks += [(0, 64)]
    top = np.argsort(-deg)[:4]
    blocks += [(int(i), int(i) + 1) for i in top]
    for r0, r1 in blocks:
        ref = oracle.spgemm(g, g, r0, r1)
        rp, col, val = rows_of(c, r0, r1)
        assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
        assert np.array_equal(val, ref.val)
    # symmetry: c_ij == c_ji on sampled entries
    r0 = blocks[0][0]
    rp, col, val = rows_of(c, r0, r0 + 20)
    crp = c.row_ptr.cpu()
    for t in range(0, len(col), max(1, len(col) // 300)):
        i = r0 + int(np.searchsorted(rp, t, side="right")) - 1
        j = int(col[t])
        p0, p1 = int(crp[j]), int(crp[j + 1])
        rowj = c.col[p0:p1]
        k = int(torch.searchsorted(rowj, torch.tensor([i], device=rowj.device, dtype=rowj.dtype)))
        assert k < p1 - p0 and int(rowj[k]) == i and float(c.val[p0 + k]) == val[t]


def laplace27_row_lengths(n):
    l2 = np.array([3, 4] + [5] * (n - 4) + [4, 3], dtype=np.int64)
    return (l2[:, None, None] * l2[None, :, None] * l2[None, None, :]).reshape(-1)


def test_chunked256_full(cuda_lib):
    """256^3 27-point Laplacian, C = A*A in FP64 with A, B and C in pinned host
    memory and a 4 GB device budget: every row length against the closed form
    (5n-6)^3 pattern, sampled row blocks against the oracle (exact integers)."""
    n = 256
    a = I.laplace3d_27pt(n)
    assert a.nnz == 449455096
    h = sg.Handle()
    A = sg.HostCsr.from_numpy(a)
    budget = 4 * 10 ** 9
    rp, nnz = h.chunked_symbolic(A, A, budget)
    assert nnz == 2067798824
    lens = laplace27_row_lengths(n)
    assert np.array_equal(np.diff(rp.numpy()), lens)
    c = h.chunked_numeric(A, A, rp, nnz, budget)
    st = h.chunked_stats()
    assert st["device_bytes"] <= budget and st["n_ac"] > 1
    rng = np.random.default_rng(11)
    starts = [0, a.nrows - 300] + [int(x) for x in rng.integers(0, a.nrows - 300, size=10)]
    for r0 in starts:
        r1 = r0 + 300
        ref = oracle.spgemm(a, a, r0, r1)
        p0, p1 = int(rp[r0]), int(rp[r1])
        assert np.array_equal(c.col[p0:p1].numpy(), ref.col)
        assert np.array_equal(c.val[p0:p1].numpy(), ref.val)


def test_batched256_full(cuda_lib):
    """256 random products (rows log-uniform in [1024, 65536], 4-32 columns per
    row, N(0,1) FP32) in one batched call, forward and backward: sampled
    instances (the largest, the smallest, and a spread) against the oracle."""
    import torch
    pairs = I.random_batch(256, 1024, 65536, 1, dtype=np.float64)
    As = [to_dev(a, np.float32) for a, _ in pairs]
    Bs = [to_dev(b, np.float32) for _, b in pairs]
    h = sg.Handle()
    bt = sg.Batch(h, As, Bs)
    Cm = bt.run()
    h.check()
    parts = bt.split(Cm)
    dc = torch.cos(torch.arange(Cm.nnz, device="cuda", dtype=torch.float32) * 0.37)
    da, db = bt.backward(Cm, dc)
    ga, gb = bt.split_grads(da, db)
    sizes = [a.nrows for a, _ in pairs]
    pick = sorted({int(np.argmax(sizes)), int(np.argmin(sizes)), 0, 77, 128, 255})
    offs = np.concatenate([[0], np.cumsum(bt.inst_nnz)])
    for i in pick:
        a, b = pairs[i]
        a32 = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, a.val.astype(np.float32).astype(np.float64))
        b32 = I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, b.val.astype(np.float32).astype(np.float64))
        ref = oracle.spgemm(a32, b32)
        c = parts[i]
        assert np.array_equal(c.row_ptr.cpu().numpy(), ref.row_ptr)
        assert np.array_equal(c.col.cpu().numpy(), ref.col)
        assert np.all(np.abs(c.val.double().cpu().numpy() - ref.val) <= TOL["f32"] * ref.bound)
        d = dc[int(offs[i]):int(offs[i + 1])].double().cpu().numpy()
        ra, rb = oracle.backward(a32, b32, ref.row_ptr, ref.col, d)
        absb = I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, np.abs(b32.val))
        boa, _ = oracle.backward(I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, np.ones(a.nnz)), absb,
                                 ref.row_ptr, ref.col, np.abs(d))
        assert np.all(np.abs(ga[i].double().cpu().numpy() - ra) <= TOL["f32"] * boa + 1e-30)
        absa = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, np.abs(a32.val))
        _, bob = oracle.backward(absa, I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, np.ones(b.nnz)),
                                 ref.row_ptr, ref.col, np.abs(d))
        assert np.all(np.abs(gb[i].double().cpu().numpy() - rb) <= TOL["f32"] * bob + 1e-30)
