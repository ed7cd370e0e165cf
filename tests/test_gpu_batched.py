"""GPU parity of the batched form (many products in one launch per kernel),
its CUDA-graph replay, the autotuner and the batched backward."""
import numpy as np
import pytest

import oracle
import paper_1804_00695_gb300 as sg
from paper_1804_00695_gb300 import inputs as I
from gpu_helpers import assert_grads_match, assert_matches, oracle_product, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h(cuda_lib):
    return sg.Handle()


def make_batch(count=12, lo=64, hi=3000, seed=5, dtype=np.float32):
    pairs = I.random_batch(count, lo, hi, seed, dtype=np.float64)
    return pairs, [to_dev(a, dtype) for a, _ in pairs], [to_dev(b, dtype) for _, b in pairs]


@pytest.mark.parametrize("dtype,tag", [(np.float32, "f32"), (np.float64, "f64")])
def test_batched_matches_oracle_and_single(h, dtype, tag):
    pairs, As, Bs = make_batch(dtype=dtype)
    bt = sg.Batch(h, As, Bs)
    Cm = bt.run()
    h.check()
    parts = bt.split(Cm)
    single = sg.Handle()
    for (a, b), c, A, B in zip(pairs, parts, As, Bs):
        ref = oracle_product(a, b, dtype)
        assert_matches(c, ref, tag)
        one = single.spgemm(A, B)
        assert np.array_equal(one.row_ptr.cpu().numpy(), c.row_ptr.cpu().numpy())
        assert np.array_equal(one.col.cpu().numpy(), c.col.cpu().numpy())


def test_batched_graph_replay(h):
    import torch
    pairs, As, Bs = make_batch(count=6, seed=9)
    bt = sg.Batch(h, As, Bs)
    bt.symbolic()
    Cm = bt.alloc()
    bt.numeric_into(Cm)           # first call builds row lists outside the graph
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            bt.numeric_into(Cm)
    # new values in the same arrays, then replay
    for A in As:
        A.val.mul_(-2.0)
    g.replay()
    torch.cuda.synchronize()
    for (a, b), c in zip(pairs, bt.split(Cm)):
        a2 = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, (a.val.astype(np.float32) * -2.0).astype(np.float64))
        assert_matches(c, oracle_product(a2, b, np.float32), "f32")


def test_autotune_keeps_results(h):
    a, p, r = I.galerkin_problem(20)
    A, P = to_dev(a), to_dev(p)
    Cm = h.spgemm(A, P)
    choice, ms = h.autotune(reps=2)
    assert choice[0] in (8, 16, 32) and choice[1] in (16, 32) and choice[2] in (2, 4) and ms > 0
    assert_matches(Cm, oracle.spgemm(a, p), "f64")
    c2 = h.spgemm(A, P)
    assert_matches(c2, oracle.spgemm(a, p), "f64")
    for opt, v in ((sg.OPT_LANES_NUMERIC, 0), (sg.OPT_SMALL_CAP, 32), (sg.OPT_SLOT_FACTOR, 2)):
        h.set_option(opt, v)


def test_batched_backward(h):
    import torch
    pairs, As, Bs = make_batch(count=5, seed=13, dtype=np.float64)
    bt = sg.Batch(h, As, Bs)
    Cm = bt.run()
    dc = torch.linspace(-1, 1, Cm.nnz, dtype=torch.float64, device="cuda")
    da, db = bt.backward(Cm, dc)
    ga, gb = bt.split_grads(da, db)
    p0 = 0
    for (a, b), c, x, y in zip(pairs, bt.split(Cm), ga, gb):
        d = dc[p0:p0 + c.nnz].cpu().numpy()
        p0 += c.nnz
        assert_grads_match(a, b, c.row_ptr.cpu().numpy(), c.col.cpu().numpy(), d,
                           x.cpu().numpy(), y.cpu().numpy(), 1e-12)
