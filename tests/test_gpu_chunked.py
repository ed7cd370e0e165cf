"""GPU parity of the chunked product (Section 3.3.1, Algorithms 2-4) with
operands in host memory: the result equals the oracle (pattern exact, values
within tolerance) for budgets from "everything fits" down to many parts,
both loop orders run, and the bytes copied follow the copy-cost formulas."""
import numpy as np
import pytest

import oracle
import paper_1804_00695_gb300 as sg
from oracle import chunking as CH
from paper_1804_00695_gb300 import inputs as I
from gpu_helpers import TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h(cuda_lib):
    return sg.Handle()


def check(c, ref, tag):
    assert np.array_equal(c.row_ptr.numpy(), ref.row_ptr)
    assert np.array_equal(c.col.numpy(), ref.col)
    err = np.abs(c.val.double().numpy() - ref.val)
    assert np.all(err <= TOL[tag] * ref.bound)


def find_budget(a, c_rp, b, vb, alg, min_ac=1, min_b=1):
    """A budget whose Algorithm 4 plan uses `alg` with at least the given
    numbers of parts (searched on the CPU with the native planner)."""
    tot = sum(CH.range_bytes(x, 0, len(x) - 1, vb) for x in (a, c_rp, b))
    for frac in np.geomspace(3.0, 0.02, 160):
        f = int(tot * frac)
        try:
            p = sg.plan_chunks(a, c_rp, b, vb, f)
        except sg.SpgemmError:
            continue
        if p["algorithm"] == alg and len(p["p_ac"]) >= min_ac and len(p["p_b"]) >= min_b:
            return f, p
    return None, None


@pytest.mark.parametrize("dtype,tag", [(np.float64, "f64"), (np.float32, "f32")])
def test_chunked_everything_fits(h, dtype, tag):
    a, p, r = I.galerkin_problem(12)
    A, P = sg.HostCsr.from_numpy(a, dtype), sg.HostCsr.from_numpy(p, dtype)
    c = h.chunked(A, P, 1 << 28)
    ref = oracle.spgemm(I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, a.val.astype(dtype).astype(np.float64)),
                        I.Csr(p.nrows, p.ncols, p.row_ptr, p.col, p.val.astype(dtype).astype(np.float64)))
    check(c, ref, tag)
    st = h.chunked_stats()
    assert st["n_ac"] == 1 and st["n_b"] == 1


def expected_bytes(st, a, b, c_rp, nnz_c, vb=8):
    """Bytes Algorithm 3 copies for the plan the driver reports: B once, A
    and C offsets every pass, C entries in after the first pass and out every
    pass; each extra part boundary re-sends one 8-byte offset.  (The paper
    counts size(C)(|P_B|-1) for C; the copies out are counted here too.)"""
    nac, nb = st["n_ac"], st["n_b"]
    sa = CH.range_bytes(a.row_ptr, 0, a.nrows, vb)
    sb = CH.range_bytes(b.row_ptr, 0, b.nrows, vb)
    ent = nnz_c * (4 + vb)
    assert st["algorithm"] == 3   # Algorithm 2 bytes depend on skipped parts: formula test below
    h2d = (sb + 8 * (nb - 1)) + nb * (sa + 8 * (nac - 1)) + nb * (a.nrows + nac) * 8 + (nb - 1) * ent
    return h2d, nb * ent


def run_chunked(h, a, b, budget):
    ref = oracle.spgemm(a, b)
    A, B = sg.HostCsr.from_numpy(a), sg.HostCsr.from_numpy(b)
    rp, nnz = h.chunked_symbolic(A, B, max(budget, 1 << 22))
    assert np.array_equal(rp.numpy(), ref.row_ptr) and nnz == ref.nnz
    c = h.chunked_numeric(A, B, rp, nnz, budget)
    check(c, ref, "f64")
    return ref, h.chunked_stats()


def test_chunked_many_parts(h):
    """Random unsorted matrices, many parts on both sides."""
    a = I.random_csr(900, 700, 0.02, 71, shuffle_cols=True)
    b = I.random_csr(700, 800, 0.03, 72, shuffle_cols=True)
    ref = oracle.spgemm(a, b)
    budget, plan = find_budget(a.row_ptr, ref.row_ptr, b.row_ptr, 8, 2, 2, 2)
    assert budget is not None
    ref, st = run_chunked(h, a, b, budget)
    assert st["n_ac"] >= 2 and st["n_b"] >= 2


def test_chunked_alg3_b_larger(h):
    """B much larger than A and C: Algorithm 3 with several parts of B, so
    partial rows of C go out and come back in."""
    a = I.random_csr(200, 20000, 0.0005, 83, shuffle_cols=True)
    b = I.random_csr(20000, 300, 0.033, 84, shuffle_cols=True)
    ref = oracle.spgemm(a, b)
    # the driver re-plans on a smaller budget to double buffer, so try the
    # budgets for which the plain plan is Algorithm 3 until the driver's is
    tot = sum(CH.range_bytes(x, 0, len(x) - 1, 8) for x in (a.row_ptr, ref.row_ptr, b.row_ptr))
    hit = False
    for frac in np.geomspace(0.2, 0.04, 30):
        f = int(tot * frac)
        try:
            p = sg.plan_chunks(a.row_ptr, ref.row_ptr, b.row_ptr, 8, f)
        except sg.SpgemmError:
            continue
        if p["algorithm"] != 3 or len(p["p_b"]) < 2:
            continue
        try:
            ref, st = run_chunked(h, a, b, f)
        except sg.SpgemmError as e:
            assert e.status == 5
            continue
        if st["algorithm"] == 3 and st["n_b"] >= 2:
            h2d, d2h = expected_bytes(st, a, b, ref.row_ptr, ref.nnz)
            assert st["h2d_bytes"] == h2d and st["d2h_bytes"] == d2h
            hit = True
            break
    assert hit


def test_chunked_alg2_bytes_match_formula(h):
    """Algorithm 2 with every B part needed: bytes = size(A) + size(C) +
    size(B)|P_AC| (the paper's copy cost, on the parts the driver ran: it
    cuts A/C parts again to double buffer them and B parts finer to skip
    them precisely) plus 8 bytes per extra part boundary."""
    a0 = I.random_csr(1500, 400, 0.05, 91)
    # every row reaches the first and the last row of B, so no B part is skipped
    d = a0.to_dense() != 0
    d[:, 0] = d[:, -1] = True
    rows, cols = np.nonzero(d)
    rp = np.zeros(a0.nrows + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=a0.nrows), out=rp[1:])
    a = I.Csr(a0.nrows, a0.ncols, rp, cols.astype(np.int32),
              I.uniform01(np.arange(len(cols), dtype=np.uint64), 93) - 0.5)
    b = I.random_csr(400, 600, 0.04, 92)
    ref = oracle.spgemm(a, b)
    budget, plan = find_budget(a.row_ptr, ref.row_ptr, b.row_ptr, 8, 2, 2, 2)
    assert budget is not None
    ref, st = run_chunked(h, a, b, budget)
    assert st["algorithm"] == 2 and st["skipped_b_parts"] == 0
    nac, nb, nw = st["n_ac"], st["n_b"], st["b_windows"]
    sa = CH.range_bytes(a.row_ptr, 0, a.nrows, 8)
    sb = CH.range_bytes(b.row_ptr, 0, b.nrows, 8)
    sc = CH.range_bytes(ref.row_ptr, 0, a.nrows, 8)
    # parts of A whose rows of B came as one window (here all of B) copy B
    # whole; the others copy its fixed parts, re-sending one offset per boundary
    extra = 2 * 8 * (nac - 1) + 8 * (nb - 1) * (nac - nw)
    assert st["h2d_bytes"] + st["d2h_bytes"] == sa + sc + sb * nac + extra


def test_chunked_banded_skips_b_parts(h):
    """A banded operand (3D 27-point Laplacian): parts of B outside the A
    part's column range are skipped; the product is unchanged."""
    a = I.laplace3d_27pt(14)
    ref = oracle.spgemm(a, a)
    budget, plan = find_budget(a.row_ptr, ref.row_ptr, a.row_ptr, 8, 2, 3, 4)
    assert budget is not None
    ref, st = run_chunked(h, a, a, budget)
    assert st["algorithm"] == 2 and (st["skipped_b_parts"] > 0 or st["b_windows"] > 0)
    # fewer bytes of B than every part of A taking all of B
    sa = CH.range_bytes(a.row_ptr, 0, a.nrows, 8)
    sb = CH.range_bytes(a.row_ptr, 0, a.nrows, 8)
    sc = CH.range_bytes(ref.row_ptr, 0, a.nrows, 8)
    assert st["h2d_bytes"] + st["d2h_bytes"] < sa + sc + sb * st["n_ac"]


def test_chunked_numeric_recorded_and_measured_ranges(h):
    """The numeric call takes the rows of B that each part of A reaches from
    the row-block column ranges its symbolic call recorded; a handle without
    them measures each part's range on the device.  Same product both ways,
    and the recorded ranges (supersets) never copy fewer bytes of B."""
    a = I.laplace3d_27pt(20)
    ref = oracle.spgemm(a, a)
    A = sg.HostCsr.from_numpy(a)
    budget, plan = find_budget(a.row_ptr, ref.row_ptr, a.row_ptr, 8, 2, 3, 2)
    assert budget is not None
    rp, nnz = h.chunked_symbolic(A, A, max(budget, 1 << 22))
    c1 = h.chunked_numeric(A, A, rp, nnz, budget)
    st1 = h.chunked_stats()
    check(c1, ref, "f64")
    h2 = sg.Handle()
    c2 = h2.chunked_numeric(A, A, rp.clone().pin_memory(), nnz, budget)
    st2 = h2.chunked_stats()
    check(c2, ref, "f64")
    assert st1["n_ac"] == st2["n_ac"] >= 3
    assert st1["h2d_bytes"] >= st2["h2d_bytes"]


def test_chunked_numeric_flags_a_changed_after_symbolic(h):
    """Columns of A moved outside the ranges its symbolic call recorded (same
    host arrays) are caught by the window check: SPGEMM_ERR_NOT_SYMBOLIC."""
    a = I.laplace3d_27pt(20)
    ref = oracle.spgemm(a, a)
    A, B = sg.HostCsr.from_numpy(a), sg.HostCsr.from_numpy(a)
    rp, nnz = h.chunked_symbolic(A, B, 1 << 26)
    tot = sum(CH.range_bytes(x, 0, len(x) - 1, 8) for x in (a.row_ptr, ref.row_ptr, a.row_ptr))
    budget, seen = None, []
    for frac in np.geomspace(1.5, 0.1, 40):
        f = int(tot * frac)
        try:
            c = h.chunked_numeric(A, B, rp, nnz, f)
        except sg.SpgemmError as e:
            assert e.status == 5
            continue
        st = h.chunked_stats()
        seen.append((round(frac, 3), st["algorithm"], st["n_ac"], st["n_b"], st["b_windows"]))
        if st["algorithm"] == 2 and st["n_ac"] >= 2 and st["b_windows"] >= 1:
            check(c, ref, "f64")
            budget = f
            break
    assert budget is not None, seen
    # every 50th row reaches a column no part of its half reaches: the last
    # column of B (first half of the rows) or column 0 (second half); the
    # rows stay ascending
    col = A.col.numpy()
    for r in range(0, a.nrows, 50):
        if r < a.nrows // 2:
            col[int(a.row_ptr[r + 1]) - 1] = a.ncols - 1
        else:
            col[int(a.row_ptr[r])] = 0
    with pytest.raises(sg.SpgemmError) as ei:
        h.chunked_numeric(A, B, rp, nnz, budget)
    assert ei.value.status == 8


def test_chunked_one_call_with_allocator(h):
    """spgemm_chunked runs both phases with the caller's allocator for the
    entries of C; an allocator that fails gives SPGEMM_ERR_NOMEM."""
    import ctypes
    import torch
    a = I.laplace3d_27pt(10)
    ref = oracle.spgemm(a, a)
    A = sg.HostCsr.from_numpy(a)
    c = h.chunked(A, A, 1 << 22)
    check(c, ref, "f64")
    lib = sg.load()
    fail = sg.ALLOC_FN(lambda user, nnz, col_p, val_p: 1)
    rp = torch.empty(a.nrows + 1, dtype=torch.int64).pin_memory()
    dc = sg.CsrDesc(a.nrows, a.ncols, 0, rp.data_ptr(), None, None)
    da = A.desc()
    st = lib.spgemm_chunked(h._h, sg.F64, ctypes.byref(da), ctypes.byref(da), ctypes.byref(dc), fail, None,
                            1 << 22, torch.cuda.current_stream().cuda_stream)
    assert st == 4
    assert np.array_equal(rp.numpy(), ref.row_ptr)   # the symbolic phase ran


def test_chunked_budget_errors(h):
    a = I.random_csr(50, 40, 0.2, 95)
    A = sg.HostCsr.from_numpy(a)
    with pytest.raises(sg.SpgemmError) as ei:
        h.chunked(A, sg.HostCsr.from_numpy(I.random_csr(40, 30, 0.2, 96)), 512)
    assert ei.value.status == 5


def test_chunked_symbolic_compressed_and_fallbacks(h):
    """Chunked counts from the compressed pattern of B, with rows whose blocks
    overflow the per-warp map (bitmap path), and from the columns when B has
    unsorted rows; every count against the oracle."""
    nb, ncols = 600, 100000
    k = np.repeat(np.arange(nb), 10)
    t = np.tile(np.arange(10), nb)
    key = np.unique(k * ncols + (k * 7919 + t * 9973) % ncols)
    rp = np.zeros(nb + 1, dtype=np.int64)
    np.cumsum(np.bincount(key // ncols, minlength=nb), out=rp[1:])
    b = I.Csr(nb, ncols, rp, (key % ncols).astype(np.int32), np.ones(len(key)))
    d = I.random_csr(40, nb, 0.02, 97).to_dense() != 0
    d[0, :] = True                         # a row reaching every row of B: ~6000 blocks
    r, cidx = np.nonzero(d)
    arp = np.zeros(41, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=40), out=arp[1:])
    a = I.Csr(40, nb, arp, cidx.astype(np.int32), np.ones(len(cidx)))
    ref = oracle.spgemm(a, b)
    for bb in (b, I.random_csr(nb, 900, 0.05, 98, shuffle_cols=True)):
        ref = oracle.spgemm(a, bb)
        rp_c, nnz = h.chunked_symbolic(sg.HostCsr.from_numpy(a), sg.HostCsr.from_numpy(bb), 1 << 26)
        assert nnz == ref.nnz
        assert np.array_equal(rp_c.numpy(), ref.row_ptr)


def test_chunked_symbolic_tight_budget_recuts_a(h):
    """A budget that holds the pattern of B but not two of Algorithm 4's A
    parts: the parts of A are cut again, finer; counts still exact."""
    a = I.laplace3d_27pt(20)
    ref = oracle.spgemm(a, a)
    A = sg.HostCsr.from_numpy(a)
    raw_b = 8 * (a.nrows + 1) + 4 * a.nnz
    hit = False
    for budget in (int(raw_b * f) for f in (1.35, 1.45, 1.6, 1.8, 2.2)):
        try:
            rp, nnz = h.chunked_symbolic(A, A, budget)
        except sg.SpgemmError as e:
            assert e.status == 5
            continue
        assert nnz == ref.nnz and np.array_equal(rp.numpy(), ref.row_ptr)
        st = h.chunked_stats()
        assert st["device_bytes"] <= budget
        hit = hit or st["n_ac"] >= 3
    assert hit


def _with_bad_column(a, part_rows, col_value):
    """Copy of A whose rows in `part_rows` (a slice) all take column
    `col_value` in their first entry (rows keep their other entries)."""
    col = a.col.copy()
    for r in range(part_rows.start, part_rows.stop):
        if a.row_ptr[r + 1] > a.row_ptr[r]:
            col[int(a.row_ptr[r])] = col_value
    return I.Csr(a.nrows, a.ncols, a.row_ptr, col, a.val)


def test_chunked_numeric_bad_columns_without_recorded_ranges():
    """A fresh handle (no symbolic call, so no recorded ranges) measures each
    part's column range on the device: a column beyond the rows of B in a
    middle part, and a part whose every column is negative, both give
    SPGEMM_ERR_INDEX.  The same handle then multiplies correct operands, with
    the same budget and with another one (the arena freed and taken again
    after the error return), against the oracle."""
    a = I.laplace3d_27pt(20)
    ref = oracle.spgemm(a, a)
    budget, plan = find_budget(a.row_ptr, ref.row_ptr, a.row_ptr, 8, 2, 3, 2)
    assert budget is not None
    part = slice(*plan["p_ac"][len(plan["p_ac"]) // 2])
    import torch
    rp_host = torch.from_numpy(ref.row_ptr.copy()).pin_memory()
    B = sg.HostCsr.from_numpy(a)
    beyond = _with_bad_column(a, part, a.nrows + 5)
    col = a.col.copy()
    for r in range(part.start, part.stop):
        s0, s1 = int(a.row_ptr[r]), int(a.row_ptr[r + 1])
        col[s0:s1] = -1 - np.arange(s1 - s0)
    negative = I.Csr(a.nrows, a.ncols, a.row_ptr, col, a.val)
    for bad in (beyond, negative):
        h = sg.Handle()
        with pytest.raises(sg.SpgemmError) as ei:
            h.chunked_numeric(sg.HostCsr.from_numpy(bad), B, rp_host, ref.nnz, budget)
        assert ei.value.status == 3
        for bud in (budget, budget + (1 << 20)):
            c = h.chunked_numeric(sg.HostCsr.from_numpy(a), B, rp_host, ref.nnz, bud)
            check(c, ref, "f64")


@pytest.fixture()
def h3(cuda_lib):
    """A handle whose chunked calls triple buffer (SPGEMM_OPT_CHUNK_BUFFERS = 3)."""
    hh = sg.Handle()
    hh.set_option(sg.OPT_CHUNK_BUFFERS, 3)
    return hh


def test_chunked_triple_buffering_many_parts(h3):
    """Triple buffering (the budget in three segments per streamed operand,
    the closing discussion of Section 4): the same product as the oracle on
    random unsorted operands cut into many parts on both sides, with at
    least four A/C parts so that every buffer is used and reused."""
    a = I.random_csr(900, 700, 0.02, 171, shuffle_cols=True)
    b = I.random_csr(700, 800, 0.03, 172, shuffle_cols=True)
    ref = oracle.spgemm(a, b)
    budget, plan = find_budget(a.row_ptr, ref.row_ptr, b.row_ptr, 8, 2, 2, 2)
    assert budget is not None
    ref, st = run_chunked(h3, a, b, budget)
    assert st["algorithm"] == 2 and st["n_ac"] >= 4 and st["n_b"] >= 2


@pytest.mark.parametrize("fresh", [False, True])
def test_chunked_triple_buffering_banded(h3, fresh):
    """Banded operand, B windows in three buffers; with recorded column
    ranges (symbolic call first) and measured ones (fresh handle)."""
    a = I.laplace3d_27pt(20)
    ref = oracle.spgemm(a, a)
    A = sg.HostCsr.from_numpy(a)
    budget, plan = find_budget(a.row_ptr, ref.row_ptr, a.row_ptr, 8, 2, 3, 2)
    assert budget is not None
    if fresh:
        hh = sg.Handle()
        hh.set_option(sg.OPT_CHUNK_BUFFERS, 3)
        import torch
        c = hh.chunked_numeric(A, A, torch.from_numpy(ref.row_ptr.copy()).pin_memory(), ref.nnz, budget)
        st = hh.chunked_stats()
    else:
        rp, nnz = h3.chunked_symbolic(A, A, max(budget, 1 << 22))
        c = h3.chunked_numeric(A, A, rp, nnz, budget)
        st = h3.chunked_stats()
    check(c, ref, "f64")
    assert st["algorithm"] == 2 and st["n_ac"] >= 4 and st["device_bytes"] <= budget


def test_chunked_triple_buffering_alg3_bytes(h3):
    """Algorithm 3 (B outer, several parts) with three A/C buffers: partial
    rows of C go out and come back in across the buffers; the product equals
    the oracle and the bytes copied follow the same formula as with two."""
    a = I.random_csr(200, 20000, 0.0005, 83, shuffle_cols=True)
    b = I.random_csr(20000, 300, 0.033, 84, shuffle_cols=True)
    ref = oracle.spgemm(a, b)
    tot = sum(CH.range_bytes(x, 0, len(x) - 1, 8) for x in (a.row_ptr, ref.row_ptr, b.row_ptr))
    hit = False
    for frac in np.geomspace(0.2, 0.04, 30):
        f = int(tot * frac)
        try:
            p = sg.plan_chunks(a.row_ptr, ref.row_ptr, b.row_ptr, 8, f)
        except sg.SpgemmError:
            continue
        if p["algorithm"] != 3 or len(p["p_b"]) < 2:
            continue
        try:
            ref, st = run_chunked(h3, a, b, f)
        except sg.SpgemmError as e:
            assert e.status == 5
            continue
        if st["algorithm"] == 3 and st["n_b"] >= 2:
            h2d, d2h = expected_bytes(st, a, b, ref.row_ptr, ref.nnz)
            assert st["h2d_bytes"] == h2d and st["d2h_bytes"] == d2h
            hit = True
            break
    assert hit


def test_chunked_buffers_option_values(cuda_lib):
    hh = sg.Handle()
    for v in (2, 3):
        hh.set_option(sg.OPT_CHUNK_BUFFERS, v)
    for v in (0, 1, 4):
        with pytest.raises(sg.SpgemmError) as ei:
            hh.set_option(sg.OPT_CHUNK_BUFFERS, v)
        assert ei.value.status == 1
