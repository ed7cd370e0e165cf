"""Benchmark workloads besides the default Galerkin product; each measure_*
function returns a dict that bench.py puts under "secondary" in its default
line, and ``python bench.py --workload rmat20|triangles20|chunked256|batched256`` prints
one of them as a full line.

* rmat20     - C = A*A, A symmetrised R-MAT scale 20, edge factor 16, FP32.
* triangles20 - triangles of the same graph by the masked product L*L .* L.
* chunked256 - C = A*A, A the 27-point Laplacian on 256^3, FP64, operands and
               result in pinned host memory, 4 GB device budget (Section 3.3.1).
* placement128 - the Galerkin products with A, B, C each in HBM, pinned host
               or managed memory (the placements of Table 3).
* families   - R*A and A*P of the 7-point, 13-point, 27-point and elasticity
               multigrid families (Section 4's input families).
* density    - Elasticity's R and A times random right-hand sides with
               delta = 1, 4, 16, 64, 256 entries per row (Table 2).
* weak27     - (own line only) R*A and A*P of the 27-point family with A of
               about 1, 2, 4 and 8 GB.
* budget256  - (own line only) the chunked workload at device budgets 4-64 GB.
* batched256 - 256 products A_i*B_i, rows log-uniform in [1024, 65536], 4-32
               random columns per row, FP32: batched forward and backward
               against a per-instance loop on the same GPU.

Every entry carries a CPU baseline: the oracle timed on a bounded sample of
the same workload (rows of C, or instances), on all host cores; the same
oracle output is compared with the device result for that sample (pattern
exact, values within the stated tolerance), reported as "parity".
The large inputs are generated in a process pool (spawn) that bench.py starts
before its first CUDA call.
"""
from __future__ import annotations

import concurrent.futures as cf
import json
import multiprocessing as mp
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import bench  # noqa: E402  (shared helpers: clocks, peaks, bytes)

TOL = {"f64": 1e-12, "f32": 1e-5}
CPU_SAMPLE_S = 4.0   # target seconds of oracle work per CPU-baseline sample


# ---------------------------------------------------------------- inputs
def _gen_rmat(scale):
    from paper_1804_00695_gb300 import inputs as I
    return I.rmat_symmetric(scale, 16, seed=1)


def _gen_pair(n, s):
    from paper_1804_00695_gb300 import inputs as I
    return I.random_square(n, 2 * s, dtype=np.float32), I.random_square(n, 2 * s + 1, dtype=np.float32)


def _gen_family(name, n):
    from paper_1804_00695_gb300 import inputs as I
    return I.family_problem(name, n)


def _gen_density(n, deltas):
    """Elasticity's A and R on an n^3 grid and a random right-hand side per
    delta (seed 100 + delta), for the density experiment."""
    from paper_1804_00695_gb300 import inputs as I
    a, _, r = I.family_problem("elasticity3d_81", n)
    return a, r, {d: I.random_rhs(a.ncols, a.ncols, d, seed=100 + d) for d in deltas}


# the multigrid families at about 0.6-0.75 GB of A each (the 27-point one is
# the default workload's problem)
FAMILY_SIZES = {"laplace3d_7pt": 200, "bigstar2d_13pt": 2000, "elasticity3d_81": 64}
# 27-point A of about 1, 2, 4 and 8 GB (324 bytes per interior row)
WEAK_SIZES = (146, 184, 231, 291)
# density experiment (Table 2): Elasticity on 24^3 (41,472 rows) times random
# right-hand sides with delta entries per row; at delta = 256 A*RHS has
# 0.86e9 multiplications and 0.68e9 entries (8 GB in FP64)
DENSITY_GRID = 24
DENSITY_DELTAS = (1, 4, 16, 64, 256)


class Inputs:
    """The secondary workloads' inputs, generated in worker processes (spawn)
    while the caller measures: the R-MAT graph, the batch instances
    (instance i: n_i from the log-uniform sizes, seeds 2(1+i), 2(1+i)+1, as
    inputs.random_batch) and the multigrid families."""

    def __init__(self, args, workers=None, families=True):
        from paper_1804_00695_gb300 import inputs as I
        workers = workers or max(1, min(16, (os.cpu_count() or 2) - 1))
        self.pool = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
        self.fam = {k: self.pool.submit(_gen_family, k, n) for k, n in FAMILY_SIZES.items()} if families else {}
        self.dens = self.pool.submit(_gen_density, DENSITY_GRID, DENSITY_DELTAS) if families else None
        self.rmat = self.pool.submit(_gen_rmat, args.rmat_scale)
        sizes = I.batch_sizes(args.batch_count, 1024, args.batch_max, 1)
        self.batch = [self.pool.submit(_gen_pair, n, 1 + i) for i, n in enumerate(sizes)]

    def rmat_graph(self):
        return self.rmat.result()

    def batch_pairs(self):
        return [f.result() for f in self.batch]

    def families(self):
        return {k: f.result() for k, f in self.fam.items()}

    def density(self):
        return self.dens.result()

    def close(self):
        self.pool.shutdown(wait=False, cancel_futures=True)


# ---------------------------------------------------------------- helpers
def _mults(a, b_rp):
    return int(np.diff(b_rp)[a.col.astype(np.int64)].sum())


def _row_flops(a, b):
    """Multiplications per row of A*B (sum over stored a_ik of nnz(B_k))."""
    rows = np.repeat(np.arange(a.nrows), np.diff(a.row_ptr))
    per = np.diff(b.row_ptr)[a.col.astype(np.int64)].astype(np.float64)
    return np.rint(np.bincount(rows, weights=per, minlength=a.nrows)).astype(np.int64)


def _hbm_peak():
    peaks = bench.measured_peaks()
    return (peaks["hbm_gbs"], "measured") if peaks else (6800.0, "fallback")


def _compare_rows(got_rp, got_col, got_val, ref, tol):
    """Device rows (host copies) against an oracle Result of the same rows:
    pattern exact, values within tol * sum|a||b| (exact where that is 0)."""
    got_rp = got_rp - got_rp[0]
    ok_pat = np.array_equal(got_rp, ref.row_ptr) and np.array_equal(got_col, ref.col)
    err = np.abs(got_val.astype(np.float64) - ref.val) if ok_pat else None
    ok_val = bool(ok_pat and np.all(err <= tol * ref.bound))
    worst = float(np.max(err / np.maximum(ref.bound, 1e-300))) if ok_pat and len(err) else 0.0
    return {"pattern_exact": bool(ok_pat), "values_in_tolerance": ok_val, "max_err_over_bound": worst}


def _row_block(fl, target_mults, start):
    """Rows [start, end) whose products add up to about target_mults."""
    cum = np.cumsum(fl[start:])
    end = start + int(np.searchsorted(cum, target_mults)) + 1
    return start, min(end, len(fl))


def _oracle_rows_sample(a, b, fl, start, tol_tag, device_rows, label, seconds=CPU_SAMPLE_S, probe_mults=2e8,
                        keep=None):
    """CPU baseline leg: the oracle on a block of rows of about `seconds`
    seconds (grown from a small probe), timed on all host cores; its output
    is compared with the device rows (device_rows(r0, r1) -> rp, col, val).
    `keep` (a dict), if given, receives the oracle rows for later checks."""
    import oracle
    r0, r1 = _row_block(fl, probe_mults, start)
    t0 = time.perf_counter()
    oracle.spgemm(a, b, r0, r1)
    probe = max(time.perf_counter() - t0, 1e-3)
    rate = max(int(fl[r0:r1].sum()), 1) / probe
    r0, r1 = _row_block(fl, rate * seconds, start)
    t0 = time.perf_counter()
    ref = oracle.spgemm(a, b, r0, r1)
    dt = time.perf_counter() - t0
    m = int(fl[r0:r1].sum())
    par = _compare_rows(*device_rows(r0, r1), ref, TOL[tol_tag])
    par["rows"] = [int(r0), int(r1)]
    if keep is not None:
        keep.update(ref=ref, r0=r0, r1=r1)
    return ({"value": 2 * m / dt / 1e9, "unit": "GFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
             "sample": f"{label}: rows [{r0}, {r1}) of C ({m} multiplications), {dt:.2f} s"}, par)


# ---------------------------------------------------------------- R-MAT
def measure_rmat(args, g, local):
    """C = A*A on the R-MAT graph: GFLOP/s, % of the HBM-byte roofline, the
    dominant kernel's roofline, a CPU baseline on a block of rows and the
    parity of that block."""
    import torch
    import paper_1804_00695_gb300 as sg
    A = sg.Csr.from_host(g, "cuda", np.float32)
    h = sg.Handle(local)
    mults = _mults(g, g.row_ptr)
    fl = _row_flops(g, g)
    stream = torch.cuda.current_stream()
    steps, warm = 2, 2
    c = h.spgemm(A, A)
    h.check()
    crp = c.row_ptr.cpu().numpy()
    nnz = c.nnz

    def rows(r0, r1):
        p0, p1 = int(crp[r0]), int(crp[r1])
        return crp[r0:r1 + 1].copy(), c.col[p0:p1].cpu().numpy(), c.val[p0:p1].cpu().numpy()

    # sample rows where the degrees are mixed (away from the hub at row 0)
    cpu, par = _oracle_rows_sample(g, g, fl, g.nrows // 3, "f32", rows, "R-MAT scale %d" % args.rmat_scale)
    del c
    for _ in range(warm - 1):
        del_c = h.spgemm(A, A)
        del del_c
    h.set_timing(True)
    h.reset_timings()
    clocks = bench.ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        c = h.spgemm(A, A)
        del c
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    tim = h.timings()
    h.set_timing(False)
    hbm, src = _hbm_peak()
    step_bytes = bench.kernel_bytes(g, g.row_ptr, crp, np.ones(g.nrows, dtype=bool), 4)
    nar = bench.narrow_numeric_rows(g, g, crp, fl)
    bb = np.where(nar, 7, bench.bins_of(np.diff(crp), fl))
    kern = []
    for key, (nl, nrows, tms) in tim.items():
        parts = key.split(".")
        if parts[0] != "numeric":
            continue
        lab = parts[1]
        if lab == "narrow":
            mask = nar
        elif lab == "small":
            mask = (bb == 1) | (bb == 2)
        elif lab.startswith("bin"):
            mask = bb == int(lab[3:4])
        else:
            continue
        kern.append((tms / nl, key, bench.kernel_bytes(g, g.row_ptr, crp, mask, 4, True), nl))
    roof = None
    if kern:
        per_ms, key, byt, nl = max(kern, key=lambda x: x[0] * x[3])
        ach = byt / (per_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "kernel": key, "bytes_per_launch": byt, "ms_per_launch": per_ms,
                "peak_source": src}
    return {"metric_value": 2 * mults / (ms / 1e3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms, "steps": steps,
            "warmup": warm, "dtype": "f32",
            "config": {"workload": f"C = A*A, A symmetrised R-MAT scale {args.rmat_scale}, edge factor 16, "
                                   "(a,b,c,d) = (.57,.19,.19,.05), seed 1, FP32", "mults": mults, "nnz_C": nnz},
            "pct_hbm_byte_roofline": 100 * step_bytes / (ms / 1e3) / 1e9 / hbm,
            "step_algorithmic_bytes": step_bytes, "roofline": roof,
            "kernels_ms_per_step": {k: v[2] / steps for k, v in sorted(tim.items())},
            "gpu_launches": sum(v[0] for v in tim.values()), "clocks": clk, "cpu_baseline": cpu,
            "parity": par}


# ---------------------------------------------------------------- triangles
def measure_triangles(args, g, local):
    """Triangle counting by the masked product L*L .* L on the R-MAT graph
    (the paper's triangle-counting experiment): time per count, the
    masked product's multiplications (sum over stored L_ik of nnz(L_k), from
    the library's own labels), a CPU baseline (the oracle on the whole graph)
    and the parity of the count."""
    import torch
    import oracle
    import paper_1804_00695_gb300 as sg
    G = sg.Csr.from_host(g, "cuda", np.float32)
    h = sg.Handle(local)
    total, perm, _ = h.triangles(G, labels=True)
    perm = perm.cpu().numpy()
    rows = np.repeat(np.arange(g.nrows), np.diff(g.row_ptr))
    pr, pc = perm[rows], perm[g.col.astype(np.int64)]
    low = pc < pr
    llen = np.bincount(pr[low], minlength=g.nrows)
    lmults = int(llen[pc[low]].sum())
    steps, warm = 10, 3
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        h.triangles(G)
    h.set_timing(True)
    h.reset_timings()
    clocks = bench.ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        h.triangles(G)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    tim = h.timings()
    h.set_timing(False)
    t0 = time.perf_counter()
    ref, _ = oracle.triangles(g)
    dt = time.perf_counter() - t0
    return {"metric_value": 2 * lmults / (ms / 1e3) / 1e9, "unit": "GFLOP/s (2 x masked-product multiplications/s)",
            "ms_per_step": ms, "steps": steps, "warmup": warm, "dtype": "int (pattern only)",
            "config": {"workload": f"triangles of the R-MAT scale {args.rmat_scale} graph (edge factor 16) by "
                                   "L*L .* L, L the degree-ordered lower triangle", "triangles": total,
                       "edges": int(g.nnz // 2), "nnz_L": int(low.sum()), "masked_product_mults": lmults},
            "triangles_per_s": total / (ms / 1e3), "edges_per_s": (g.nnz // 2) / (ms / 1e3),
            "kernels_ms_per_step": {k: v[2] / steps for k, v in sorted(tim.items())}, "clocks": clk,
            "cpu_baseline": {"value": 2 * lmults / dt / 1e9, "unit": "GFLOP/s (2 x masked-product multiplications/s)",
                             "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"the whole graph, sorted-row merges, {dt:.2f} s"},
            "parity": {"count_exact": total == ref, "oracle_count": ref}}


# ---------------------------------------------------------------- chunked
def _link_bandwidth():
    import torch
    n = 1 << 30
    hbuf = torch.empty(n, dtype=torch.uint8).pin_memory()
    dbuf = torch.empty(n, dtype=torch.uint8, device="cuda")
    h2 = torch.empty(n, dtype=torch.uint8).pin_memory()
    d2 = torch.empty(n, dtype=torch.uint8, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    out = {}
    for name, fn in (("h2d", lambda: dbuf.copy_(hbuf, non_blocking=True)),
                     ("d2h", lambda: hbuf.copy_(dbuf, non_blocking=True))):
        ts = []
        for _ in range(5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(s1):
                fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        out[name] = n / statistics.median(ts) / 1e9
    ts = []
    for _ in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s1):
            dbuf.copy_(hbuf, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    out["bidir"] = 2 * n / statistics.median(ts) / 1e9
    return out


def measure_chunked(args, local, a=None, triple_buffers=True):
    """Chunked C = A*A with operands and C in pinned host memory and a device
    budget: algorithmic GFLOP/s including every copy (symbolic + numeric),
    the fraction of the measured host link, bytes copied against the minimal
    bytes, the plan, a CPU baseline on a block of rows and its parity."""
    import torch
    import paper_1804_00695_gb300 as sg
    from paper_1804_00695_gb300 import inputs as I
    n = args.chunk_grid
    if a is None:
        a = I.laplace3d_27pt(n)
    A = sg.HostCsr.from_numpy(a)
    budget = int(args.budget)
    h = sg.Handle(local)
    mults = _mults(a, a.row_ptr)
    link = _link_bandwidth()
    steps = 2
    rp, nnz = h.chunked_symbolic(A, A, budget)
    col = torch.empty(nnz, dtype=torch.int32).pin_memory()
    val = torch.empty(nnz, dtype=torch.float64).pin_memory()
    Cm = sg.HostCsr(a.nrows, a.ncols, rp, col, val)
    clocks = bench.ClockSampler(local)
    times, sym_times, stats, sym = [], [], None, None
    clocks.start()
    for it in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, nnz2 = h.chunked_symbolic(A, A, budget, out=Cm.row_ptr)
        t1 = time.perf_counter()
        sym = h.chunked_stats()
        assert nnz2 == nnz
        h.chunked_numeric_into(A, A, Cm, budget)
        dt = time.perf_counter() - t0
        stats = h.chunked_stats()
        if it > 0:
            times.append(dt)
            sym_times.append(t1 - t0)
    clk = clocks.stop()
    ms = 1e3 * statistics.median(times)
    size_a = 8 * (a.nrows + 1) + 12 * a.nnz
    size_c = 8 * (a.nrows + 1) + 12 * nnz
    minimal = 2 * size_a + size_c            # A and B in, C out, each once
    moved = stats["h2d_bytes"] + stats["d2h_bytes"] + sym["h2d_bytes"] + sym["d2h_bytes"]
    peak = max(link["bidir"], link["h2d"], link["d2h"])
    fl = _row_flops(a, a)
    crp = Cm.row_ptr.numpy()

    def rows(r0, r1):
        p0, p1 = int(crp[r0]), int(crp[r1])
        return crp[r0:r1 + 1].copy(), Cm.col[p0:p1].numpy(), Cm.val[p0:p1].numpy()

    kept = {}
    cpu, par = _oracle_rows_sample(a, a, fl, a.nrows // 2, "f64", rows, f"27-point {n}^3 A*A", keep=kept)
    triple = None
    if triple_buffers:
        # the same step with every streamed operand in three buffers (the
        # closing discussion of Section 4), into the same C arrays
        h.set_option(sg.OPT_CHUNK_BUFFERS, 3)
        t3, st3 = [], None
        clocks.start()
        for it in range(steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.chunked_symbolic(A, A, budget, out=Cm.row_ptr)
            h.chunked_numeric_into(A, A, Cm, budget)
            dt = time.perf_counter() - t0
            st3 = h.chunked_stats()
            if it > 0:
                t3.append(dt)
        clk3 = clocks.stop()
        h.set_option(sg.OPT_CHUNK_BUFFERS, 2)
        ms3 = 1e3 * statistics.median(t3)
        p3 = _compare_rows(*rows(kept["r0"], kept["r1"]), kept["ref"], TOL["f64"])
        triple = {"ms": ms3, "gflops": 2 * mults / (ms3 / 1e3) / 1e9,
                  "link_frac": minimal / (ms3 / 1e3) / 1e9 / peak,
                  "bytes_copied_over_minimal": (st3["h2d_bytes"] + st3["d2h_bytes"] + sym["h2d_bytes"]
                                                + sym["d2h_bytes"]) / minimal,
                  "numeric_plan": st3, "parity": p3, "vs_double": ms / ms3, "clocks": clk3}
    return {"metric_value": 2 * mults / (ms / 1e3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms, "steps": steps,
            "warmup": 1, "dtype": "f64",
            "config": {"workload": f"chunked C = A*A, 27-point 3D Laplacian on {n}^3, FP64, operands and C in "
                                   f"pinned host memory, {budget:.3g}-byte device budget", "mults": mults,
                       "nnz_C": nnz, "budget_bytes": budget},
            "roofline": {"bound": "host-link", "achieved": minimal / (ms / 1e3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": minimal / (ms / 1e3) / 1e9 / peak, "traffic": moved,
                         "note": "achieved = minimal bytes (A, B in and C out once) over the step time; "
                                 "peak = the best of the pinned H2D, D2H and both-ways copies measured in "
                                 "the same run; traffic = bytes actually copied (symbolic + numeric)"},
            "bytes_copied_over_minimal": moved / minimal, "link_gbs_measured": link, "numeric_plan": stats,
            "symbolic_plan": sym, "symbolic_ms": 1e3 * statistics.median(sym_times), "clocks": clk,
            "cpu_baseline": cpu, "parity": par, "triple_buffering": triple}


# ---------------------------------------------------------------- batched
def _grad_check(a, b, c_rp, c_col, dc, da, db, tol):
    """Oracle gradients of <dC, A*B> for one instance, and the device ones
    against them (each entry within tol * the sum of the absolute terms it
    adds)."""
    import oracle
    from paper_1804_00695_gb300 import inputs as I
    a64 = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, a.val.astype(np.float64))
    b64 = I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, b.val.astype(np.float64))
    dc64 = dc.astype(np.float64)
    ra, rb = oracle.backward(a64, b64, c_rp, c_col, dc64)
    ones_a = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, np.ones(a.nnz))
    ones_b = I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, np.ones(b.nnz))
    abs_a = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, np.abs(a64.val))
    abs_b = I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, np.abs(b64.val))
    ba, _ = oracle.backward(ones_a, abs_b, c_rp, c_col, np.abs(dc64))
    _, bb = oracle.backward(abs_a, ones_b, c_rp, c_col, np.abs(dc64))
    return bool(np.all(np.abs(da - ra) <= tol * ba) and np.all(np.abs(db - rb) <= tol * bb))


def measure_batched(args, pairs, local):
    """Batched forward and backward against a per-instance loop on the same
    GPU (speedups), a CPU baseline on a sample of instances and the parity of
    that sample (forward and backward)."""
    import torch
    import oracle
    import paper_1804_00695_gb300 as sg
    from paper_1804_00695_gb300 import inputs as I
    As = [sg.Csr.from_host(a, "cuda") for a, _ in pairs]
    Bs = [sg.Csr.from_host(b, "cuda") for _, b in pairs]
    mults = sum(_mults(a, b.row_ptr) for a, b in pairs)
    h = sg.Handle(local)
    hl = sg.Handle(local)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    steps, warm = 5, 2

    def timed(fn, reps):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    clocks = bench.ClockSampler(local)
    clocks.start()
    bt = sg.Batch(h, As, Bs)
    fwd_batched = timed(lambda: bt.run(), steps)
    loop_out = []

    def loop_fwd():
        loop_out.clear()
        for A, B in zip(As, Bs):
            loop_out.append(hl.spgemm(A, B))
    fwd_loop = timed(loop_fwd, 2)
    bt.symbolic()
    Cm = bt.alloc()
    bt.numeric_into(Cm)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            bt.numeric_into(Cm)
    num_graph = timed(lambda: g.replay(), steps)
    singles = []
    for A, B in zip(As, Bs):
        hh = sg.Handle(local)
        rp, nz = hh.symbolic(A, B)
        singles.append((hh, A, B, hh.numeric(A, B, rp, nz)))
    num_loop = timed(lambda: [hh.numeric_into(A, B, c) for hh, A, B, c in singles], steps)
    dc = torch.cos(torch.arange(Cm.nnz, device="cuda", dtype=torch.float32))
    bwd_batched = timed(lambda: bt.backward(Cm, dc), steps)
    parts = bt.split(Cm)
    dcs = []
    p0 = 0
    for c in parts:
        dcs.append(dc[p0:p0 + c.nnz])
        p0 += c.nnz
    bwd_loop = timed(lambda: [hh.backward(A, B, c, d) for (hh, A, B, c), d in zip(singles, dcs)], 2)
    clk = clocks.stop()
    # CPU baseline leg: the oracle forward on instances in order until about
    # CPU_SAMPLE_S seconds; the same outputs (and the oracle backward of the
    # first sampled instance) against the device results
    da, db = bt.backward(Cm, dc)
    ga, gb = bt.split_grads(da, db)
    t_cpu, m_cpu, done, par_ok = 0.0, 0, [], True
    k = len(pairs) // 2
    while k < len(pairs) and t_cpu < CPU_SAMPLE_S:
        a, b = pairs[k]
        a64 = I.Csr(a.nrows, a.ncols, a.row_ptr, a.col, a.val.astype(np.float64))
        b64 = I.Csr(b.nrows, b.ncols, b.row_ptr, b.col, b.val.astype(np.float64))
        t0 = time.perf_counter()
        ref = oracle.spgemm(a64, b64)
        t_cpu += time.perf_counter() - t0
        m_cpu += int(ref.mults.sum())
        c = parts[k]
        r = _compare_rows(c.row_ptr.cpu().numpy(), c.col.cpu().numpy(), c.val.cpu().numpy(), ref, TOL["f32"])
        par_ok = par_ok and r["pattern_exact"] and r["values_in_tolerance"]
        done.append(k)
        k += 1
    i0 = done[0]
    c0 = parts[i0]
    bwd_ok = _grad_check(pairs[i0][0], pairs[i0][1], c0.row_ptr.cpu().numpy(), c0.col.cpu().numpy(),
                         dcs[i0].cpu().numpy(), ga[i0].double().cpu().numpy(), gb[i0].double().cpu().numpy(),
                         TOL["f32"])
    gf = lambda ms: 2 * mults / (ms / 1e3) / 1e9
    return {"metric_value": gf(fwd_batched), "unit": "GFLOP/s", "ms_per_step": fwd_batched, "steps": steps,
            "warmup": warm, "dtype": "f32",
            "config": {"workload": f"{args.batch_count} products A_i*B_i, n_i log-uniform in [1024, "
                                   f"{args.batch_max}], 4-32 random columns per row, N(0,1) FP32",
                       "mults": mults, "nnz_C": int(Cm.nnz), "rows": int(sum(a.nrows for a, _ in pairs))},
            "batched_forward_ms": fwd_batched, "loop_forward_ms": fwd_loop,
            "forward_speedup": fwd_loop / fwd_batched,
            "batched_numeric_graph_ms": num_graph, "loop_numeric_ms": num_loop,
            "numeric_speedup": num_loop / num_graph,
            "batched_backward_ms": bwd_batched, "loop_backward_ms": bwd_loop,
            "backward_speedup": bwd_loop / bwd_batched, "loop_forward_gflops": gf(fwd_loop), "clocks": clk,
            "cpu_baseline": {"value": 2 * m_cpu / t_cpu / 1e9, "unit": "GFLOP/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"forward of instances {done[0]}..{done[-1]} ({m_cpu} multiplications), "
                                       f"{t_cpu:.2f} s"},
            "parity": {"instances": [done[0], done[-1]], "forward_pattern_exact_and_in_tolerance": bool(par_ok),
                       "backward_instance": i0, "backward_in_tolerance": bwd_ok}}


# ---------------------------------------------------------------- multigrid families
def _time_product(h, X, Y, warm, steps, stream):
    """Median ms of symbolic + numeric (C allocated by the caching allocator
    as in the default step), CUDA events on the launching stream."""
    import torch
    ms = []
    for it in range(warm + steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        c = h.spgemm(X, Y)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        del c
    return statistics.median(ms[warm:])


def _product_entry(h, x, y, label, local, warm=2, steps=3, cpu_seconds=1.0):
    """One product of a family: GFLOP/s, % of the HBM-byte roofline of the
    whole product (symbolic + numeric bytes), an oracle CPU baseline on a
    block of rows and the parity of that block."""
    import torch
    import paper_1804_00695_gb300 as sg
    X, Y = sg.Csr.from_host(x, "cuda"), sg.Csr.from_host(y, "cuda")
    stream = torch.cuda.current_stream()
    c = h.spgemm(X, Y)
    h.check()
    crp = c.row_ptr.cpu().numpy()

    def rows(r0, r1):
        p0, p1 = int(crp[r0]), int(crp[r1])
        return crp[r0:r1 + 1].copy(), c.col[p0:p1].cpu().numpy(), c.val[p0:p1].cpu().numpy()

    fl = _row_flops(x, y)
    cpu, par = _oracle_rows_sample(x, y, fl, x.nrows // 2, "f64", rows, label, seconds=cpu_seconds,
                                   probe_mults=2e7)
    nnz = c.nnz
    del c
    ms = _time_product(h, X, Y, warm, steps, stream)
    mults = int(fl.sum())
    allrows = np.ones(x.nrows, dtype=bool)
    byt = (bench.kernel_bytes(x, y.row_ptr, crp, allrows, 8, True)
           + bench.kernel_bytes(x, y.row_ptr, crp, allrows, 8, False))
    hbm, src = _hbm_peak()
    del X, Y
    torch.cuda.empty_cache()
    return {"ms": ms, "gflops": 2 * mults / (ms / 1e3) / 1e9, "mults": mults, "nnz_C": nnz,
            "rows": x.nrows, "pct_hbm_byte_roofline": 100 * byt / (ms / 1e3) / 1e9 / hbm,
            "algorithmic_bytes": byt, "peak_source": src, "cpu_baseline": cpu, "parity": par}


def measure_families(args, problems, local):
    """R*A and A*P of every multigrid family (Section 4's input families),
    reported separately as in the paper; problems: name -> (A, P, R)."""
    import paper_1804_00695_gb300 as sg
    h = sg.Handle(local)
    clocks = bench.ClockSampler(local)
    clocks.start()
    out = {}
    for name, (a, p, r) in problems.items():
        n = FAMILY_SIZES.get(name, args.grid)
        out[name] = {"grid": n, "A_rows": a.nrows, "A_nnz": a.nnz, "A_gb": (8 * (a.nrows + 1) + 12 * a.nnz) / 1e9,
                     "P_nnz": p.nnz,
                     "R*A": _product_entry(h, r, a, f"{name} R*A", local),
                     "A*P": _product_entry(h, a, p, f"{name} A*P", local)}
    clk = clocks.stop()
    ok = all(v[k]["parity"]["pattern_exact"] and v[k]["parity"]["values_in_tolerance"]
             for v in out.values() for k in ("R*A", "A*P"))
    return {"config": {"workload": "R*A and A*P of the multigrid families: 7-point 3D Laplacian, 13-point 2D "
                                   "biharmonic star, 27-point 3D brick, 3D elasticity (81 per row); smoothed "
                                   "aggregation P (3 points per dimension, omega 2/3), FP64",
                       "steps": 3, "warmup": 2},
            "families": out, "clocks": clk, "parity": {"all_rows_sampled_match": ok}}


def measure_density(args, problem, local):
    """The right-hand-side density experiment of Section 4 (Table 2):
    Elasticity's R and A times random right-hand sides with delta entries per
    row, GFLOP/s and % of the HBM-byte roofline per delta (the paper lists
    GFLOP/s and cache miss ratios on its two memories)."""
    import paper_1804_00695_gb300 as sg
    a, r, rhs = problem
    h = sg.Handle(local)
    clocks = bench.ClockSampler(local)
    clocks.start()
    rows = {}
    for d, y in sorted(rhs.items()):
        rows[str(d)] = {"R*RHS": _product_entry(h, r, y, f"elasticity R*RHS delta {d}", local, cpu_seconds=0.5),
                        "A*RHS": _product_entry(h, a, y, f"elasticity A*RHS delta {d}", local, cpu_seconds=0.5)}
    clk = clocks.stop()
    ok = all(v[k]["parity"]["pattern_exact"] and v[k]["parity"]["values_in_tolerance"]
             for v in rows.values() for k in ("R*RHS", "A*RHS"))
    return {"config": {"workload": f"density experiment: Elasticity (81 per row) on {DENSITY_GRID}^3 "
                                   f"({a.nrows} rows), R and A times random right-hand sides with delta "
                                   f"entries per row (N(0,1)), FP64", "deltas": list(DENSITY_DELTAS),
                       "steps": 3, "warmup": 2},
            "deltas": rows, "clocks": clk, "parity": {"all_rows_sampled_match": ok}}


def measure_weak(args, local):
    """Throughput against problem size (the paper's growing problems): R*A
    and A*P of the 27-point family with A of about 1, 2, 4 and 8 GB, inputs
    generated in worker processes."""
    import paper_1804_00695_gb300 as sg
    workers = max(1, min(len(WEAK_SIZES), (os.cpu_count() or 2) - 1))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as pool:
        futs = {n: pool.submit(_gen_family, "brick3d_27pt", n) for n in WEAK_SIZES}
        h = sg.Handle(local)
        clocks = bench.ClockSampler(local)
        rows = {}
        for n in WEAK_SIZES:
            a, p, r = futs.pop(n).result()
            clocks.start()
            rows[str(n)] = {"A_gb": (8 * (a.nrows + 1) + 12 * a.nnz) / 1e9, "A_rows": a.nrows,
                            "R*A": _product_entry(h, r, a, f"27-point {n}^3 R*A", local, cpu_seconds=0.5),
                            "A*P": _product_entry(h, a, p, f"27-point {n}^3 A*P", local, cpu_seconds=0.5)}
            rows[str(n)]["clocks"] = clocks.stop()
            del a, p, r
    last = rows[str(WEAK_SIZES[-1])]
    return {"metric_value": last["A*P"]["gflops"], "unit": "GFLOP/s", "ms_per_step": last["A*P"]["ms"],
            "steps": 3, "warmup": 2, "dtype": "f64",
            "config": {"workload": "27-point 3D brick family, smoothed aggregation P, FP64: R*A and A*P with A of "
                                   "about 1, 2, 4 and 8 GB (value: A*P at the largest)", "grids": list(WEAK_SIZES)},
            "sizes": rows,
            "parity": {"all_rows_sampled_match": all(v[k]["parity"]["pattern_exact"] and
                                                     v[k]["parity"]["values_in_tolerance"]
                                                     for v in rows.values() for k in ("R*A", "A*P"))}}


def measure_budget(args, local):
    """Device-budget sweep of the chunked product (the paper's Chunk8 /
    Chunk16 runs, Section 4): the chunked workload at several budgets."""
    from paper_1804_00695_gb300 import inputs as I
    a = I.laplace3d_27pt(args.chunk_grid)
    runs = {}
    # below about 4 GB the symbolic call cannot hold B's pattern (1.9 GB) in
    # the budget's large portion and refuses with ERR_BUDGET; at 64 GB A and
    # C (30 GB) fit whole
    for b in (4e9, 8e9, 16e9, 32e9, 64e9):
        args.budget = b
        r = measure_chunked(args, local, a, triple_buffers=False)
        runs[f"{b / 1e9:g}GB"] = {"gflops": r["metric_value"], "ms": r["ms_per_step"],
                                  "symbolic_ms": r["symbolic_ms"], "link_frac": r["roofline"]["frac"],
                                  "bytes_copied_over_minimal": r["bytes_copied_over_minimal"],
                                  "numeric_plan": r["numeric_plan"], "clocks": r["clocks"], "parity": r["parity"]}
    best = max(runs.values(), key=lambda v: v["gflops"])
    return {"metric_value": runs["4GB"]["gflops"], "unit": "GFLOP/s", "ms_per_step": runs["4GB"]["ms"],
            "steps": 2, "warmup": 1, "dtype": "f64",
            "config": {"workload": f"chunked C = A*A, 27-point 3D Laplacian on {args.chunk_grid}^3, FP64, "
                                   "operands and C in pinned host memory, device budgets 4-64 GB (value: 4 GB)"},
            "budgets": runs, "best_gflops": best["gflops"],
            "parity": {"all_rows_sampled_match": all(v["parity"]["values_in_tolerance"] for v in runs.values())}}


# ---------------------------------------------------------------- placements
PLACEMENTS = (("HBM", "device", "device", "device"), ("A_Pin", "pinned", "device", "device"),
              ("B_Pin", "device", "pinned", "device"), ("C_Pin", "device", "device", "pinned"),
              ("HostPin", "pinned", "pinned", "pinned"), ("UVM", "managed", "managed", "managed"))


def measure_placement(args, problem, local, steps=3, warmup=2):
    """The columns of Table 3 (Section 3.3.1) on this GPU: GFLOP/s of the two
    Galerkin products A*P and R*(AP) (AP the oracle's) with A, B and C each in
    HBM, pinned host memory (read and written in place over the host link)
    or managed memory.  Each product is timed with CUDA events over the
    symbolic and numeric calls into preallocated C arrays of the placement;
    the first call (cold: page migration for UVM) is reported apart.  Every
    placement's C is compared with the oracle's whole product."""
    import torch
    import oracle
    import paper_1804_00695_gb300 as sg
    from paper_1804_00695_gb300 import inputs as I
    a, p, r = problem
    t0 = time.perf_counter()
    ap_o = oracle.spgemm(a, p)
    ap = I.Csr(a.nrows, p.ncols, ap_o.row_ptr, ap_o.col, ap_o.val)
    rap_o = oracle.spgemm(r, ap)
    t_oracle = time.perf_counter() - t0
    dev = torch.device("cuda", local)
    h = sg.Handle(local)
    stream = torch.cuda.current_stream()
    out = {}
    for label, x, y, ref in (("A*P", a, p, ap_o), ("R*AP", r, ap, rap_o)):
        flops = 2 * int(ref.mults.sum())
        res = {}
        for name, pa, pb, pc in PLACEMENTS:
            X, Y = sg.Csr.placed(x, pa, device=dev), sg.Csr.placed(y, pb, device=dev)
            nnz = ref.nnz
            Cm = sg.Csr(x.nrows, y.ncols, sg.placed_empty(x.nrows + 1, torch.int64, pc, dev),
                        sg.placed_empty(nnz, torch.int32, pc, dev), sg.placed_empty(nnz, torch.float64, pc, dev))
            ms = []
            for it in range(warmup + steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                _, n2 = h.symbolic(X, Y, out=Cm.row_ptr)
                h.numeric_into(X, Y, Cm)
                e1.record(stream)
                torch.cuda.synchronize()
                assert n2 == nnz
                ms.append(e0.elapsed_time(e1))
            par = _compare_rows(Cm.row_ptr.cpu().numpy(), Cm.col.cpu().numpy(), Cm.val.cpu().numpy(), ref,
                                TOL["f64"])
            t = statistics.median(ms[warmup:])
            res[name] = {"A": pa, "B": pb, "C": pc, "ms": t, "gflops": flops / (t / 1e3) / 1e9,
                         "first_call_ms": ms[0], "parity": par}
            del X, Y, Cm
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        base = res["HBM"]["gflops"]
        for v in res.values():
            v["vs_hbm"] = v["gflops"] / base
        out[label] = {"mults": flops // 2, "nnz_C": ref.nnz, "placements": res}
    return {"config": {"workload": f"placements of Table 3: A*P and R*(AP) of the 27-point {args.grid}^3 "
                                   f"Galerkin problem, FP64, AP from the oracle",
                       "steps": steps, "warmup": warmup},
            "products": out, "oracle_s": t_oracle,
            "parity": {"all_exact_patterns": all(v["parity"]["pattern_exact"] for o in out.values()
                                                 for v in o["placements"].values()),
                       "all_values_in_tolerance": all(v["parity"]["values_in_tolerance"] for o in out.values()
                                                      for v in o["placements"].values())}}


# ---------------------------------------------------------------- one workload as a full line
def run(args, rank, world, local):
    """`--workload X`: one secondary workload as a full JSON line (measured on
    one GPU: under a multi-rank launch rank 0 runs it, the others exit)."""
    import torch
    if world > 1 and rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_1804_00695_gb300 import inputs as I
    if args.workload == "rmat20":
        r = measure_rmat(args, I.rmat_symmetric(args.rmat_scale, 16, seed=1), local)
    elif args.workload == "triangles20":
        r = measure_triangles(args, I.rmat_symmetric(args.rmat_scale, 16, seed=1), local)
    elif args.workload == "chunked256":
        r = measure_chunked(args, local)
    elif args.workload == "weak27":
        r = measure_weak(args, local)
    elif args.workload == "budget256":
        r = measure_budget(args, local)
    elif args.workload == "density":
        r = measure_density(args, _gen_density(DENSITY_GRID, DENSITY_DELTAS), local)
        top = r["deltas"][str(DENSITY_DELTAS[-1])]["A*RHS"]
        r.update({"metric_value": top["gflops"], "unit": "GFLOP/s", "ms_per_step": top["ms"], "steps": 3,
                  "warmup": 2, "dtype": "f64"})
        r["config"]["workload"] += f" (value: A*RHS at delta {DENSITY_DELTAS[-1]})"
    else:
        r = measure_batched(args, I.random_batch(args.batch_count, 1024, args.batch_max, 1, dtype=np.float32),
                            local)
    line = {"metric": bench.METRIC, "value": r.pop("metric_value"), "unit": r.pop("unit"), "n_gpus": 1,
            "steps": r.pop("steps"), "warmup": r.pop("warmup"), "ms_per_step": r.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": r.pop("dtype"),
            "data": "synthetic (seeded generators)", "config": r.pop("config")}
    line.update(r)
    print(json.dumps(line), flush=True)
