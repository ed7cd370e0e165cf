"""Benchmark workloads besides the default Galerkin product (run with
``python bench.py --workload rmat20|chunked256|batched256``); each prints one
JSON line in the same format as bench.py.

* rmat20     - C = A*A, A symmetrised R-MAT scale 20, edge factor 16, FP32.
* chunked256 - C = A*A, A the 27-point Laplacian on 256^3, FP64, operands and
               result in pinned host memory, 4 GB device budget (Section 3.3.1).
* batched256 - 256 products A_i*B_i, rows log-uniform in [1024, 65536], 4-32
               random columns per row, FP32: batched forward and backward
               against a per-instance loop on the same GPU.
"""
from __future__ import annotations

import json
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import bench  # noqa: E402  (shared helpers: clocks, peaks, bytes)


def _line(args, world, metric_value, ms, dtype, config, extra):
    line = {"metric": bench.METRIC, "value": metric_value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic (seeded generators)", "config": config}
    line.update(extra)
    print(json.dumps(line), flush=True)


def _mults(a, b_rp):
    return int(np.diff(b_rp)[a.col.astype(np.int64)].sum())


def run(args, rank, world, local):
    """The secondary workloads are measured on one GPU: under a multi-rank
    launch rank 0 runs and reports them, the other ranks exit at once."""
    import torch
    if world > 1 and rank != 0:
        return
    world = 1
    torch.cuda.set_device(local)
    if args.workload == "rmat20":
        return rmat20(args, world, local)
    if args.workload == "chunked256":
        return chunked256(args, world, local)
    return batched256(args, world, local)


def rmat20(args, world, local):
    import torch
    import paper_1804_00695_gb300 as sg
    from paper_1804_00695_gb300 import inputs as I
    g = I.rmat_symmetric(args.rmat_scale, 16, seed=1)
    A = sg.Csr.from_host(g, "cuda", np.float32)
    h = sg.Handle(local)
    mults = _mults(g, g.row_ptr)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        c = h.spgemm(A, A)
        del c
    h.check()
    h.set_timing(True)
    h.reset_timings()
    clocks = bench.ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        c = h.spgemm(A, A)
        del c
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    tim = h.timings()
    c = h.spgemm(A, A)
    nnz = c.nnz
    crp = c.row_ptr.cpu().numpy()
    del c
    peaks = bench.measured_peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    step_bytes = bench.kernel_bytes(g, g.row_ptr, crp, np.ones(g.nrows, dtype=bool), 4)
    dom = max(tim.items(), key=lambda kv: kv[1][2])
    _line(args, world, 2 * mults / (ms / 1e3) / 1e9, ms, "f32",
          {"workload": f"C = A*A, A symmetrised R-MAT scale {args.rmat_scale}, edge factor 16, "
                       "(a,b,c,d) = (.57,.19,.19,.05), seed 1, FP32", "mults": mults, "nnz_C": nnz},
          {"pct_hbm_byte_roofline": 100 * step_bytes / (ms / 1e3) / 1e9 / hbm,
           "step_algorithmic_bytes": step_bytes,
           "dominant_kernel": {"label": dom[0], "ms_per_step": dom[1][2] / args.steps},
           "kernels_ms_per_step": {k: v[2] / args.steps for k, v in sorted(tim.items())},
           "gpu_launches": sum(v[0] for v in tim.values()) // max(args.steps, 1) * args.steps,
           "clocks": clk})


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


def chunked256(args, world, local):
    import torch
    import paper_1804_00695_gb300 as sg
    from paper_1804_00695_gb300 import inputs as I
    n = args.chunk_grid
    a = I.laplace3d_27pt(n)
    A = sg.HostCsr.from_numpy(a)
    budget = int(args.budget)
    h = sg.Handle(local)
    mults = _mults(a, a.row_ptr)
    link = _link_bandwidth()
    steps = max(1, min(args.steps, 3))
    rp, nnz = h.chunked_symbolic(A, A, budget)
    col = torch.empty(nnz, dtype=torch.int32).pin_memory()
    val = torch.empty(nnz, dtype=torch.float64).pin_memory()
    Cm = sg.HostCsr(a.nrows, a.ncols, rp, col, val)
    clocks = bench.ClockSampler(local)
    times, sym_times, stats = [], [], None
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
    # per-kernel device time of one more (untimed) step
    h.set_timing(True)
    h.reset_timings()
    h.chunked_symbolic(A, A, budget, out=Cm.row_ptr)
    h.chunked_numeric_into(A, A, Cm, budget)
    torch.cuda.synchronize()
    kern = {k: round(v[2], 3) for k, v in h.timings().items()}
    h.set_timing(False)
    size_a = 8 * (a.nrows + 1) + 12 * a.nnz
    size_c = 8 * (a.nrows + 1) + 12 * nnz
    minimal = 2 * size_a + size_c            # A and B in, C out, each once
    moved = stats["h2d_bytes"] + stats["d2h_bytes"] + sym["h2d_bytes"] + sym["d2h_bytes"]
    peak = max(link["bidir"], link["h2d"], link["d2h"])
    _line(args, world, 2 * mults / (ms / 1e3) / 1e9, ms, "f64",
          {"workload": f"chunked C = A*A, 27-point 3D Laplacian on {n}^3, FP64, operands and C in "
                       f"pinned host memory, {budget:.3g}-byte device budget", "mults": mults, "nnz_C": nnz,
           "budget_bytes": budget},
          {"roofline": {"bound": "host-link", "achieved": minimal / (ms / 1e3) / 1e9, "peak": peak,
                        "unit": "GB/s", "frac": minimal / (ms / 1e3) / 1e9 / peak,
                        "traffic": moved, "note": "achieved = minimal bytes (A, B in and C out "
                        "once) over time; traffic = bytes actually copied (symbolic + numeric)"},
           "link_gbs_measured": link, "numeric_plan": stats, "symbolic_plan": sym,
           "symbolic_ms": 1e3 * statistics.median(sym_times), "kernels_ms": kern,
           "clocks": clk})


def batched256(args, world, local):
    import torch
    import paper_1804_00695_gb300 as sg
    from paper_1804_00695_gb300 import inputs as I
    pairs = I.random_batch(args.batch_count, 1024, args.batch_max, 1, dtype=np.float32)
    As = [sg.Csr.from_host(a, "cuda") for a, _ in pairs]
    Bs = [sg.Csr.from_host(b, "cuda") for _, b in pairs]
    mults = sum(_mults(a, b.row_ptr) for a, b in pairs)
    h = sg.Handle(local)
    hl = sg.Handle(local)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    bt = sg.Batch(h, As, Bs)
    fwd_batched = timed(lambda: bt.run(), args.steps)
    loop_out = []

    def loop_fwd():
        loop_out.clear()
        for A, B in zip(As, Bs):
            loop_out.append(hl.spgemm(A, B))
    fwd_loop = timed(loop_fwd, max(1, args.steps // 2))
    # numeric only, replayed from a CUDA graph vs a loop of numeric calls
    bt.symbolic()
    Cm = bt.alloc()
    bt.numeric_into(Cm)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            bt.numeric_into(Cm)
    num_graph = timed(lambda: g.replay(), args.steps)
    singles = []
    for A, B in zip(As, Bs):
        hh = sg.Handle(local)
        rp, nz = hh.symbolic(A, B)
        singles.append((hh, A, B, hh.numeric(A, B, rp, nz)))
    num_loop = timed(lambda: [hh.numeric_into(A, B, c) for hh, A, B, c in singles], args.steps)
    # backward: batched vs loop
    dc = torch.cos(torch.arange(Cm.nnz, device="cuda", dtype=torch.float32))
    bwd_batched = timed(lambda: bt.backward(Cm, dc), args.steps)
    parts = bt.split(Cm)
    dcs = []
    p0 = 0
    for c in parts:
        dcs.append(dc[p0:p0 + c.nnz])
        p0 += c.nnz
    bwd_loop = timed(lambda: [hh.backward(A, B, c, d) for (hh, A, B, c), d in zip(singles, dcs)],
                     max(1, args.steps // 2))
    # per-kernel breakdown of one batched forward and backward (untimed pass)
    h.set_timing(True)
    h.reset_timings()
    bt.run()
    bt.backward(Cm, dc)
    torch.cuda.synchronize()
    kern = {k: round(v[2], 4) for k, v in h.timings().items()}
    h.set_timing(False)
    gf = lambda ms: 2 * mults / (ms / 1e3) / 1e9
    _line(args, world, gf(fwd_batched), fwd_batched, "f32",
          {"workload": f"{args.batch_count} products A_i*B_i, n_i log-uniform in [1024, {args.batch_max}], "
                       "4-32 random columns per row, N(0,1) FP32", "mults": mults, "nnz_C": int(Cm.nnz),
           "rows": int(sum(a.nrows for a, _ in pairs))},
          {"batched_forward_ms": fwd_batched, "loop_forward_ms": fwd_loop,
           "forward_speedup": fwd_loop / fwd_batched,
           "batched_numeric_graph_ms": num_graph, "loop_numeric_ms": num_loop,
           "numeric_speedup": num_loop / num_graph,
           "batched_backward_ms": bwd_batched, "loop_backward_ms": bwd_loop,
           "backward_speedup": bwd_loop / bwd_batched,
           "loop_forward_gflops": gf(fwd_loop), "kernels_ms": kern})
