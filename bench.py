#!/usr/bin/env python
"""Benchmark of the two-phase CSR SpGEMM on the multigrid Galerkin triple
product R*(A*P): A = 27-point 3D Laplacian on a 128^3 grid, P the smoothed
aggregation prolongator over 3x3x3 aggregates, R = P^T, FP64 (synthetic,
seeded).  One step = symbolic + numeric of A*P, then symbolic + numeric of
R*(AP).  Metric: GFLOP/s = 2 x multiplications / second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 (torchrun, one process per GPU) runs independent replicas (the path
has no exchange step): value = all ranks' multiplications / max time.
--impl reference times the CPU oracle on the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpGEMM GFLOP/s (2×mults/s) & % of HBM-byte roofline; batched/bwd vs plain"
BIN_CAP = [0, 16, 32, 128, 1024, 4096]
BIN_FLOPS = [0, 8192, 8192, 65536, 1048576, 16777216]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--grid", type=int, default=128, help="grid of the Galerkin workload (profiling cases)")
    ap.add_argument("--chunk-grid", type=int, default=256, help="grid of the chunked workload (profiling cases)")
    ap.add_argument("--budget", type=float, default=4e9, help="device budget of the chunked workload, bytes")
    ap.add_argument("--rmat-scale", type=int, default=20, help="scale of the R-MAT workload (profiling cases)")
    ap.add_argument("--batch-count", type=int, default=256, help="instances of the batched workload (profiling cases)")
    ap.add_argument("--batch-max", type=int, default=65536, help="largest instance order of the batched workload")
    ap.add_argument("--workload", default="galerkin128",
                    choices=["galerkin128", "rmat20", "triangles20", "chunked256", "batched256", "weak27",
                             "budget256", "density"])
    ap.add_argument("--no-secondary", action="store_true",
                    help="default line without the R-MAT, chunked and batched workloads")
    return ap.parse_args()


def workload_name(n):
    return (f"Galerkin R*(A*P): 27-point 3D Laplacian on {n}^3, smoothed aggregation P "
            f"(3x3x3 aggregates, omega 2/3), R = P^T, FP64")


def mults_of(a_col, a_rp_unused, b_rp):
    return int(np.diff(b_rp)[a_col.astype(np.int64)].sum())


def bins_of(keys, flops):
    """Vectorised copy of the library's bin rule (checked against bin_of)."""
    b = np.where(keys > 0, 1, 0)
    for k in range(1, 6):
        up = (b == k) & ((keys > BIN_CAP[k]) | (flops > BIN_FLOPS[k]))
        b = np.where(up, k + 1, b)
    return b


NARROW_W, NARROW_NMAX, NARROW_FLOPS, NARROW_PAIRS = 128, 32, 8192, 4096


def _seg_reduce(ufunc, vals, rp, empty):
    """ufunc.reduceat over the rows of a CSR (empty rows get `empty`)."""
    n = len(rp) - 1
    out = np.full(n, empty, dtype=np.int64)
    lens = np.diff(rp)
    nz = np.nonzero(lens > 0)[0]
    if len(nz):
        out[nz] = ufunc.reduceat(vals, rp[nz])
    return out


def narrow_numeric_rows(a, b, c_rp, flops):
    """Rows the narrow numeric kernel takes (the library's rule): columns of
    the rows of B they reach within NARROW_W blocks of 32, at most
    NARROW_PAIRS compressed pairs, at most NARROW_NMAX outputs and
    NARROW_FLOPS products."""
    big = np.iinfo(np.int64).max
    blk = b.col.astype(np.int64) >> 5
    brp = np.asarray(b.row_ptr, dtype=np.int64)
    bmin = _seg_reduce(np.minimum, blk, brp, big)
    bmax = _seg_reduce(np.maximum, blk, brp, -1)
    # pairs of a row: runs of consecutive entries in one block
    starts = np.ones(len(blk), dtype=np.int64)
    if len(blk):
        starts[1:] = blk[1:] != blk[:-1]
        starts[brp[:-1][np.diff(brp) > 0]] = 1
    bpairs = _seg_reduce(np.add, starts, brp, 0)
    k = a.col.astype(np.int64)
    arp = np.asarray(a.row_ptr, dtype=np.int64)
    lo = _seg_reduce(np.minimum, bmin[k], arp, big)
    hi = _seg_reduce(np.maximum, bmax[k], arp, -1)
    cp = _seg_reduce(np.add, bpairs[k], arp, 0)
    nn = np.diff(c_rp)
    return ((hi >= lo) & (hi - lo < NARROW_W) & (cp <= NARROW_PAIRS) & (nn > 0) & (nn <= NARROW_NMAX)
            & (flops <= NARROW_FLOPS))


def row_flops_np(a, b_rp):
    per = np.diff(b_rp)[a.col.astype(np.int64)]
    out = np.zeros(a.nrows, dtype=np.int64)
    np.add.at(out, np.repeat(np.arange(a.nrows), np.diff(a.row_ptr)), per)
    return out


def kernel_bytes(a, b_rp, c_rp, rows_mask, vb, numeric=True):
    """Algorithmic bytes of one kernel over the rows in rows_mask: the A rows
    it reads, the B rows they touch (each once), the C rows it writes."""
    alen = np.diff(a.row_ptr)[rows_mask]
    clen = np.diff(c_rp)[rows_mask]
    sel = np.repeat(rows_mask, np.diff(a.row_ptr))
    touched = np.unique(a.col[sel])
    blen = np.diff(b_rp)[touched]
    if numeric:
        return int(alen.size * 8 + alen.sum() * (4 + vb) + touched.size * 8 + blen.sum() * (4 + vb)
                   + clen.size * 8 + clen.sum() * (4 + vb))
    # symbolic: A columns, B pattern (compressed pairs bounded by entries), counts written
    return int(alen.size * 8 + alen.sum() * 4 + touched.size * 8 + blen.sum() * 4 + clen.size * 8)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def source_hash():
    """Hash of the translation units that hold the numeric kernels (the
    dominant kernel of the default line and the headers it includes): a
    stored DRAM-traffic figure is used only while these are unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1804_00695_gb300", "csrc")
    for f in (os.path.join(csrc, "numeric.cu"), os.path.join(csrc, "narrow.cu"), os.path.join(csrc, "internal.cuh"),
              os.path.join(csrc, "dword.cuh"), os.path.join(ROOT, "include", "spgemm.h")):
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def max_over_ranks(ms, dist, device):
    """Step time of the job: the slowest rank's (every rank runs one replica
    of the workload; with no process group, the local time)."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_throughput(flops_per_replica, world, ms):
    """Whole-job GFLOP/s: the work of all replicas over the slowest rank's time."""
    return world * flops_per_replica / (ms / 1e3) / 1e9


# FP64 on GB300: NVIDIA's figure is 1.25 TFLOP/s, i.e. two FP64 FMAs per SM
# per cycle at the 2070 MHz maximum SM clock (152 SMs); the profile of the
# narrow numeric kernel agrees (its FP64 pipe, 42% active, retires 1.9 lane
# FMAs per SM and cycle).  The peak uses the maximum clock seen in the run.
FP64_FMA_PER_SM_CYCLE = 2
FP64_PEAK_NOTE = ("derived: SMs x 2 FP64 FMAs per SM per cycle x 2 flops x the maximum SM clock "
                  "(GB300's nominal 1.25 TFLOP/s FP64)")


def fp64_peak_tflops(nsm, clk):
    mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    return nsm * FP64_FMA_PER_SM_CYCLE * 2 * mhz * 1e6 / 1e12


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return None


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_1804_00695_gb300 import inputs as I
    a, p, r = I.galerkin_problem(args.grid)

    def step():
        ap = oracle.spgemm(a, p)
        rap = oracle.spgemm(r, I.Csr(a.nrows, p.ncols, ap.row_ptr, ap.col, ap.val))
        return int(ap.mults.sum() + rap.mults.sum())

    mults = 0
    for _ in range(args.warmup):
        mults = step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        mults = step()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    val = 2 * mults / (ms / 1e3) / 1e9
    cores = oracle.num_threads()
    line = {"metric": METRIC, "value": val, "unit": "GFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generators)",
            "impl": "reference",
            "config": {"workload": workload_name(args.grid), "grid": args.grid},
            "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": "the full workload (both products) every step"},
            "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload != "galerkin128":
        import bench_workloads
        return bench_workloads.run(args, rank, world, local)

    # inputs of the secondary workloads (one GPU only), generated in worker
    # processes before any CUDA call and before anything is timed
    gen = None
    if world == 1 and not args.no_secondary:
        import bench_workloads
        gen = bench_workloads.Inputs(args)
        gen.rmat_graph()
        gen.batch_pairs()
        gen.families()
        gen.density()

    import torch
    import paper_1804_00695_gb300 as sg
    from paper_1804_00695_gb300 import inputs as I

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # CPU baseline first (rank 0, N = 1): the oracle on the same workload.
    cpu = None
    a, p, r = I.galerkin_problem(args.grid)
    if rank == 0 and world == 1:
        import oracle
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            ap_o = oracle.spgemm(a, p)
            rap_o = oracle.spgemm(r, I.Csr(a.nrows, p.ncols, ap_o.row_ptr, ap_o.col, ap_o.val))
            ts.append(time.perf_counter() - t0)
        om = int(ap_o.mults.sum() + rap_o.mults.sum())
        cpu = {"value": 2 * om / statistics.median(ts) / 1e9, "unit": "GFLOP/s",
               "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "full workload (A*P then R*(AP)), median of 3 runs"}
        del ap_o, rap_o

    dev = torch.device("cuda", local)
    A, P, R = (sg.Csr.from_host(m, dev) for m in (a, p, r))
    h1, h2 = sg.Handle(local), sg.Handle(local)
    stream = torch.cuda.current_stream()

    def step():
        rp1, n1 = h1.symbolic(A, P)
        AP = h1.numeric(A, P, rp1, n1)
        rp2, n2 = h2.symbolic(R, AP)
        RAP = h2.numeric(R, AP, rp2, n2)
        return AP, RAP

    AP, RAP = step()
    h1.check(); h2.check()
    ap_rp = AP.row_ptr.cpu().numpy()
    rap_rp = RAP.row_ptr.cpu().numpy()
    mults_ap = mults_of(a.col, a.row_ptr, p.row_ptr)
    mults_rap = mults_of(r.col, r.row_ptr, ap_rp)
    mults = mults_ap + mults_rap
    for _ in range(max(0, args.warmup - 1)):
        step()
    # inside the timed region only the numeric-phase kernels carry CUDA
    # events (the dominant kernel's live duration for the roofline); every
    # kernel's share comes from an instrumented pass after it
    for h in (h1, h2):
        h.set_timing(2)
        h.reset_timings()
    l0 = h1.launch_count() + h2.launch_count()
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = h1.launch_count() + h2.launch_count() - l0
    ms = max_over_ranks(ms, dist, dev)
    value = replicas_throughput(2 * mults, world, ms)

    # CUDA-event timings of the numeric-phase kernels from the timed region
    tim = {}
    for tag, h in (("AP", h1), ("RAP", h2)):
        for lab, (nl, rows, tms) in h.timings().items():
            tim[f"{tag}.{lab}"] = (nl, rows, tms)
        h.set_timing(1)
        h.reset_timings()
    # every kernel, events around each, over a few more steps
    ki = max(1, min(args.steps, 5))
    for _ in range(ki):
        step()
    all_kernels = {}
    for tag, h in (("AP", h1), ("RAP", h2)):
        for lab, (nl, rows, tms) in h.timings().items():
            all_kernels[f"{tag}.{lab}"] = tms / ki
        h.set_timing(False)
    # algorithmic bytes of every numeric/symbolic bin kernel
    peaks = measured_peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    peak_src = "measured" if peaks else "fallback"
    fl_ap = row_flops_np(a, p.row_ptr)
    fl_rap = row_flops_np(r, ap_rp)
    ap_host = I.Csr(a.nrows, p.ncols, ap_rp, AP.col.cpu().numpy(), None)
    prod = {"AP": (a, p, ap_rp, fl_ap), "RAP": (r, ap_host, rap_rp, fl_rap)}
    kern = []
    for key, (nl, rows, tms) in tim.items():
        parts = key.split(".")
        if len(parts) != 3 or parts[1] != "numeric":
            continue
        am, bm, crp, fl = prod[parts[0]]
        nar = narrow_numeric_rows(am, bm, crp, fl)
        bb = np.where(nar, 7, bins_of(np.diff(crp), fl))
        if parts[2] == "narrow":
            mask = nar
        elif parts[2] == "small":
            mask = (bb == 1) | (bb == 2)
        elif parts[2].startswith("bin"):
            mask = bb == int(parts[2][3:])
            assert mask.sum() == rows // nl, (key, mask.sum(), rows, nl)
        else:
            continue
        brp = bm.row_ptr
        kern.append((tms / nl, key, kernel_bytes(am, brp, crp, mask, 8, True), nl, 2 * int(fl[mask].sum())))
    roof = None
    fp64_peak = fp64_peak_tflops(torch.cuda.get_device_properties(dev).multi_processor_count, clk)
    if kern:
        # dominant kernel: the numeric bin kernel with the largest total time
        best = max(kern, key=lambda x: x[0] * x[3])
        per_ms, key, byt, nl, flop = best
        ach = byt / (per_ms / 1e3) / 1e9
        traffic = None
        tf = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tf):
            t = json.load(open(tf))
            if t.get("source_hash") == source_hash() and key in t.get("kernels", {}):
                traffic = t["kernels"][key]
        # the binding roof: the FP64 FMA rate or the HBM bandwidth, whichever
        # allows less (A*P: 0.445 FLOP per algorithmic byte, above the FP64
        # ridge of about 0.19 FLOP/B)
        hbm_roof = {"achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "peak_source": peak_src}
        fl_ach = flop / (per_ms / 1e3) / 1e12
        fp64_roof = {"achieved": fl_ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": fl_ach / fp64_peak,
                     "peak_source": FP64_PEAK_NOTE}
        if flop / (fp64_peak * 1e12) > byt / (hbm * 1e9):
            roof = {"bound": "alu", "pipe": "fp64", **fp64_roof, "hbm": hbm_roof}
        else:
            roof = {"bound": "hbm", **hbm_roof, "fp64": fp64_roof}
        roof.update({"traffic": traffic, "kernel": key, "bytes_per_launch": byt, "flop_per_launch": flop,
                     "ms_per_launch": per_ms})
    # whole-step HBM-byte roofline: A + B rows touched + C of both products
    allr = np.ones(a.nrows, dtype=bool)
    step_bytes = (kernel_bytes(a, p.row_ptr, ap_rp, allr, 8) +
                  kernel_bytes(r, ap_rp, rap_rp, np.ones(r.nrows, dtype=bool), 8))
    step_frac = step_bytes / (ms / 1e3) / 1e9 / hbm
    step_fp64_frac = 2 * mults / (ms / 1e3) / 1e12 / fp64_peak

    # end to end through the library's host-operand call (spgemm_host): A, P
    # and R in pinned host memory are copied in by the library, A*P stays on
    # the device, R*(AP) comes back to pinned host memory
    Ah, Ph, Rh = (sg.HostCsr.from_numpy(m) for m in (a, p, r))
    h2d = sum(x.numel() * x.element_size() for m in (Ah, Ph, Rh) for x in (m.row_ptr, m.col, m.val))

    def e2e_step():
        APd = h1.host_product(Ah, Ph, keep_on_device=True)
        return h2.host_product(Rh, APd)

    o = e2e_step()
    d2h = sum(x.numel() * x.element_size() for x in (o.row_ptr, o.col, o.val))
    ke = max(1, min(args.steps, 5))
    barrier()
    e0.record(stream)
    for _ in range(ke):
        e2e_step()
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / ke
    e2e_ms = max_over_ranks(e2e_ms, dist, dev)

    a_bytes = 8 * (a.nrows + 1) + 12 * a.nnz
    secondary = None
    if gen is not None:
        # the other workloads (graph product, triangles, chunked, placements,
        # multigrid families, density, batched), measured on this GPU after the
        # default one
        del A, P, R, AP, RAP, h1, h2, Ah, Ph, Rh, o
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        secondary = {}
        for name, fn in (("rmat20", lambda: bench_workloads.measure_rmat(args, gen.rmat_graph(), local)),
                         ("triangles20", lambda: bench_workloads.measure_triangles(args, gen.rmat_graph(), local)),
                         ("chunked256", lambda: bench_workloads.measure_chunked(args, local)),
                         ("placement128", lambda: bench_workloads.measure_placement(args, (a, p, r), local)),
                         ("families", lambda: bench_workloads.measure_families(
                             args, {**gen.families(), "brick3d_27pt": (a, p, r)}, local)),
                         ("density", lambda: bench_workloads.measure_density(args, gen.density(), local)),
                         ("batched256", lambda: bench_workloads.measure_batched(args, gen.batch_pairs(), local))):
            t0 = time.perf_counter()
            try:
                secondary[name] = fn()
            except Exception as exc:   # one workload failing does not lose the others
                secondary[name] = {"error": f"{type(exc).__name__}: {exc}"}
            secondary[name]["wall_s"] = time.perf_counter() - t0
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        gen.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded generators)",
                "config": {"workload": workload_name(args.grid), "grid": args.grid,
                           "mults": mults, "nnz_AP": int(ap_rp[-1]), "nnz_RAP": int(rap_rp[-1]),
                           "l2": (f"inputs larger than L2 (A alone {a_bytes / 1e6:.0f} MB), no flush"
                                  if a_bytes > 129e6 else "inputs smaller than L2, no flush"),
                           "parallelism": f"replicas x{world}"},
                "pct_hbm_byte_roofline": 100 * step_frac,
                "pct_fp64_roofline": 100 * step_fp64_frac,
                "step_algorithmic_bytes": step_bytes,
                "roofline": roof,
                "kernels_ms_per_step": dict(sorted(all_kernels.items())),
                "kernels_ms_note": ("every kernel bracketed by CUDA events, in steps after the timed region; "
                                    "inside it only the numeric-phase kernels carry events"),
                "gpu_launches": launches,
                "clocks": clk,
                "e2e": {"value": world * 2 * mults / (e2e_ms / 1e3) / 1e9, "unit": "GFLOP/s",
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                        "entry_point": "spgemm_host (A, P host -> AP device; R host * AP -> RAP host)"},
                "cpu_baseline": cpu}
        if secondary is not None:
            line["secondary"] = secondary
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
