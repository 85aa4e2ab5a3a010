"""Benchmark of the PageRank pipeline hot path on GB300.

One step = Kernel 1 (sort) + Kernel 2 (build/filter/normalise) + Kernel 3
(20 PageRank iterations, binary32 ranks) on one synthetic Kronecker graph
of scale 24 (N = 2^24 vertices, M = 2^28 edges, initiator
0.57/0.19/0.19/0.05), with the edge list already resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is the whole-pipeline rate M / (time of one
K1+K2+K3 step), summed over ranks; per-kernel rates (K1: M/t, K2: M/t, K3:
20 M/t, as the paper defines them) are under "kernels".  With --gpus N > 1
(launched by torchrun) every rank runs its own independent graph (different
seed): weak scaling, no collective on the data path.

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload instead.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "K3 PageRank edges/s and K1-K3 edges/s at scale 24; FP32 vs FP64 at L1 err<=1e-6"
SCALE = 24
ITERS = 20
DAMPING = 0.85
SEED = 1
WORKLOAD = ("Kronecker graph, scale 24 (N=2^24, M=16N=268,435,456 edges, initiator A/B/C/D=0.57/0.19/0.19/0.05, "
            "seeded Philox), Kernel 1 sort + Kernel 2 filter/normalise + Kernel 3 20 damped iterations (c=0.85)")

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of
# each stage's dominant kernel from one ncu capture (profiles/), valid while
# its source file is unchanged.
TRAFFIC = {
    "k3_pagerank": {"source": "paper_1603_01876_gb300/csrc/k3_pagerank.cu", "sha": "db2b7e9a0668a0ea",
                    "bytes_per_launch": 1320004000 + 38381312, "dtype": "fp32", "scale": 24,
                    "capture": "profiles/k3_iterate_fp32_scale24.md"},
}


def _sha(path):
    with open(os.path.join(ROOT, path), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def _smi_time(ts):
    """Seconds since the epoch of an nvidia-smi timestamp ("YYYY/MM/DD HH:MM:SS.mmm", local time)."""
    import datetime

    return datetime.datetime.strptime(ts.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()


def clock_summary(lines, begin=None, end=None, slack=0.05):
    """Median SM clock, maximum clock and throttle reasons of the samples taken
    between begin and end (host seconds since the epoch, widened by `slack`
    for the sampling granularity).  Each line is one nvidia-smi sample:
    timestamp, index, clocks.sm, clocks.max.sm, power.draw,
    clocks_event_reasons.active, then the four reasons of REASONS."""
    rows = []
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 10:
            continue
        try:
            rows.append((_smi_time(f[0]), float(f[2]), float(f[3]), f[6:10]))
        except ValueError:
            continue
    inside = rows
    if begin is not None and end is not None:
        inside = [r for r in rows if begin - slack <= r[0] <= end + slack]
    if not inside:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "samples_outside": len(rows)}
    reasons = set()
    for r in inside:
        for n, val in zip(REASONS, r[3]):
            if val.lower() == "active":
                reasons.add(n)
    return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
            "reasons": sorted(reasons), "samples": len(inside), "samples_outside": len(rows) - len(inside)}


class ClockSampler:
    """nvidia-smi samples of the SM clock and the throttle reasons, every 50 ms.

    Start it before the warm-up (nvidia-smi takes a moment to begin), call
    begin() and end() around the timed region, stop() after it; summary()
    keeps the samples whose nvidia-smi timestamps fall inside the region."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, index, exe="nvidia-smi"):
        self.index = index
        self.exe = exe
        self.proc = None
        self.lines = []
        self.t_begin = self.t_end = None

    def start(self):
        try:
            self.proc = subprocess.Popen([self.exe, "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def begin(self):
        self.t_begin = time.time()

    def end(self):
        self.t_end = time.time()

    def stop(self):
        if self.proc:
            # the samples of the region's last moments are written a period later
            time.sleep(2 * self.PERIOD_MS / 1000.0)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=5)

    def __enter__(self):
        self.start()
        self.begin()
        return self

    def __exit__(self, *a):
        self.end()
        self.stop()

    def summary(self):
        return clock_summary(list(self.lines), self.t_begin, self.t_end, slack=self.PERIOD_MS / 1000.0)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seed(rank):
    """Each rank generates its own graph and start vector (weak scaling)."""
    return SEED + rank


def max_over_ranks(x, world, device="cpu"):
    """The largest x over all ranks (the slowest rank's time); x itself on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: the units every rank processed over the slowest rank's time (ms)."""
    return world * units_per_rank / (ms * 1e-3)


def k3_bytes_per_iter(nnz, N, dtype):
    """Algorithmic bytes of one Kernel 3 iteration: packed entries, column ends,
    one read of each gathered x, 1/d_out, the new x."""
    xs = {"fp64": 8, "fp32": 4, "bf16": 2, "fp16": 2}[dtype]
    inv = 8 if dtype == "fp64" else 4
    return 4 * nnz + 4 * N + xs * N + inv * N + xs * N


def k1_bytes(M, scale):
    """Algorithmic bytes of Kernel 1: one read of (u, v) for the histograms, then
    per pass a read and a write of every key (4-byte keys when 2*scale <= 32,
    8-byte otherwise)."""
    P = -(-2 * scale // 8)
    kb = 4 if 2 * scale <= 32 else 8
    return M * (8 + 2 * kb * P), P


def k2_bytes(M, N, nnz0, nnz, scale):
    """Algorithmic bytes of Kernel 2 as a design-independent count: read the
    sorted edges, write and re-read (u, v, count) triples, write the filtered
    matrix, transpose it (read + write), and about 25 bytes of per-vertex
    vectors (d_in, mask, d_out, column pointers, 1/d_out)."""
    return 8 * M + 12 * nnz0 + 12 * nnz0 + 12 * nnz + 24 * nnz + 25 * N


def run_ours(args):
    import numpy as np
    import torch

    import kernel0
    import paper_1603_01876_gb300 as pp

    world, rank, local = dist_env()
    # the oracle on the same graph, in a child process started before the
    # first CUDA call, for the errors against it reported per run
    oracle_run = None
    if rank == 0 and not args.no_oracle:
        from oracle import fullsize

        import atexit

        oracle_run = fullsize.start(args.scale, rank_seed(rank))
        atexit.register(oracle_run.cancel)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    scale, iters = args.scale, ITERS
    N = 1 << scale
    M = 16 * N
    seed = rank_seed(rank)
    u, v = kernel0.edges_device(scale, seed, device=dev)
    r0h = kernel0.r0_host(N, seed)
    r0 = torch.from_numpy(r0h).to(dev)
    us = torch.empty_like(u)
    vs = torch.empty_like(v)
    g = pp.Graph(M, scale, dev)
    ws_bytes = max(pp.workspace_bytes("sort", M, scale), pp.workspace_bytes("build", M, scale),
                   pp.workspace_bytes("pagerank", M, scale, iters, "fp64"))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    r_out = torch.empty(N, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None, dtype=args.dtype, out=r_out):
        if ev:
            ev[0].record(stream)
        pp.sort_edges(u, v, scale, out=(us, vs), workspace=ws)
        if ev:
            ev[1].record(stream)
        pp.build_filter_normalize(us, vs, scale, "lowest", graph=g, workspace=ws)
        if ev:
            ev[2].record(stream)
        pp.pagerank(g, r0, iters, DAMPING, dtype, out=out, workspace=ws)
        if ev:
            ev[3].record(stream)

    clocks = ClockSampler(local).start()  # running by the time the timed region starts
    try:
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        err = pp.last_device_error()
        if err:
            raise RuntimeError("device error word %#x during warm-up" % err)
        info = g.info_dict()

        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        launches0 = pp.launch_count()
        clocks.begin()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(args.steps):
            step(evs[k])
        t1.record(stream)
        torch.cuda.synchronize()
        clocks.end()
    finally:
        clocks.stop()
    launches = pp.launch_count() - launches0
    total_ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
    if world > 1:
        torch.distributed.barrier()
    k1 = [e[0].elapsed_time(e[1]) for e in evs]
    k2 = [e[1].elapsed_time(e[2]) for e in evs]
    k3 = [e[2].elapsed_time(e[3]) for e in evs]
    err = pp.last_device_error()
    if err:
        raise RuntimeError("device error word %#x in the timed region" % err)
    ms_step = total_ms / args.steps

    def time_k3(dtype, out, n_iters, reps=3):
        pp.pagerank(g, r0, n_iters, DAMPING, dtype, out=out, workspace=ws)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        for _ in range(reps):
            pp.pagerank(g, r0, n_iters, DAMPING, dtype, out=out, workspace=ws)
        e[1].record(stream)
        torch.cuda.synchronize()
        return e[0].elapsed_time(e[1]) / reps

    # Kernel 3 in binary64 and with the gathered vector in bfloat16 on the same
    # graph; errors of the binary32 and bfloat16 ranks against binary64
    r64 = torch.empty(N, dtype=torch.float64, device=dev)
    k3_64 = time_k3("fp64", r64, iters)
    r_bf = torch.empty(N, dtype=torch.float32, device=dev)
    k3_bf = time_k3("bf16", r_bf, iters)
    r_h = torch.empty(N, dtype=torch.float32, device=dev)
    k3_h = time_k3("fp16", r_h, iters)
    # the iteration kernel alone: the stage minus its set-up (the same call with 0 iterations)
    r_tmp = torch.empty(N, dtype=torch.float64 if args.dtype == "fp64" else torch.float32, device=dev)
    k3_setup = time_k3(args.dtype, r_tmp, 0)
    del r_tmp

    # the gather ceiling of an iteration on this graph: its nnz packed entries
    # streamed and x gathered with nothing else done (pp_gather_probe)
    gather_ms = time_gather_probe(g, nnz_of(g), dev)

    def errors(r):
        d = (r.double() - r64).abs()
        return float(d.sum() / r64.abs().sum()), float((d / r64.abs()).max())

    l1_fp32, maxrel_fp32 = errors(r_out)
    l1_bf, maxrel_bf = errors(r_bf)
    ranks_host = {"fp64": r64.cpu().numpy(), args.dtype: r_out.cpu().numpy(), "bf16": r_bf.cpu().numpy(),
                  "fp16": r_h.cpu().numpy()}

    # Kernel 3 variants on the same graph (pp_pagerank_ex): the dangling-node
    # term (20 iterations), and with the convergence test as well
    variants = {}
    ws_ex = torch.empty(pp.workspace_bytes("pagerank_ex", M, scale, 200, args.dtype), dtype=torch.uint8, device=dev)
    for name, kw, n_it in (("dangling_20", dict(dangling=True), 20),
                           ("dangling_converge_1e-6", dict(dangling=True, tol=1e-6), 200)):
        rv, done = pp.pagerank_ex(g, r0, n_it, DAMPING, args.dtype, workspace=ws_ex, **kw)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        for _ in range(3):
            rv, done = pp.pagerank_ex(g, r0, n_it, DAMPING, args.dtype, workspace=ws_ex, **kw)
        e[1].record(stream)
        torch.cuda.synchronize()
        k = int(done.item())
        ms = e[0].elapsed_time(e[1]) / 3
        variants[name] = {"ms": ms, "iterations": k, "edges_per_s": k * M / (ms * 1e-3),
                          "sum_r": float(rv.double().sum())}
    del ws_ex

    # Kernel 1 with its files (Sec. IV-B): the edge-file text sits in pinned
    # host memory (standing in for storage); copied in, parsed, sorted,
    # formatted and copied out on the GPU
    files = {}
    if not args.no_files:
        text, n = pp.format_tsv(u, v)  # Kernel 0's file (untimed)
        tlen = int(n.item())
        host_in = text[:tlen].cpu().pin_memory()
        del text
        torch.cuda.empty_cache()
        dev_in = torch.empty(tlen, dtype=torch.uint8, device=dev)
        dev_out = torch.empty(M * pp.TSV_MAX_LINE, dtype=torch.uint8, device=dev)
        host_out = torch.empty(tlen, dtype=torch.uint8).pin_memory()
        pu, pv = torch.empty_like(u), torch.empty_like(v)
        su, sv = torch.empty_like(u), torch.empty_like(v)

        def k1_files(ev=None):
            if ev:
                ev[0].record(stream)
            dev_in.copy_(host_in, non_blocking=True)
            if ev:
                ev[1].record(stream)
            pp.parse_tsv(dev_in, tlen, M, out=(pu, pv))
            if ev:
                ev[2].record(stream)
            pp.sort_edges(pu, pv, scale, out=(su, sv), workspace=ws)
            if ev:
                ev[3].record(stream)
            pp.format_tsv(su, sv, out=dev_out)
            if ev:
                ev[4].record(stream)
            host_out.copy_(dev_out[:tlen], non_blocking=True)
            if ev:
                ev[5].record(stream)

        k1_files()
        torch.cuda.synchronize()
        if pp.last_device_error():
            raise RuntimeError("device error in the edge-file path")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        k1_files(ev)
        torch.cuda.synchronize()
        t = [ev[i].elapsed_time(ev[i + 1]) for i in range(5)]
        total_f = sum(t)
        files = {"text_bytes": tlen, "h2d_ms": t[0], "parse_ms": t[1], "sort_ms": t[2], "format_ms": t[3],
                 "d2h_ms": t[4], "k1_with_files_ms": total_f, "k1_with_files_edges_per_s": M / (total_f * 1e-3),
                 "parse_gbs": tlen / t[1] / 1e6, "format_gbs": tlen / t[3] / 1e6,
                 "storage": "pinned host memory (no disk)"}
        del dev_in, dev_out, host_in, host_out, pu, pv, su, sv
        torch.cuda.empty_cache()

    # end to end through the host-buffer entry point
    uh = u.cpu().pin_memory()
    vh = v.cpu().pin_memory()
    r0p = torch.from_numpy(r0h).pin_memory()
    rh = torch.empty(N, dtype=torch.float32).pin_memory()
    infoh = torch.zeros(pp.INFO_LEN, dtype=torch.int64).pin_memory()
    del ws
    torch.cuda.empty_cache()
    pws = torch.empty(pp.workspace_bytes("pipeline", M, scale, iters, args.dtype), dtype=torch.uint8, device=dev)
    pp.pipeline_host(uh, vh, scale, r0p, iters, DAMPING, args.dtype, out=rh, info=infoh, workspace=pws)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 5))
    te = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    te[0].record(stream)
    for _ in range(e2e_steps):
        pp.pipeline_host(uh, vh, scale, r0p, iters, DAMPING, args.dtype, out=rh, info=infoh, workspace=pws)
    te[1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(te[0].elapsed_time(te[1]) / e2e_steps, world, dev)

    nnz, nnz0 = info["nnz"], info["nnz0"]
    peak, peak_kind = _peaks()
    b1, P = k1_bytes(M, scale)
    b2 = k2_bytes(M, N, nnz0, nnz, scale)
    b3_iter = k3_bytes_per_iter(nnz, N, args.dtype)
    b3 = b3_iter * iters
    med = statistics.median
    stages = {"k1_sort": (med(k1), b1), "k2_filter": (med(k2), b2), "k3_pagerank": (med(k3), b3)}
    dom = max(stages, key=lambda s: stages[s][0])
    dom_ms, dom_bytes = stages[dom]
    iter_ms = (med(k3) - k3_setup) / iters
    if dom == "k3_pagerank":
        # per launch of the iteration kernel: one iteration's bytes over its average duration
        kname, launches_per_stage = "k3 iterate_kernel (warp-tiled, degree-bucketed pull SpMV)", iters
        achieved = b3_iter / (iter_ms * 1e-3) / 1e9
        per_launch = {"bytes": b3_iter, "ms": iter_ms,
                      "how": "(K3 stage time - same call with 0 iterations) / iterations, CUDA events; bytes: "
                             "4 nnz (packed entries) + 4 N (column ends) + N (x gathered once, 1/d_out, x written) "
                             "at the stored widths; r itself is written only in the last iteration, so no "
                             "per-iteration write of r is counted"}
    else:
        kname = "k1 onesweep pass_kernel (8-bit LSD pass)" if dom == "k1_sort" else "k2 stage"
        launches_per_stage = P if dom == "k1_sort" else 1
        achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
        per_launch = {"bytes": dom_bytes, "ms": dom_ms, "how": "whole stage, CUDA events"}
    gather_ceiling = {"ms": gather_ms, "gathers": nnz, "kernel": "pp_gather_probe (nnz packed entries streamed, x "
                      "gathered through L1, 8 loads in flight per thread, nothing else)",
                      "iteration_frac_of_ceiling": gather_ms / iter_ms}
    tr = TRAFFIC.get(dom)
    traffic = None
    if tr and tr.get("sha") == _sha(tr["source"]) and (tr.get("dtype"), tr.get("scale")) == (args.dtype, scale):
        traffic = tr["bytes_per_launch"]

    out = {
        "metric": METRIC,
        "value": job_rate(M, world, ms_step),
        "unit": "edges/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.dtype == "fp32" else args.dtype,
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "scale": scale, "vertices": N, "edges": M, "iters": iters,
                   "rank_dtype": args.dtype, "supernode_rule": "lowest", "nnz0": nnz0, "nnz": nnz,
                   "l2": "inputs larger than L2 (2 GiB edge list; 126 MB L2), no flush",
                   "parallelism": "independent graph per GPU" if world > 1 else "single GPU",
                   "tuning": dict(args.tuned, **{kv.split("=")[0]: int(kv.split("=")[1]) for kv in args.tune})},
        "kernels": {
            "k1_sort": {"ms": med(k1), "edges_per_s": M / (med(k1) * 1e-3), "gbs": b1 / med(k1) / 1e6},
            "k2_filter": {"ms": med(k2), "edges_per_s": M / (med(k2) * 1e-3), "gbs": b2 / med(k2) / 1e6},
            "k3_pagerank": {"ms": med(k3), "edges_per_s": iters * M / (med(k3) * 1e-3), "gbs": b3 / med(k3) / 1e6},
            "k3_pagerank_fp64": {"ms": k3_64, "edges_per_s": iters * M / (k3_64 * 1e-3),
                                 "gbs": k3_bytes_per_iter(nnz, N, "fp64") * iters / k3_64 / 1e6},
            "k3_pagerank_bf16": {"ms": k3_bf, "edges_per_s": iters * M / (k3_bf * 1e-3),
                                 "gbs": k3_bytes_per_iter(nnz, N, "bf16") * iters / k3_bf / 1e6},
            "k3_pagerank_fp16": {"ms": k3_h, "edges_per_s": iters * M / (k3_h * 1e-3),
                                 "gbs": k3_bytes_per_iter(nnz, N, "fp16") * iters / k3_h / 1e6},
            "k3_iteration": {"ms": iter_ms, "setup_ms": k3_setup},
        },
        "binary64_step": {"ms": med(k1) + med(k2) + k3_64,
                          "edges_per_s": job_rate(M, world, med(k1) + med(k2) + k3_64),
                          "how": "Kernels 1 and 2 of the timed steps plus Kernel 3 in binary64 (the paper's "
                                 "language-default precision), each timed with CUDA events"},
        "k3_variants": variants,
        "k1_files": files,
        "accuracy": {"fp32_vs_gpu_fp64_l1": l1_fp32, "fp32_vs_gpu_fp64_max_rel": maxrel_fp32,
                     "bf16_vs_gpu_fp64_l1": l1_bf, "bf16_vs_gpu_fp64_max_rel": maxrel_bf},
        "roofline": {"bound": "hbm", "kernel": kname, "stage": dom, "launches_per_step": launches_per_stage,
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "per_launch": per_launch,
                     "algorithmic_bytes_per_step": dom_bytes, "gather_ceiling": gather_ceiling},
        "e2e": {"value": job_rate(M, world, e2e_ms), "unit": "edges/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": 8 * M + 8 * N, "d2h_bytes_per_step": 4 * N + 8 * pp.INFO_LEN},
        "gpu_launches": launches,
        "clocks": clocks.summary(),
    }
    if not args.no_batched:
        del pws
        torch.cuda.empty_cache()
        out["batched"] = run_batched(dev)
    if oracle_run is not None:
        out["accuracy_vs_oracle"] = accuracy_vs_oracle(oracle_run, ranks_host, info)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(scale, seed, max_seconds=args.cpu_seconds)
        secs = out.get("accuracy_vs_oracle", {}).get("oracle_seconds")
        if secs:
            # the oracle's whole-graph run the accuracy block compares with: the full configuration's rate
            t = secs["k1"] + secs["k2"] + secs["k3"]
            out["cpu_baseline"]["full_config"] = {
                "edges_per_s": M / t, "seconds": secs, "cores": 1,
                "what": "the oracle on the whole scale-24 graph (Kernels 1-3, 20 binary64 iterations, one core), "
                        "run in a child process beside the GPU timing (or the cached result of an earlier such "
                        "run); `value` above is the bounded sample"}
    if rank == 0:
        line = json.dumps(out)
        print(line)
        if args.log:
            with open(args.log, "a") as f:  # one run per line
                f.write(line + "\n")
    if world > 1:
        torch.distributed.destroy_process_group()


def nnz_of(g):
    return g.info_dict()["nnz"]


def time_gather_probe(g, n, dev, reps=5):
    """Best of `reps` CUDA-event timings (ms) of pp_gather_probe over the
    graph's first n packed entries, x a random binary32 vector."""
    import torch

    import paper_1603_01876_gb300 as pp

    x = torch.rand(g.N, device=dev)
    out = torch.zeros(1, device=dev)
    pp.gather_probe(g, x, out, n)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record()
        pp.gather_probe(g, x, out, n)
        e[1].record()
        torch.cuda.synchronize()
        best = min(best, e[0].elapsed_time(e[1]))
    return best


def accuracy_vs_oracle(run, ranks, info, timeout=3600):
    """Errors of this run's ranks against the oracle's (binary64, one thread,
    the same graph and start vector), relative to norm(r, 1), and whether
    Kernel 2's scalars agree."""
    import numpy as np

    want = run.wait(timeout=timeout)
    r = want["r"]
    out = {"reference": "CPU oracle, binary64, one thread, the same graph and start vector",
           "k2_scalars_equal": all(info[k] == want[k] for k in ("nnz0", "nnz", "dmax", "vmax", "ties")),
           "oracle_seconds": want["seconds"]}
    for name, got in ranks.items():
        d = np.abs(got.astype(np.float64) - r)
        nz = r != 0
        out[name] = {"l1": float(d.sum() / np.abs(r).sum()),
                     "max_rel": float((d[nz] / np.abs(r[nz])).max()) if nz.any() else 0.0}
    return out


def run_k3_only(args):
    """Kernel 3 alone on a graph built by Kernels 1-2, with everything else freed
    (about 1.6 GB resident at scale 24): for per-kernel timing and profiling."""
    import torch

    import kernel0
    import paper_1603_01876_gb300 as pp

    dev = torch.device("cuda", 0)
    scale, iters = args.scale, ITERS
    N = 1 << scale
    M = 16 * N
    u, v = kernel0.edges_device(scale, SEED, device=dev)
    us, vs = pp.sort_edges(u, v, scale)
    del u, v
    g = pp.build_filter_normalize(us, vs, scale, "lowest")
    info = g.info_dict()
    del us, vs
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    r0 = torch.from_numpy(kernel0.r0_host(N, SEED)).to(dev)
    ws = torch.empty(pp.workspace_bytes("pagerank", M, scale, iters, args.dtype), dtype=torch.uint8, device=dev)
    out = torch.empty(N, dtype=torch.float64 if args.dtype == "fp64" else torch.float32, device=dev)
    for _ in range(args.warmup):
        pp.pagerank(g, r0, iters, DAMPING, args.dtype, out=out, workspace=ws)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record()
    for _ in range(args.steps):
        pp.pagerank(g, r0, iters, DAMPING, args.dtype, out=out, workspace=ws)
    e[1].record()
    torch.cuda.synchronize()
    ms = e[0].elapsed_time(e[1]) / args.steps
    # the same call with 0 iterations: the set-up alone
    for _ in range(2):
        pp.pagerank(g, r0, 0, DAMPING, args.dtype, out=out, workspace=ws)
    torch.cuda.synchronize()
    e[0].record()
    for _ in range(args.steps):
        pp.pagerank(g, r0, 0, DAMPING, args.dtype, out=out, workspace=ws)
    e[1].record()
    torch.cuda.synchronize()
    setup_ms = e[0].elapsed_time(e[1]) / args.steps
    b = k3_bytes_per_iter(info["nnz"], N, args.dtype) * iters
    gather_ms = time_gather_probe(g, info["nnz"], dev)
    print(json.dumps({"stage": "k3", "scale": scale, "dtype": args.dtype, "tune": args.tune, "tuned": args.tuned,
                      "ms": ms, "setup_ms": setup_ms, "iter_ms": (ms - setup_ms) / iters, "nnz": info["nnz"],
                      "gather_ceiling_ms": gather_ms, "iteration_frac_of_gather_ceiling": gather_ms / ((ms - setup_ms) / iters),
                      "edges_per_s": iters * M / (ms * 1e-3), "gbs": b / ms / 1e6,
                      "device_error": pp.last_device_error()}))


def run_k1_k2_only(args):
    """Kernel 1 (--stage k1) or Kernel 2 (--stage k2) alone on the graph of
    --scale, with its workspace allocated once: for per-kernel timing and
    profiling (the launch order of one call: Kernel 1's histogram and its
    passes; Kernel 2's kernels as listed in k2_build.cu)."""
    import torch

    import kernel0
    import paper_1603_01876_gb300 as pp

    dev = torch.device("cuda", 0)
    scale = args.scale
    M = 16 << scale
    u, v = kernel0.edges_device(scale, SEED, device=dev)
    us, vs = torch.empty_like(u), torch.empty_like(v)
    if args.stage == "k1":
        ws = torch.empty(pp.workspace_bytes("sort", M, scale), dtype=torch.uint8, device=dev)
        call = lambda: pp.sort_edges(u, v, scale, out=(us, vs), workspace=ws)
        nbytes = k1_bytes(M, scale)[0]
    else:
        pp.sort_edges(u, v, scale, out=(us, vs))
        del u, v
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        ws = torch.empty(pp.workspace_bytes("build", M, scale), dtype=torch.uint8, device=dev)
        g = pp.Graph(M, scale, dev)
        call = lambda: pp.build_filter_normalize(us, vs, scale, "lowest", graph=g, workspace=ws)
        call()
        info = g.info_dict()
        nbytes = k2_bytes(M, 1 << scale, info["nnz0"], info["nnz"], scale)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record()
    for _ in range(args.steps):
        call()
    e[1].record()
    torch.cuda.synchronize()
    ms = e[0].elapsed_time(e[1]) / args.steps
    print(json.dumps({"stage": args.stage, "scale": scale, "edges": M, "ms": ms, "edges_per_s": M / (ms * 1e-3),
                      "gbs": nbytes / ms / 1e6, "device_error": pp.last_device_error()}))


def run_batched(dev, steps=3, warmup=1, nrhs=32, n_graphs=64, lo=12, hi=18):
    """The batched configuration: 64 Kronecker graphs of scales drawn from
    12..18, each with 32 start vectors.  Kernels 1 and 2 for all graphs at
    once (one set of launches), Kernel 3 as one SpMM launch per iteration
    (binary32), timed per stage and as one CUDA-graph replay of the whole
    pipeline; against 64 sequential single-graph pipelines (Kernels 1 and 2,
    then the 32 start vectors as 32 binary64 runs) on the same GPU."""
    import numpy as np
    import torch

    import kernel0
    import paper_1603_01876_gb300 as pp

    scales = kernel0.batch_scales(n_graphs, lo, hi, seed=SEED)
    us, vs = [], []
    for g, sc in enumerate(scales):
        u, v = kernel0.edges_device(sc, SEED, graph=g, device=dev)
        us.append(u)
        vs.append(v)
    r0 = np.concatenate([np.stack([kernel0.r0_host(1 << sc, SEED, graph=g, rhs=j) for j in range(nrhs)], axis=1)
                         for g, sc in enumerate(scales)])
    r0d = torch.from_numpy(r0).to(dev)
    edges = int(sum(u.numel() for u in us))
    stream = torch.cuda.current_stream(dev)

    def timed(fn, n=steps, w=warmup):
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        for _ in range(n):
            fn()
        e[1].record(stream)
        torch.cuda.synchronize()
        return e[0].elapsed_time(e[1]) / n

    # the stages with stream launches, in buffers reused between steps
    sorted_b = pp.sort_edges_batched(us, vs, scales)
    graphs = pp.build_filter_normalize_batched(sorted_b, scales)
    out = pp.pagerank_batched(graphs, r0d, nrhs, ITERS, DAMPING)
    torch.cuda.synchronize()
    k1_ms = timed(lambda: pp.sort_edges_batched(us, vs, scales, outs=sorted_b))
    k2_ms = timed(lambda: pp.build_filter_normalize_batched(sorted_b, scales, graphs=graphs))
    k3_ms = timed(lambda: pp.pagerank_batched(graphs, r0d, nrhs, ITERS, DAMPING, out=out))
    out0 = torch.empty_like(out)
    k3_setup_ms = timed(lambda: pp.pagerank_batched(graphs, r0d, nrhs, 0, DAMPING, out=out0))
    del out0
    # Kernel 3 alone and the whole pipeline, each recorded once as a CUDA graph and replayed
    ex3 = pp.BatchedExec(graphs, r0d, nrhs, ITERS, DAMPING, out=out)
    k3_graph_ms = timed(ex3.launch)
    ex3.close()
    exp = pp.BatchedPipelineExec(us, vs, scales, r0d, nrhs, ITERS, DAMPING)
    pipe_ms = timed(exp.launch)
    pipe_out = exp.out
    same = bool(torch.equal(pipe_out, out))
    exp.close()
    # the sequential single-graph pipelines: Kernels 1-2 per graph, then 32 binary64 runs each
    row = np.cumsum([0] + [1 << sc for sc in scales])
    cols = [[r0d[row[g]:row[g + 1], j].contiguous() for j in range(nrhs)] for g in range(n_graphs)]
    ref = torch.empty(int(row[-1]), nrhs, dtype=torch.float64, device=dev)
    ws = torch.empty(max(max(pp.workspace_bytes("sort", gr.M, gr.scale), pp.workspace_bytes("build", gr.M, gr.scale),
                             pp.workspace_bytes("pagerank", gr.M, gr.scale, ITERS, "fp64")) for gr in graphs),
                     dtype=torch.uint8, device=dev)
    seq_sorted = [(torch.empty_like(u), torch.empty_like(v)) for u, v in zip(us, vs)]
    seq_graphs = [pp.Graph(u.numel(), sc, dev) for u, sc in zip(us, scales)]

    def seq_k12():
        for g, sc in enumerate(scales):
            pp.sort_edges(us[g], vs[g], sc, out=seq_sorted[g], workspace=ws)
            pp.build_filter_normalize(seq_sorted[g][0], seq_sorted[g][1], sc, graph=seq_graphs[g], workspace=ws)

    def seq_k3():
        for g in range(n_graphs):
            for j in range(nrhs):
                ref[row[g]:row[g + 1], j] = pp.pagerank(seq_graphs[g], cols[g][j], ITERS, DAMPING, "fp64",
                                                        workspace=ws)

    seq_k12_ms = timed(seq_k12, n=1, w=1)
    seq_k3_ms = timed(seq_k3, n=1, w=0)
    d = (out.double() - ref).abs()
    l1 = max(float((d[row[g]:row[g + 1], j].sum() / ref[row[g]:row[g + 1], j].abs().sum()))
             for g in range(n_graphs) for j in range(nrhs))
    nz = ref != 0
    # the iteration kernel's roofline: per iteration the packed entries, column
    # ends, 1/d_out and the nrhs-wide rows of X gathered once and written once
    nnzs = [nnz_of(gr) for gr in graphs]
    b_iter = sum(4 * z + 4 * (gr.N + 1) + 4 * gr.N + 2 * 4 * nrhs * gr.N for z, gr in zip(nnzs, graphs))
    iter_ms = (k3_ms - k3_setup_ms) / ITERS
    peak, peak_kind = _peaks()
    roof = {"bound": "hbm", "kernel": "k3b iterate_vec_kernel (one launch per iteration over all graphs)",
            "achieved": b_iter / (iter_ms * 1e-3) / 1e9, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
            "frac": b_iter / (iter_ms * 1e-3) / 1e9 / peak,
            "per_launch": {"bytes": b_iter, "ms": iter_ms,
                           "how": "(Kernel 3 stage, stream launches - the same call with 0 iterations) / "
                                  "iterations; bytes: 4 nnz + 8 N + 8 nrhs N per graph (entries, column ends, "
                                  "1/d_out, the nrhs-wide rows gathered once and written once)"}}
    seq_ms = seq_k12_ms + seq_k3_ms
    return {"graphs": n_graphs, "scales": "%d..%d" % (lo, hi), "start_vectors": nrhs, "edges": edges,
            "pipeline_ms": pipe_ms, "launch": "Kernels 1-3 recorded once as one CUDA graph and replayed",
            "pipeline_edge_vectors_per_s": ITERS * edges * nrhs / (pipe_ms * 1e-3),
            "pipeline_equals_stage_calls": same,
            "stages": {"k1_sort_ms": k1_ms, "k1_edges_per_s": edges / (k1_ms * 1e-3),
                       "k2_filter_ms": k2_ms, "k2_edges_per_s": edges / (k2_ms * 1e-3),
                       "k3_pagerank_ms": k3_ms, "k3_graph_replay_ms": k3_graph_ms,
                       "k3_edge_vectors_per_s": ITERS * edges * nrhs / (k3_ms * 1e-3)},
            "sequential": {"k1_k2_ms": seq_k12_ms, "k3_fp64_ms": seq_k3_ms, "total_ms": seq_ms,
                           "what": "64 single-graph Kernel 1 + Kernel 2 calls, then 2048 single-vector binary64 "
                                   "Kernel 3 runs"},
            "speedup_vs_sequential": seq_ms / pipe_ms,
            "max_l1_err_vs_fp64": l1, "max_rel_err_vs_fp64": float((d[nz] / ref[nz].abs()).max()),
            "roofline": roof, "device_error": pp.last_device_error()}


def cpu_baseline(scale, seed, max_seconds=20.0, sample_div=16):
    """The oracle, single-threaded, on the first M/sample_div edges of the same edge list."""
    import kernel0
    import oracle

    N = 1 << scale
    Ms = (16 * N) // sample_div
    u, v = kernel0.edges_host(scale, seed, M=Ms)
    r0 = kernel0.r0_host(N, seed)
    O = oracle.default()
    t0 = time.perf_counter()
    us, vs = O.k1_sort(u, v)
    t1 = time.perf_counter()
    R = O.k2_filter(us, vs, N)
    t2 = time.perf_counter()
    O.k3_pagerank(R, r0, ITERS, DAMPING)
    t3 = time.perf_counter()
    return {"value": Ms / (t3 - t0), "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": "first %d of the %d scale-%d edges (1/%d), N=2^%d, K1+K2+K3 (20 iterations, binary64)"
                      % (Ms, 16 * N, scale, sample_div, scale),
            "seconds": t3 - t0, "host_cores": os.cpu_count(),
            "kernels": {"k1_edges_per_s": Ms / (t1 - t0), "k2_edges_per_s": Ms / (t2 - t1),
                        "k3_edges_per_s": ITERS * Ms / (t3 - t2)}}


def run_reference(args):
    """The CPU oracle as the reference arm: each step is the oracle pipeline on a sample."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import kernel0
    import oracle

    scale = args.scale
    N = 1 << scale
    sample_div = 64
    Ms = (16 * N) // sample_div
    u, v = kernel0.edges_host(scale, SEED, M=Ms)
    r0 = kernel0.r0_host(N, SEED)
    O = oracle.default()

    def step():
        us, vs = O.k1_sort(u, v)
        R = O.k2_filter(us, vs, N)
        O.k3_pagerank(R, r0, ITERS, DAMPING)

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    val = Ms / (ms * 1e-3)
    sample = "first %d of the %d scale-%d edges (1/%d), N=2^%d, K1+K2+K3 binary64" % (Ms, 16 * N, scale, sample_div,
                                                                                      scale)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "scale": scale, "sample": sample},
        "cpu_baseline": {"value": val, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--dtype", choices=["fp32", "fp64", "bf16", "fp16"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle", action="store_true",
                    help="skip the errors against the oracle run on the whole graph (a few minutes of one host core)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-batched", action="store_true", help="skip the batched Kernel 3 section")
    ap.add_argument("--no-files", action="store_true", help="skip the edge-file (Kernel 1 with files) section")
    ap.add_argument("--tune", action="append", default=[], metavar="KEY=VALUE",
                    help="set a library tuning knob before running (repeatable)")
    ap.add_argument("--stage", choices=["all", "k1", "k2", "k3", "gather-ceiling", "batched"], default="all",
                    help="k1 / k2 / k3: time one kernel alone (profiling aid); the default times the whole pipeline")
    ap.add_argument("--log", default=None, metavar="FILE",
                    help="also append the result line to FILE (JSON lines, one per run)")
    ap.add_argument("--tuning", default="default",
                    help="autotuner result to apply (JSON from paper_1603_01876_gb300.tune; 'none' to skip)")
    args = ap.parse_args()
    args.tuned = {}
    if args.impl == "ours" and args.tuning != "none":
        from paper_1603_01876_gb300 import tune

        args.tuned = tune.apply(tune.DEFAULT_PATH if args.tuning == "default" else args.tuning, scale=args.scale)
    if args.tune:
        import paper_1603_01876_gb300 as pp

        for kv in args.tune:
            k, v = kv.split("=")
            pp.set_tuning(k, int(v))
    if args.stage in ("k1", "k2"):
        run_k1_k2_only(args)
    elif args.stage in ("k3", "gather-ceiling"):
        # Kernel 3 alone, with the gather ceiling of an iteration on the same graph
        run_k3_only(args)
    elif args.stage == "batched":
        import torch

        print(json.dumps({"stage": "batched", **run_batched(torch.device("cuda", 0), args.steps, args.warmup)}))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
