"""Autotuner for Kernel 3's work split (the knobs of pp_set_tuning).

The threshold that decides which columns are cut into chunks (the others
are summed one per lane in 32-column slices), how long a chunk is, plus the
unroll depth and the register budget, are measured on the GPU at hand: each setting runs the
20-iteration Kernel 3 on a graph of the requested scale (CUDA events, after
warm-up) and the fastest setting is kept.  The single-vector search is a
coordinate descent over the knobs (two rounds), the batched one a full grid.

    python -m paper_1603_01876_gb300.tune --scales 20,24,26 --out paper_1603_01876_gb300/tuning/gb300.json

The file keeps one entry per searched scale.  apply(path, scale=S) sets the
knobs of the entry for scale S (the nearest searched scale at or below it)
in the library, if the file was measured on a GPU of the same name.  Every setting gives results within the stated
tolerances; the thresholds only change the order of some column sums.
"""
import argparse
import json
import os
import time

SINGLE_KNOBS = {
    "k3_shortmax": [128, 256, 512],
    "k3_chunk": [2048, 4096],
    "k3_minblocks": [4, 6, 8],
    "k3_unroll_f32": [4, 8],
}
BATCH_KNOBS = {
    "k3b_vec": [1, 0],
    "k3b_shortmax": [128, 256],
    "k3b_chunk": [256, 512, 1024],
}
DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning", "gb300.json")


def _time_ms(fn, reps, warmup):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record()
    for _ in range(reps):
        fn()
    e[1].record()
    torch.cuda.synchronize()
    return e[0].elapsed_time(e[1]) / reps


def _with_knobs(pp, knobs, fn):
    old = {k: pp.get_tuning(k) for k in knobs}
    try:
        for k, v in knobs.items():
            pp.set_tuning(k, v)
        return fn()
    finally:
        for k, v in old.items():
            pp.set_tuning(k, v)


def tune_single(graph, r0, iters=20, c=0.85, dtype="fp32", reps=3, warmup=1, knobs=None, rounds=2, log=print):
    """Coordinate descent over `knobs` (default SINGLE_KNOBS) for one graph."""
    import torch

    import paper_1603_01876_gb300 as pp

    knobs = dict(SINGLE_KNOBS if knobs is None else knobs)
    if dtype == "fp64":
        knobs.pop("k3_unroll_f32", None)
        knobs.setdefault("k3_unroll_f64", [4, 8])
    ws = torch.empty(pp.workspace_bytes("pagerank", graph.M, graph.scale, iters, dtype), dtype=torch.uint8,
                     device=r0.device)
    out = torch.empty(graph.N, dtype=torch.float64 if dtype == "fp64" else torch.float32, device=r0.device)
    best = {k: pp.get_tuning(k) for k in knobs}
    seen = {}

    def measure(setting):
        key = tuple(sorted(setting.items()))
        if key not in seen:
            run = lambda: pp.pagerank(graph, r0, iters, c, dtype, out=out, workspace=ws)
            seen[key] = _with_knobs(pp, setting, lambda: _time_ms(run, reps, warmup))
            if log:
                log("  %s  %.3f ms" % (" ".join("%s=%d" % kv for kv in key), seen[key]))
        return seen[key]

    best_ms = measure(best)
    for _ in range(rounds):
        changed = False
        for k, values in knobs.items():
            for v in values:
                trial = dict(best, **{k: v})
                ms = measure(trial)
                if ms < best_ms * 0.995:
                    best, best_ms, changed = trial, ms, True
        if not changed:
            break
    return {"knobs": best, "ms": best_ms, "trials": len(seen)}


def tune_batched(graphs, r0, nrhs, iters=20, c=0.85, reps=3, warmup=1, knobs=None, log=print):
    """Full grid over `knobs` (default BATCH_KNOBS) for the batched Kernel 3."""
    import itertools

    import torch

    import paper_1603_01876_gb300 as pp

    knobs = dict(BATCH_KNOBS if knobs is None else knobs)
    out = torch.empty(r0.shape, dtype=torch.float32, device=r0.device)
    best, best_ms = None, float("inf")
    for values in itertools.product(*knobs.values()):
        setting = dict(zip(knobs.keys(), values))
        run = lambda: pp.pagerank_batched(graphs, r0, nrhs, iters, c, out=out)
        ms = _with_knobs(pp, setting, lambda: _time_ms(run, reps, warmup))
        if log:
            log("  %s  %.3f ms" % (" ".join("%s=%d" % kv for kv in setting.items()), ms))
        if ms < best_ms:
            best, best_ms = setting, ms
    return {"knobs": best, "ms": best_ms, "trials": len(list(itertools.product(*knobs.values())))}


def entry_for_scale(data, scale):
    """The stored single-graph entry for this scale: the exact scale if it was
    searched, else the nearest searched scale below it (the smallest one for
    smaller graphs)."""
    single = data.get("single", {})
    if "knobs" in single:  # a file with one entry
        return single
    scales = sorted(int(k) for k in single)
    if not scales:
        return {}
    below = [x for x in scales if x <= scale] if scale is not None else []
    pick = below[-1] if below else (scales[0] if scale is not None else max(scales))
    if scale is None and 24 in scales:
        pick = 24
    return single[str(pick)]


def apply(path=DEFAULT_PATH, device=None, scale=None):
    """Set the knobs stored in `path` for graphs of this scale (the entry of
    the nearest searched scale; scale None: the scale-24 entry), if the file
    was measured on this GPU's model; returns the knobs set (empty if the
    file is missing or for another GPU)."""
    import torch

    import paper_1603_01876_gb300 as pp

    if not path or not os.path.exists(path):
        return {}
    with open(path) as f:
        data = json.load(f)
    name = torch.cuda.get_device_name(device)
    if data.get("device") != name:
        return {}
    knobs = dict(entry_for_scale(data, scale).get("knobs", {}))
    knobs.update(data.get("batched", {}).get("knobs", {}))
    for k, v in knobs.items():
        pp.set_tuning(k, v)
    return knobs


def _graph(scale, seed, dev):
    import torch

    import kernel0
    import paper_1603_01876_gb300 as pp

    u, v = kernel0.edges_device(scale, seed, device=dev)
    us, vs = pp.sort_edges(u, v, scale)
    del u, v
    g = pp.build_filter_normalize(us, vs, scale, "lowest")
    del us, vs
    torch.cuda.empty_cache()
    return g, torch.from_numpy(kernel0.r0_host(1 << scale, seed)).to(dev)


def main(argv=None):
    import torch

    import kernel0
    import paper_1603_01876_gb300 as pp

    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--scales", default="20,24,26", help="graph scales to search, comma-separated")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--out", default=DEFAULT_PATH)
    args = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    t0 = time.time()
    result = {"device": torch.cuda.get_device_name(dev), "iters": 20, "single": {}}
    for scale in [int(x) for x in args.scales.split(",")]:
        g, r0 = _graph(scale, args.seed, dev)
        print("single-vector Kernel 3, binary32, scale %d" % scale)
        ent = tune_single(g, r0, reps=args.reps)
        print("single-vector Kernel 3, binary64 unroll, scale %d" % scale)
        shared = {k: v for k, v in ent["knobs"].items() if k != "k3_unroll_f32"}
        f64 = _with_knobs(pp, shared, lambda: tune_single(g, r0, dtype="fp64", reps=max(1, args.reps - 1),
                                                          knobs={"k3_unroll_f64": [4, 8]}))
        ent["knobs"]["k3_unroll_f64"] = f64["knobs"]["k3_unroll_f64"]
        ms = {"fp32": ent.pop("ms"), "fp64": f64["ms"]}
        ent["ms_20_iterations"] = ms
        ent["edges"] = g.M
        result["single"][str(scale)] = ent
        del g, r0
        torch.cuda.empty_cache()
    if not args.no_batched:
        print("batched Kernel 3: 64 graphs of scales 12..18, 32 start vectors")
        scales = kernel0.batch_scales(64, 12, 18, seed=args.seed)
        graphs = []
        for i, s in enumerate(scales):
            a, b = kernel0.edges_device(s, args.seed, graph=i, device=dev)
            sa, sb = pp.sort_edges(a, b, s)
            graphs.append(pp.build_filter_normalize(sa, sb, s))
        import numpy as np

        r0b = np.concatenate([np.stack([kernel0.r0_host(1 << s, args.seed, graph=i, rhs=j) for j in range(32)],
                                       axis=1) for i, s in enumerate(scales)])
        result["batched"] = tune_batched(graphs, torch.from_numpy(r0b).to(dev), 32, reps=args.reps)
    result["seconds"] = round(time.time() - t0, 1)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    with open(args.out, "w") as f:
        json.dump(result, f, indent=1, sort_keys=True)
    print(json.dumps(result))


if __name__ == "__main__":
    main()
