#!/usr/bin/env python3
"""Throughput of direct-search interval lookup on GB300.

Default workload (the largest single-GPU configuration): batched learned
lookup fused with linear interpolation, float32, 256 arrays of 2^10..2^22
knots with mixed gap laws (127.7M knots), 2^28 queries in proportion to the
array sizes, int32 index and float32 interpolant per query.  One step is one
search pass over all queries (the paper's Algorithm harness: tables are built
before the clock starts; the build is timed separately in the same run).  The
same run measures workloads 1-4 (``per_config``): lookups/s, the fraction of
the HBM peak and the mismatches of every result against the definition.

Prints ONE JSON line (rank 0).  Multi-GPU (torchrun): every rank builds its
own replica and searches its own queries (weak scaling, no collective on the
data path).

--impl reference times the CPU oracle on a bounded sample of the same
workload on the host cores.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = ("direct_f64", "direct_f64_sorted", "direct_f32", "batched_f32", "learned_f64", "learned_interp_f32",
             "gapq_f64", "paper_tables")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="learned_interp_f32", choices=WORKLOADS)
    p.add_argument("--cells-per-knot", type=float, default=0.0,
                   help="learned workloads: cells of the learned cell map per knot (0: the library's default)")
    p.add_argument("--arrays", type=int, default=0,
                   help="learned + interpolation workload: number of arrays (profiling runs; default 256)")
    p.add_argument("--no-per-config", action="store_true",
                   help="skip the per-configuration figures of workloads 1-4 (default run only)")
    p.add_argument("--variant", default="plain", choices=["plain", "fma", "cache", "fma_cache", "gap2", "fma_gap2"])
    p.add_argument("--no-extras", action="store_true", help="skip the secondary measurements")
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="target CPU time of the oracle baseline")
    p.add_argument("--queries", type=int, default=0, help="override the query count (profiling runs)")
    p.add_argument("--tune", default="auto",
                   help="batched/learned launch configuration: auto (autotuned), default (the library's), "
                        "or block,items,smem_limit")
    p.add_argument("--record-traffic", default="", metavar="NCU_CSV",
                   help="write the timed kernel's DRAM bytes per launch from an ncu CSV to profiles/traffic.json "
                        "(no GPU needed; give the --workload/--variant/--queries of the captured run)")
    return p.parse_args()


# ----------------------------------------------------------------------------- helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the sources each timed kernel is compiled from (a capture stays valid while they are unchanged)
_COMMON = ["ds_common.cuh", "ds_search.cuh", "ds_index.cuh"]
KERNEL_SOURCES = {
    "search": _COMMON + ["ds_search_impl.cuh", "ds_search_f32.cu", "ds_search_f64.cu", "ds_build.cu"],
    "batch": _COMMON + ["ds_multi.cuh", "ds_multi_kernels.cuh", "ds_engine.cuh", "ds_batch.cu"],
    "learned": _COMMON + ["ds_multi.cuh", "ds_multi_kernels.cuh", "ds_engine.cuh", "ds_batch.cu", "ds_learned.cu"],
}


def _code_of(text):
    """The source without its comments and blank space (a comment edit leaves a capture valid)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_hash(kernel_key):
    family = kernel_key.split("_")[0]
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(family, KERNEL_SOURCES["search"]):
        h.update(_code_of(open(os.path.join(ROOT, "paper_1506_08620_gb300", "csrc", f)).read()).encode())
    return h.hexdigest()[:16]


TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")


def traffic_for(kernel_key):
    """Per-launch DRAM bytes from a committed ncu capture, if it was taken on the
    current kernel sources; else None."""
    if not os.path.exists(TRAFFIC_PATH):
        return None
    d = json.load(open(TRAFFIC_PATH))
    e = d.get(kernel_key)
    if not e or e.get("source_hash") != source_hash(kernel_key):
        return None
    return e.get("bytes_per_search", e.get("bytes_per_launch"))


def kernel_key_of(args):
    if args.workload.startswith("direct"):
        return "search_%s_%s" % ("f32" if args.workload == "direct_f32" else "f64", args.variant)
    return {"gapq_f64": "search_f64_gapq", "paper_tables": "search_f64_paper_layout",
            "batched_f32": "batch_search_f32", "learned_f64": "learned_search_f64",
            "learned_interp_f32": "learned_search_f32"}[args.workload]


def record_traffic(args):
    """DRAM traffic per search call from an ncu CSV (--metrics
    dram__bytes_read.sum,dram__bytes_write.sum of a run with --queries Q over
    whole search calls: the chunk planner and one or two search kernels for the
    batched and learned forms, one kernel otherwise), scaled to the full
    workload by the query count, into profiles/traffic.json."""
    import csv
    scale_unit = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    per_launch, names = {}, {}
    with open(args.record_traffic) as f:
        lines = [l for l in f if l.startswith('"')]
    for row in csv.DictReader(lines):
        if row.get("Metric Name") not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        v = float(row["Metric Value"].replace(",", "")) * scale_unit.get(row.get("Metric Unit", "byte"), 1)
        per_launch[row["ID"]] = per_launch.get(row["ID"], 0.0) + v
        names[row["ID"]] = row.get("Kernel Name", "")
    if not per_launch or not args.queries:
        raise SystemExit("record-traffic: no dram__bytes rows in %s, or --queries not given" % args.record_traffic)
    # one planner launch per search call where there is a planner; else one launch per call
    calls = sum(1 for n in names.values() if n.startswith("k_plan_chunks")) or len(per_launch)
    captured = sum(per_launch.values()) / calls
    by_kernel = {}
    for i, n in names.items():
        short = n.split("(")[0]
        by_kernel[short] = by_kernel.get(short, 0.0) + per_launch[i] / calls
    full = workload_config(argparse.Namespace(**{**vars(args), "queries": 0}))["queries"]
    key = kernel_key_of(args)
    d = json.load(open(TRAFFIC_PATH)) if os.path.exists(TRAFFIC_PATH) else {}
    d[key] = {"bytes_per_search": captured * full / args.queries, "captured_bytes_per_search": captured,
              "captured_bytes_per_kernel": by_kernel,
              "captured_queries": args.queries, "full_queries": full, "launches": len(per_launch),
              "searches": calls,
              "scaled": ("captured at the full workload" if args.queries == full else
                         "traffic grows in proportion to the queries (tables L2-resident)"),
              "source_hash": source_hash(key)}
    with open(TRAFFIC_PATH, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps({key: d[key]}))


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value, dist=None, device=None):
    """The largest of `value` over all ranks (all ranks get it).  The only
    collective of the multi-GPU run: every rank searches its own replica and
    its own queries, so nothing else is exchanged."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(W, workload_id, rank):
    """Seed of a rank's replica workload: rank 0 uses the workload's own seed,
    other ranks draw independent queries (and knots) of the same recipe."""
    return None if rank == 0 else W.SEED_BASE + workload_id + 1000 * rank


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The reference arm: the oracle as it stands (the definition of the answer,
    and for the interpolating workload the float64 interpolant), single-threaded
    on the host, on a bounded sample of the same workload per step."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle
    oracle.lib()
    step, n, desc, dtype = reference_sample(args)
    for _ in range(max(args.warmup, 0)):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    value = n / t
    line = {"impl": "reference", "metric": "lookups/s", "value": value, "unit": "lookups/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": "lookups/s", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "lookups/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reference_sample(args, n=1 << 20):
    """(one step of the oracle, queries per step, description, dtype) on a
    bounded sample of the workload: the same knots, fewer queries of the same
    distribution."""
    import oracle
    from paper_1506_08620_gb300 import workloads as W
    if args.workload in ("learned_interp_f32", "batched_f32"):
        five = args.workload == "learned_interp_f32"
        w = W.workload5(total_queries=2 * n) if five else W.workload3(total_queries=4 * n)
        if five:
            step = lambda: oracle.interp_batch(w["Xcat"], w["Ycat"], w["x_off"], w["Zcat"], w["z_off"])
        else:
            step = lambda: oracle.upper_bound_batch(w["Xcat"], w["x_off"], w["Zcat"], w["z_off"])
        return (step, w["Zcat"].size, "%d queries of workload %s (same arrays), one pass per step"
                % (w["Zcat"].size, w["name"]), "f32")
    if args.workload.startswith("direct_f64"):
        w = W.workload2(m=n, sort=args.workload.endswith("sorted"))
    elif args.workload in ("learned_f64", "gapq_f64"):
        w = W.workload4(m=n)
    elif args.workload == "paper_tables":
        w = W.paper_layout(PAPER_SIZES[-1], n, np.float64)
    else:
        w = W.workload1()
    X, Z = w["X"], w["Z"]
    return (lambda: oracle.upper_bound(X, Z), Z.size,
            "%d queries of workload %s (same knots), one pass per step" % (Z.size, w["name"]),
            "f64" if X.dtype == np.float64 else "f32")


def cpu_baseline(X, Z, seconds):
    """The oracle (single thread) on a bounded sample sized for ~`seconds`."""
    import oracle
    oracle.lib()
    n = min(Z.size, 1 << 16)
    t0 = time.perf_counter()
    oracle.upper_bound(X, Z[:n])
    rate = n / max(time.perf_counter() - t0, 1e-9)
    n = int(min(Z.size, max(1 << 16, rate * seconds)))
    t0 = time.perf_counter()
    oracle.upper_bound(X, Z[:n])
    dt = time.perf_counter() - t0
    res = {"value": n / dt, "unit": "lookups/s", "cores": 1, "kind": "oracle",
           "sample": "first %d of the %d queries, one pass, %.1f s" % (n, Z.size, dt)}
    # the same oracle on every host core: a static partition of the sample, one
    # slice per thread (the C calls run without the interpreter lock)
    cores = os.cpu_count() or 1
    if cores > 1:
        import concurrent.futures as cf
        parts = np.array_split(np.arange(n), cores)
        with cf.ThreadPoolExecutor(cores) as ex:
            t0 = time.perf_counter()
            list(ex.map(lambda idx: oracle.upper_bound(X, Z[idx[0]:idx[-1] + 1]) if idx.size else None, parts))
            dt_all = time.perf_counter() - t0
        res["all_cores"] = {"value": n / dt_all, "cores": cores}
    # the paper's method on the host: the oracle's own Algorithm direct (scalar,
    # one thread) with its own table, on the same sample, where it is feasible
    try:
        hr, K = oracle.build_table(X)
    except ValueError:
        return res
    t0 = time.perf_counter()
    oracle.direct(X, K, hr["H"], hr["W"], hr["R"], Z[:n])
    res["direct_oracle_lookups_per_s"] = n / (time.perf_counter() - t0)
    return res


def workload_config(args):
    base = {
        "direct_f64": {"workload": "direct search f64: 2^20+1 knots, lognormal(0,0.5) gaps, 2^27 uniform queries",
                       "knots": (1 << 20) + 1, "queries": 1 << 27},
        "direct_f64_sorted": {"workload": "direct search f64: 2^20+1 knots, lognormal(0,0.5) gaps, "
                                          "2^27 sorted uniform queries", "knots": (1 << 20) + 1, "queries": 1 << 27},
        "direct_f32": {"workload": "direct search f32: 1025 knots, 1,002,048 queries tiled 512x into one stream",
                       "knots": 1025, "queries": 1002048 * 512},
        "batched_f32": {"workload": "batched direct search f32: 4096 arrays of 16..65536 knots (log-uniform), "
                                    "2^28 queries in proportion, CSR, one persistent launch", "arrays": 4096,
                        "queries": 1 << 28},
        "learned_f64": {"workload": "learned index f64: 2^24+1 knots, gaps U[1e-3,1e-2] or (1%) U[1e3,1e4], "
                                    "2^27 uniform queries, 1-32-32-1 MLP + bounded window", "knots": (1 << 24) + 1,
                        "queries": 1 << 27},
        "gapq_f64": {"workload": "Gap-q direct search f64 on the learned-index data: 2^24+1 knots, gaps "
                                 "U[1e-3,1e-2] or (1%) U[1e3,1e4], 2^27 uniform queries; smallest q whose table "
                                 "fits 4 GiB", "knots": (1 << 24) + 1, "queries": 1 << 27, "budget_bytes": 1 << 32},
        "paper_tables": {"workload": "direct search vs the logarithmic searches of Section 3 on the paper's layout "
                                     "(gaps U[1,5], queries at interval midpoints), N+1 = 15 .. 1048575, f32 and f64, "
                                     "2^26 queries per launch; the timed step is Direct f64 at 1048575 knots",
                         "queries": 1 << 26},
        "learned_interp_f32": {"workload": "batched learned lookup + linear interpolation f32: 256 arrays of "
                                           "2^10..2^22 knots, mixed gap laws, 2^28 queries", "arrays": 256,
                               "queries": 1 << 28},
    }.get(args.workload, {"workload": args.workload})
    base = dict(base)
    base["variant"] = args.variant
    if args.queries:
        base["queries"] = args.queries
    base["l2"] = "inputs larger than L2 (queries and results stream from HBM every step)"
    base["step"] = "one search pass over all queries; table built before the clock (Algorithm harness)"
    return base


# ----------------------------------------------------------------------------- our arm
class Job:
    """One timed workload: search() runs one step on device-resident inputs;
    e2e() runs one step through the public API from pinned host memory."""
    kernel_key = ""
    dtype_name = ""
    launches_per_step = 1
    bytes_per_lookup = 0
    m = 0
    build_ms = 0.0
    table = None
    extras = None


def setup_direct(args, ds, W, torch, dev, rank):
    job = Job()
    variants = {"plain": 0, "fma": ds.DS_FMA, "cache": ds.DS_CACHE_LAYOUT,
                "fma_cache": ds.DS_FMA | ds.DS_CACHE_LAYOUT, "gap2": ds.DS_GAP2, "fma_gap2": ds.DS_FMA | ds.DS_GAP2}
    flags = variants[args.variant]
    if args.workload in ("direct_f64", "direct_f64_sorted"):
        w = W.workload2(seed=rank_seed(W, 2, rank), m=args.queries or (1 << 27),
                        sort=args.workload.endswith("sorted"))
        X, Zh = w["X"], w["Z"]
        job.bytes_per_lookup, job.dtype_name = 8 + 4, "f64"
    else:
        w = W.workload1()
        X = w["X"]
        Zh = np.tile(w["Z"], 512)
        if args.queries:
            Zh = Zh[: args.queries]
        job.bytes_per_lookup, job.dtype_name = 4 + 4, "f32"
    job.m = Zh.size
    Xd = torch.from_numpy(X).to(dev)
    Zd = torch.from_numpy(Zh).to(dev)
    out = torch.empty(job.m, dtype=torch.int32, device=dev)
    builds = []
    for k in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        idx = ds.ds_build(Xd, flags)
        torch.cuda.synchronize()
        builds.append((time.perf_counter() - t0) * 1e3)
        if k < 2:
            idx.free()
    job.build_ms = float(np.median(builds))
    info = idx.info()
    job.table = {"H": info["H"], "R": info["R"], "table_bytes": info["table_bytes"],
                 "smem_resident": info["smem_resident"], "h_updates": info["h_updates"]}
    job.kernel_key = "search_%s_%s" % (job.dtype_name, args.variant)
    job.search = lambda: ds.ds_search(idx, Zd, out)
    job.out = out
    job.keep = (idx, Xd, Zd)
    pinned = {}

    def e2e():
        if not pinned:
            pinned["Z"] = torch.from_numpy(Zh).pin_memory()
            pinned["I"] = torch.empty(job.m, dtype=torch.int32).pin_memory()
            job.e2e_out = pinned["I"]
        Zp, Ip = pinned["Z"], pinned["I"]
        ds.ds_search_host(idx, Zp, Ip)
        return Zp.numel() * Zp.element_size(), Ip.numel() * 4
    job.e2e = e2e

    job.verify = lambda: answer_check(torch, job.search, Xd, Zd, out)

    def extras(stream):
        res = {}
        for name, fl in variants.items():
            if name == args.variant:
                continue
            j = ds.ds_build(Xd, fl)
            res[name] = job.m / time_calls(torch, stream, lambda: ds.ds_search(j, Zd, out), 5)
            if fl & ds.DS_GAP2:
                res[name + "_table_bytes"] = j.info()["table_bytes"]
            j.free()
        # end to end through the chunked copy pipeline instead of in-place host access
        os.environ["DS_HOST_PIPE"] = "1"
        try:
            ds.ds_search_host(idx, Zp, Ip)
            t0 = time.perf_counter()
            for _ in range(3):
                ds.ds_search_host(idx, Zp, Ip)
            res["e2e_copy_pipeline"] = job.m / ((time.perf_counter() - t0) / 3)
        finally:
            del os.environ["DS_HOST_PIPE"]
        if args.workload == "direct_f32":
            # the paper's harness: the 1,002,048 queries of one copy, searched
            # back to back (L2-resident, not an HBM figure), and one launch alone
            m1 = w["Z"].size
            Z1, o1 = Zd[:m1], out[:m1]
            res["paper_harness_host_loop"] = m1 / time_calls(torch, stream, lambda: ds.ds_search(idx, Z1, o1), 20)
            reps = 50  # back to back in one CUDA graph, as the harness repeats its queries
            gs = torch.cuda.Stream()
            gs.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(gs):
                ds.ds_search(idx, Z1, o1, stream=gs)
            torch.cuda.current_stream().wait_stream(gs)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=gs):
                for _ in range(reps):
                    ds.ds_search(idx, Z1, o1, stream=gs)
            graph.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(4):
                graph.replay()
            e1.record()
            torch.cuda.synchronize()
            res["paper_harness_l2_resident"] = 4 * reps * m1 / (e0.elapsed_time(e1) * 1e-3)
            del graph
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ds.ds_search(idx, Z1, o1)
            e1.record(stream)
            torch.cuda.synchronize()
            res["single_launch_us"] = e0.elapsed_time(e1) * 1e3
        if args.workload == "direct_f64":
            Zs = torch.sort(Zd).values
            res["sorted_queries_" + args.variant] = job.m / time_calls(torch, stream,
                                                                       lambda: ds.ds_search(idx, Zs, out), 5)
            # the O(M + N) merge of sorted queries into X (no table)
            res["sorted_queries_merge"] = job.m / time_calls(torch, stream,
                                                             lambda: ds.ds_search_sorted(Xd, Zs, out), 5)
            del Zs
            # counts per interval, fused with the search (N+2 uint64 counters)
            counts = torch.zeros(Xd.numel() + 1, dtype=torch.int64, device=dev)
            res["histogram"] = job.m / time_calls(torch, stream, lambda: ds.ds_histogram(idx, Zd, counts), 5)
            del counts
        return res
    job.extras = extras
    return job


def setup_gapq(args, ds, W, torch, dev, rank):
    """Gap-q (Section 4.7) on the two-scale data where Direct overflows: the
    network-free comparator of the learned index."""
    job = Job()
    w = W.workload4(seed=rank_seed(W, 4, rank), m=args.queries or (1 << 27))
    X, Zh = w["X"], w["Z"]
    job.bytes_per_lookup, job.dtype_name = 8 + 4, "f64"
    job.m = Zh.size
    Xd = torch.from_numpy(X).to(dev)
    Zd = torch.from_numpy(Zh).to(dev)
    out = torch.empty(job.m, dtype=torch.int32, device=dev)
    budget = 1 << 32
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    idx = ds.ds_build_q(Xd, 0, budget, q_max=1024)
    torch.cuda.synchronize()
    job.build_ms = (time.perf_counter() - t0) * 1e3
    info = idx.info()
    job.table = {"q": info["gap_q"], "H": info["H"], "R": info["R"], "table_bytes": info["table_bytes"],
                 "h_updates": info["h_updates"], "build_includes_choice_of_q": True}
    job.kernel_key = "search_f64_gapq"
    job.search = lambda: ds.ds_search(idx, Zd, out)
    job.out = out
    job.keep = (idx, Xd, Zd)
    job.verify = lambda: answer_check(torch, job.search, Xd, Zd, out)
    Zp = torch.from_numpy(Zh).pin_memory()
    Ip = torch.empty(job.m, dtype=torch.int32).pin_memory()

    def e2e():
        ds.ds_search_host(idx, Zp, Ip)
        return Zp.numel() * Zp.element_size(), Ip.numel() * 4
    job.e2e = e2e
    job.e2e_out = Ip

    def extras(stream):
        res = {}
        for q in (64, 128, 512, 1024):
            if q == info["gap_q"]:
                continue
            j = ds.ds_build_q(Xd, q)
            res["q%d" % q] = job.m / time_calls(torch, stream, lambda: ds.ds_search(j, Zd, out), 5)
            res["q%d_table_bytes" % q] = j.info()["table_bytes"]
            j.free()
        return res
    job.extras = extras
    return job


PAPER_SIZES = (15, 255, 4095, 65535, 1048575)


def setup_paper_tables(args, ds, W, torch, dev, rank):
    """The paper's throughput tables (size of X against method) on this GPU:
    direct search in its variants and the logarithmic searches, same queries."""
    job = Job()
    m = args.queries or (1 << 26)
    last = {}

    def layout(n, dtype):
        w = W.paper_layout(n, m, dtype, seed=rank_seed(W, 0, rank))
        return torch.from_numpy(w["X"]).to(dev), torch.from_numpy(w["Z"]).to(dev)

    X, Z = layout(PAPER_SIZES[-1], np.float64)
    out = torch.empty(m, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    idx = ds.ds_build(X)
    torch.cuda.synchronize()
    job.build_ms = (time.perf_counter() - t0) * 1e3
    info = idx.info()
    job.m = m
    job.bytes_per_lookup, job.dtype_name = 8 + 4, "f64"
    job.table = {"H": info["H"], "R": info["R"], "table_bytes": info["table_bytes"]}
    job.kernel_key = "search_f64_paper_layout"
    job.search = lambda: ds.ds_search(idx, Z, out)
    job.out = out
    job.keep = (idx, X, Z)
    job.verify = lambda: answer_check(torch, job.search, X, Z, out)
    Zp = Z.cpu().pin_memory()
    Ip = torch.empty(m, dtype=torch.int32).pin_memory()

    def e2e():
        ds.ds_search_host(idx, Zp, Ip)
        return Zp.numel() * 8, Ip.numel() * 4
    job.e2e = e2e
    job.e2e_out = Ip

    def extras(stream):
        direct = {"direct": 0, "direct_fma": ds.DS_FMA, "direct_cache": ds.DS_CACHE_LAYOUT, "direct_gap2": ds.DS_GAP2}
        res = {}
        for dtype in (np.float32, np.float64):
            tab = {}
            for n in PAPER_SIZES:
                Xn, Zn = layout(n, dtype)
                o = torch.empty(m, dtype=torch.int32, device=dev)
                row = {}
                for name, fl in direct.items():
                    h = ds.ds_build(Xn, fl)
                    row[name] = m / time_calls(torch, stream, lambda: ds.ds_search(h, Zn, o), 5) / 1e9
                    h.free()
                for meth, name in enumerate(ds.DS_LS_NAMES):
                    h = ds.ds_lsearch_build(Xn, meth)
                    row[name] = m / time_calls(torch, stream, lambda: ds.ds_lsearch_search(h, Zn, o), 5) / 1e9
                    h.free()
                row["direct_over_classic"] = row["direct"] / row["classic"]
                row["direct_over_best_log"] = row["direct"] / max(row[k] for k in ds.DS_LS_NAMES)
                tab[str(n)] = row
                del Xn, Zn, o
            res["G_lookups_per_s_" + ("f32" if dtype == np.float32 else "f64")] = tab
        return res
    job.extras = extras
    return job


def setup_batched(args, ds, W, torch, dev, rank):
    job = Job()
    w = W.workload3(seed=rank_seed(W, 3, rank), total_queries=args.queries or (1 << 28))
    job.dtype_name = "f32"
    job.m = int(w["z_off"][-1])
    Xd, xo = torch.from_numpy(w["Xcat"]).to(dev), torch.from_numpy(w["x_off"]).to(dev)
    Zd, zo = torch.from_numpy(w["Zcat"]).to(dev), torch.from_numpy(w["z_off"]).to(dev)
    out = torch.empty(job.m, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = ds.ds_batch_build(Xd, xo)
    torch.cuda.synchronize()
    job.build_ms = (time.perf_counter() - t0) * 1e3
    info = b.info()
    if args.tune == "auto":
        tune = ds.ds_batch_autotune(b, Zd, zo, out)
    elif args.tune == "default":
        tune = ds.ds_batch_get_tune(b)
    else:
        blk, items, smem = (int(v) for v in args.tune.split(","))
        ds.ds_batch_set_tune(b, blk, items, smem)
        tune = ds.ds_batch_get_tune(b)
    job.bytes_per_lookup = 8 + info["table_bytes"] / job.m
    job.table = {"arrays": info["n_arrays"], "R_total": info["R"], "table_bytes": info["table_bytes"],
                 "tune": tune}
    job.kernel_key = "batch_search_f32"
    job.launches_per_step = info["search_launches"]  # the planner and the search kernel
    job.search = lambda: ds.ds_batch_search(b, Zd, zo, out)
    job.out = out
    job.keep = (b, Xd, xo, Zd, zo)
    bufs = {}

    def e2e():
        if not bufs:
            bufs.update(Z=torch.from_numpy(w["Zcat"]).pin_memory(), I=torch.empty(job.m, dtype=torch.int32).pin_memory(),
                        z=torch.empty_like(Zd), o=torch.empty_like(out))
            job.e2e_out = bufs["I"]
        Zp, Ip = bufs["Z"], bufs["I"]
        bufs["z"].copy_(Zp, non_blocking=True)
        ds.ds_batch_search(b, bufs["z"], zo, bufs["o"])
        Ip.copy_(bufs["o"], non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return Zp.numel() * 4, Ip.numel() * 4
    job.e2e = e2e
    job.verify = lambda: answer_check(torch, job.search, Xd, Zd, out, xo, zo)

    def extras(stream):
        # the same engine without the knot fingerprints (every query in a cell
        # holding a knot reads the knot), autotuned the same way
        nf = ds.ds_batch_build(Xd, xo, ds.DS_NO_FINGERPRINT)
        t = ds.ds_batch_autotune(nf, Zd, zo, out)
        res = {"no_fingerprint": job.m / time_calls(torch, stream, lambda: ds.ds_batch_search(nf, Zd, zo, out), 5),
               "no_fingerprint_tune": t}
        nf.free()
        # plain Direct on the same arrays and queries: one table and one search
        # launch per array (4096 launches replayed from one CUDA graph), the
        # same-dtype comparison for the batched engine
        xo_h, zo_h = w["x_off"], w["z_off"]
        idxs = [ds.ds_build(Xd[xo_h[a]:xo_h[a + 1]]) for a in range(len(xo_h) - 1)]
        gs = torch.cuda.Stream()
        gs.wait_stream(torch.cuda.current_stream())
        # each array's queries copied to a 16-byte aligned segment (the vector path of ds_search)
        cnt = np.diff(zo_h)
        po = np.zeros(cnt.size + 1, dtype=np.int64)
        np.cumsum((cnt + 3) // 4 * 4, out=po[1:])
        Zp_d = torch.zeros(int(po[-1]), dtype=Zd.dtype, device=Zd.device)
        Op_d = torch.empty(int(po[-1]), dtype=torch.int32, device=Zd.device)
        for a in range(cnt.size):
            Zp_d[po[a]:po[a] + cnt[a]] = Zd[zo_h[a]:zo_h[a + 1]]
        views = [(Zp_d[po[a]:po[a] + cnt[a]], Op_d[po[a]:po[a] + cnt[a]]) for a in range(len(idxs))]
        with torch.cuda.stream(gs):
            for a, (zv, ov) in enumerate(views):
                if zv.numel():
                    ds.ds_search(idxs[a], zv, ov, stream=gs)
        torch.cuda.current_stream().wait_stream(gs)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            for a, (zv, ov) in enumerate(views):
                if zv.numel():
                    ds.ds_search(idxs[a], zv, ov, stream=gs)
        res["plain_direct_per_array_graph"] = job.m / time_calls(torch, stream, graph.replay, 5)
        res["plain_direct_per_array_launches"] = sum(1 for zv, _ in views if zv.numel())
        del graph
        torch.cuda.synchronize()
        for i in idxs:
            i.free()
        return res
    job.extras = extras
    return job


def setup_learned(args, ds, W, torch, dev, rank):
    """Workload 4 (one float64 array where direct search overflows) or
    workload 5 (256 float32 arrays, per-array selector, fused interpolation)."""
    job = Job()
    five = args.workload == "learned_interp_f32"
    if five:
        w = W.workload5(seed=rank_seed(W, 5, rank), total_queries=args.queries or (1 << 28),
                        n_arrays=args.arrays or 256)
        Xd, xo = torch.from_numpy(w["Xcat"]).to(dev), torch.from_numpy(w["x_off"]).to(dev)
        Yd = torch.from_numpy(w["Ycat"]).to(dev)
        Zh, zo = w["Zcat"], torch.from_numpy(w["z_off"]).to(dev)
        job.dtype_name = "f32"
    else:
        w = W.workload4(seed=rank_seed(W, 4, rank), m=args.queries or (1 << 27))
        Xd, xo, Yd, zo = torch.from_numpy(w["X"]).to(dev), None, None, None
        Zh = w["Z"]
        job.dtype_name = "f64"
    job.m = Zh.size
    Zd = torch.from_numpy(Zh).to(dev)
    out = torch.empty(job.m, dtype=torch.int32, device=dev)
    yout = torch.empty(job.m, dtype=Xd.dtype, device=dev) if five else None
    cfg = ds.ds_learned_cfg_default(n_queries=1 << 20) if not five else ds.ds_learned_cfg_default()
    cfg.cells_per_knot = args.cells_per_knot
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L = ds.ds_learned_build_xy(Xd, Yd, xo, cfg=cfg) if five else ds.ds_learned_build(Xd, cfg=cfg)
    torch.cuda.synchronize()
    job.build_ms = (time.perf_counter() - t0) * 1e3
    info = L.info()
    esz = 4 if five else 8
    # streamed: z in, i out (and y out); the interpolation also gathers X_i, X_{i+1}, Y_i, Y_{i+1}
    job.streamed_bytes_per_lookup = esz + 4 + (esz if five else 0)
    job.bytes_per_lookup = job.streamed_bytes_per_lookup + (4 * esz if five else 0)
    job.table = {k: info[k] for k in ("n_arrays", "n_direct", "n_learned", "n_fallback", "max_window",
                                      "train_steps", "train_ms", "final_loss", "table_bytes")}
    job.table["cells"] = [ds.ds_learned_cells(L, a) for a in range(info["n_arrays"])] if not five else None
    if args.tune == "auto":  # the same engine autotuner as the batched form
        job.table["tune"] = ds.ds_learned_autotune(L, Zd, zo, out, y_out=yout)
    elif args.tune != "default":
        blk, items, smem = (int(v) for v in args.tune.split(","))
        ds.ds_learned_set_tune(L, blk, items, smem)
        job.table["tune"] = ds.ds_learned_get_tune(L)
    job.kernel_key = "learned_search_%s" % job.dtype_name
    job.launches_per_step = info["search_launches"]  # the planner, then one or two search kernels
    if five:
        job.search = lambda: ds.ds_learned_search(L, Zd, zo, out=out, y_out=yout)
    else:
        job.search = lambda: ds.ds_learned_search(L, Zd, out=out)
    job.out = out
    job.keep = (L, Xd, Zd, Yd)
    job.yout = yout
    bufs = {}

    def e2e():
        # through the C ABI's host-buffer call: the kernel reads the queries from
        # and writes the results to pinned host memory over the CPU-GPU link
        if not bufs:
            bufs.update(Z=torch.from_numpy(Zh).pin_memory(), I=torch.empty(job.m, dtype=torch.int32).pin_memory(),
                        y=torch.empty(job.m, dtype=Xd.dtype).pin_memory() if five else None,
                        zo=torch.from_numpy(w["z_off"]) if five else None)
            job.e2e_out = bufs["I"]
        Zp, Ip, yp = bufs["Z"], bufs["I"], bufs["y"]
        ds.ds_learned_search_host(L, Zp, bufs["zo"], out=Ip, y_out=yp)
        return Zp.numel() * esz + (bufs["zo"].numel() * 8 if five else 0), Ip.numel() * 4 + (yp.numel() * esz if five else 0)
    job.e2e = e2e
    job.verify = lambda: answer_check(torch, job.search, Xd, Zd, out, xo, zo, Yd, yout)
    job.host = w

    def extras(stream):
        res = {}
        if not five:  # the model without the network, same search path
            lin = ds.ds_learned_build(Xd, cfg=ds.ds_learned_cfg_default(flags=ds.DS_LEARNED_LINEAR))
            if args.tune == "auto":
                ds.ds_learned_autotune(lin, Zd, None, out)
            res["linear_model"] = job.m / time_calls(torch, stream, lambda: ds.ds_learned_search(lin, Zd, out=out), 3)
            res["linear_model_max_window"] = lin.info()["max_window"]
            lin.free()
            # no network at all: Gap-q direct search (Section 4.7), smallest q with a table of at most 4 GiB
            gq = ds.ds_build_q(Xd, 0, 1 << 32, q_max=1024)
            res["gapq_direct"] = job.m / time_calls(torch, stream, lambda: ds.ds_search(gq, Zd, out), 3)
            res["gapq_q"] = gq.info()["gap_q"]
            res["gapq_table_bytes"] = gq.info()["table_bytes"]
            gq.free()
            # the paper's logarithmic fall-back over all knots (Section 3, LeadBit)
            lb = ds.ds_lsearch_build(Xd, ds.DS_LS_LEADBIT)
            res["leadbit_all_knots"] = job.m / time_calls(torch, stream, lambda: ds.ds_lsearch_search(lb, Zd, out), 3)
            lb.free()
        return res
    job.extras = extras
    return job


def time_calls(torch, stream, fn, n):
    for _ in range(2):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n * 1e-3


def answer_check(torch, search, Xd, Zd, I, xo=None, zo=None, Yd=None, y=None, chunk=1 << 25):
    """Mismatches of one step's results against the definition, at every
    position: the answer is the unique i with X_i <= z < X_{i+1} (-1 below
    X_0, N at or above X_N; the knots are strictly increasing), checked with
    plain tensor comparisons on the device.  With knot values, y is compared
    with the interpolant restated in float64 on those indices (tolerance
    1e-6 of max(|y64|, |Y_i|, |Y_{i+1}|))."""
    search()
    torch.cuda.synchronize()
    m = Zd.numel()
    bad = bad_y = 0
    for s in range(0, m, chunk):
        e = min(m, s + chunk)
        z, i = Zd[s:e], I[s:e].long()
        if zo is None:
            base = torch.zeros_like(i)
            n = torch.full_like(i, Xd.numel() - 1)
        else:
            arr = torch.searchsorted(zo, torch.arange(s, e, device=Zd.device), right=True) - 1
            base = xo[arr]
            n = xo[arr + 1] - base - 1
        mid = (i >= 0) & (i < n)
        g0 = base + i.clamp(min=0)
        g1 = torch.minimum(g0 + 1, base + n)
        ok = mid & (Xd[g0] <= z) & (z < Xd[g1])
        ok |= (i == -1) & (z < Xd[base])
        ok |= (i == n) & (z >= Xd[base + n])
        bad += int((~ok).sum())
        if y is not None:
            x0, x1, y0, y1 = Xd[g0].double(), Xd[g1].double(), Yd[g0].double(), Yd[g1].double()
            y64 = y0 + (y1 - y0) * ((z.double() - x0) / (x1 - x0))
            scale = torch.maximum(y64.abs(), torch.maximum(y0.abs(), y1.abs()))
            yy = y[s:e].double()
            ok_y = torch.where(mid, (yy - y64).abs() <= 1e-6 * scale, torch.isnan(yy))
            bad_y += int((~ok_y).sum())
    res = {"checked": "every result, against the definition (X_I <= z < X_{I+1})", "results": m,
           "mismatches": bad}
    if y is not None:
        res["y_outside_tolerance"] = bad_y
    return res


def main():
    args = parse()
    if args.record_traffic:
        return record_traffic(args)
    if args.impl == "reference":
        return run_reference(args)
    import torch
    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_1506_08620_gb300 as ds
    from paper_1506_08620_gb300 import workloads as W

    if args.workload.startswith("direct"):
        job = setup_direct(args, ds, W, torch, dev, rank)
    elif args.workload == "batched_f32":
        job = setup_batched(args, ds, W, torch, dev, rank)
    elif args.workload in ("learned_f64", "learned_interp_f32"):
        job = setup_learned(args, ds, W, torch, dev, rank)
    elif args.workload == "gapq_f64":
        job = setup_gapq(args, ds, W, torch, dev, rank)
    elif args.workload == "paper_tables":
        job = setup_paper_tables(args, ds, W, torch, dev, rank)
    else:
        raise SystemExit("workload %s: not timed by this bench" % args.workload)
    m = job.m
    stream = torch.cuda.current_stream()

    for _ in range(max(args.warmup, 3)):
        job.search()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        job.search()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    clk = clocks.stop()
    if world > 1:
        total_ms = max_over_ranks(total_ms, dist, dev)
        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = world * m / (ms_per_step * 1e-3)

    # dominant kernel: the search kernel (one launch per step, plus the chunk planner when batched)
    peak, peak_kind = peaks()
    achieved = job.bytes_per_lookup * m / (float(np.mean(per)) * 1e-3) / 1e9
    traffic = traffic_for(job.kernel_key)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind, "bytes_per_lookup": job.bytes_per_lookup,
                "algorithmic_bytes_per_launch": job.bytes_per_lookup * m, "kernel": job.kernel_key}
    if getattr(job, "streamed_bytes_per_lookup", None):
        roofline["streamed_bytes_per_lookup"] = job.streamed_bytes_per_lookup
        roofline["streamed_frac"] = achieved * job.streamed_bytes_per_lookup / job.bytes_per_lookup / peak

    line = {"metric": "lookups/s", "value": value, "unit": "lookups/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": job.dtype_name, "data": "synthetic", "config": workload_config(args),
            "roofline": roofline, "gpu_launches": args.steps * job.launches_per_step, "clocks": clk,
            "build_ms": job.build_ms, "lookups_per_s_with_build": world * m / ((ms_per_step + job.build_ms) * 1e-3),
            "table": job.table}

    # end to end through the public API from pinned host memory, copies inside the timed region
    job.e2e()
    torch.cuda.synchronize()
    e2e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        h2d, d2h = job.e2e()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        e2e_s = max_over_ranks(e2e_s, dist, dev)
    line["e2e"] = {"value": world * m / e2e_s, "unit": "lookups/s", "h2d_bytes_per_step": h2d,
                   "d2h_bytes_per_step": d2h}
    if rank == 0:
        line["e2e"]["matches_device_path"] = bool(torch.equal(job.e2e_out.to(dev), job.out))
        line["check"] = job.verify()

    if rank == 0 and not args.no_extras and job.extras:
        line["variants_lookups_per_s"] = job.extras(stream)
    if rank == 0:
        if args.workload == "learned_interp_f32":
            line["cpu_baseline"] = cpu_baseline_interp(job, args.cpu_seconds)
        elif args.workload == "batched_f32":
            line["cpu_baseline"] = cpu_baseline_batched(W, args.cpu_seconds)
        else:
            cw = W.workload2(m=1 << 24) if job.dtype_name == "f64" else W.workload1()
            if args.workload in ("learned_f64", "gapq_f64"):
                cw = W.workload4(m=1 << 22)
            if args.workload == "paper_tables":
                cw = W.paper_layout(PAPER_SIZES[-1], 1 << 24, np.float64)
            line["cpu_baseline"] = cpu_baseline(cw["X"], cw["Z"], args.cpu_seconds)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0 and args.workload == DEFAULT_WORKLOAD and not args.no_per_config and not args.queries:
        headline = {"lookups_per_s": value, "hbm_frac": roofline["frac"], "check": line["check"]}
        job.keep = job.search = job.e2e = job.verify = None
        del job
        torch.cuda.empty_cache()
        line["per_config"] = per_config(args, ds, W, torch, dev, stream, peak, headline)
    if rank == 0:
        print(json.dumps(line), flush=True)


DEFAULT_WORKLOAD = "learned_interp_f32"
# the other configurations, each measured in the default run: (name, workload, variant)
PER_CONFIG = (("1_direct_f32", "direct_f32", "plain"), ("2_direct_f64", "direct_f64", "plain"),
              ("2_direct_f64_fma", "direct_f64", "fma"), ("3_batched_f32", "batched_f32", "plain"),
              ("4_learned_f64", "learned_f64", "plain"))


def per_config(args, ds, W, torch, dev, stream, peak, headline):
    """Lookups/s, fraction of the HBM peak and mismatches (every result checked
    against the definition) of workloads 1-4, one after the other, each
    autotuned where it has a tuner, timed with CUDA events over 10 launches
    after 2 warm-up launches; and the ratios the spec bars name."""
    setups = {"direct_f32": setup_direct, "direct_f64": setup_direct, "batched_f32": setup_batched,
              "learned_f64": setup_learned}
    res = {}
    for name, wl, var in PER_CONFIG:
        a = argparse.Namespace(**{**vars(args), "workload": wl, "variant": var, "queries": 0})
        job = setups[wl](a, ds, W, torch, dev, 0)
        t = time_calls(torch, stream, job.search, 10)
        rate = job.m / t
        res[name] = {"workload": workload_config(a)["workload"], "lookups_per_s": rate, "ms_per_launch": t * 1e3,
                     "bytes_per_lookup": job.bytes_per_lookup, "hbm_frac": job.bytes_per_lookup * rate / 1e9 / peak,
                     "check": job.verify(), "build_ms": job.build_ms, "table": job.table}
        if wl == "learned_f64":  # the map without the network, same search (what the trained network gains)
            L = job.keep[0]
            lin = ds.ds_learned_build(job.keep[1], cfg=ds.ds_learned_cfg_default(flags=ds.DS_LEARNED_LINEAR))
            ds.ds_learned_autotune(lin, job.keep[2], None, job.out)
            res[name]["linear_map_lookups_per_s"] = job.m / time_calls(
                torch, stream, lambda: ds.ds_learned_search(lin, job.keep[2], out=job.out), 10)
            res[name]["linear_map_max_window"] = lin.info()["max_window"]
            lin.free()
            del L
        job.keep = job.search = job.e2e = job.verify = None
        del job
        torch.cuda.empty_cache()
    res["5_learned_interp_f32"] = headline
    f32 = res["1_direct_f32"]["lookups_per_s"]
    f64 = res["2_direct_f64"]["lookups_per_s"]
    res["vs_plain_direct"] = {"3_batched_f32 / 1_direct_f32": res["3_batched_f32"]["lookups_per_s"] / f32,
                              "3_batched_f32 / 2_direct_f64": res["3_batched_f32"]["lookups_per_s"] / f64,
                              "4_learned_f64 / 2_direct_f64": res["4_learned_f64"]["lookups_per_s"] / f64,
                              "5_learned_interp_f32 / 1_direct_f32": headline["lookups_per_s"] / f32,
                              "5_learned_interp_f32 / 2_direct_f64": headline["lookups_per_s"] / f64}
    return res


def interp_sample(w, frac_log2):
    """The first 2^-frac_log2 of every array's queries (at least one where it has any)."""
    z_off = w["z_off"]
    q = np.diff(z_off)
    take = np.where(q > 0, np.maximum(q >> frac_log2, 1), 0)
    pos = np.concatenate([np.arange(z_off[a], z_off[a] + take[a]) for a in range(q.size)])
    return pos, W_csr(take)


def W_csr(sizes):
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


def cpu_baseline_interp(job, seconds):
    """The oracle (single thread: the interval by its definition, the interpolant
    in float64) on a bounded sample of the headline workload's queries, sized
    for about `seconds`; its answers are compared with this step's GPU results."""
    import oracle
    oracle.lib()
    w = job.host
    pos, zo = interp_sample(w, 12)  # calibrate on 2^-12 of the queries, then size the sample
    t0 = time.perf_counter()
    oracle.interp_batch(w["Xcat"], w["Ycat"], w["x_off"], w["Zcat"][pos], zo)
    dt = time.perf_counter() - t0
    k = int(min(12, max(0, 12 - np.floor(np.log2(max(seconds / max(dt, 1e-6), 1.0))))))
    pos, zo = interp_sample(w, k)
    t0 = time.perf_counter()
    oracle.interp_batch(w["Xcat"], w["Ycat"], w["x_off"], w["Zcat"][pos], zo)
    dt = time.perf_counter() - t0
    n = pos.size
    rate = n / dt
    out = job.out.cpu().numpy()[pos]
    I, y64 = oracle.interp_batch(w["Xcat"], w["Ycat"], w["x_off"], w["Zcat"][pos], zo)
    yv = job.yout.cpu().numpy()[pos] if getattr(job, "yout", None) is not None else None
    res = {"value": rate, "unit": "lookups/s", "cores": 1, "kind": "oracle",
           "sample": "the first 2^-%d of every array's queries (%d of %d), one pass, %.1f s"
                     % (k, n, w["Zcat"].size, dt),
           "mismatches_vs_gpu": int((I != out).sum())}
    if yv is not None:
        arr = np.searchsorted(w["z_off"], pos, side="right") - 1
        gi = w["x_off"][arr] + np.clip(I, 0, None)
        Y = w["Ycat"]
        scale = np.maximum(np.abs(y64), np.maximum(np.abs(Y[gi]), np.abs(Y[np.minimum(gi + 1, Y.size - 1)])))
        res["y_outside_tolerance_vs_gpu"] = int((~(np.abs(yv.astype(np.float64) - y64) <= 1e-6 * scale)).sum())
    return res


def cpu_baseline_batched(W, seconds):
    import oracle
    w = W.workload3(total_queries=1 << 22)
    n_arr = len(w["x_off"]) - 1
    t0 = time.perf_counter()
    oracle.upper_bound_batch(w["Xcat"], w["x_off"], w["Zcat"], w["z_off"])
    dt = time.perf_counter() - t0
    return {"value": w["Zcat"].size / dt, "unit": "lookups/s", "cores": 1, "kind": "oracle",
            "sample": "%d arrays of the batched workload with 2^22 queries in proportion, one pass, %.1f s"
                      % (n_arr, dt)}


if __name__ == "__main__":
    main()
