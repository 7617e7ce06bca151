#!/usr/bin/env python3
"""Throughput of direct-search interval lookup on GB300.

Workload (default): float64, 2^20 + 1 knots with lognormal(0, 0.5) gaps,
2^27 queries uniform over [X_0, X_N) (unsorted), int32 results.  One step is
one search pass over all queries (Algorithm direct), as in the paper's
throughput harness (Algorithm harness: the table is built before the clock
starts); the build of the table is timed separately in the same run.

Prints ONE JSON line (rank 0).  Multi-GPU (torchrun): every rank builds its
own replica of the table and searches its own 2^27 queries (weak scaling, no
collective on the data path).

--impl reference times the CPU oracle (std::upper_bound definition) on a
bounded sample of the same workload on the host cores.
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

WORKLOADS = ("direct_f64", "direct_f64_sorted", "direct_f32", "batched_f32", "learned_f64", "learned_interp_f32")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="direct_f64", choices=WORKLOADS)
    p.add_argument("--variant", default="plain", choices=["plain", "fma", "cache", "fma_cache"])
    p.add_argument("--no-extras", action="store_true", help="skip the secondary measurements")
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="target CPU time of the oracle baseline")
    p.add_argument("--queries", type=int, default=0, help="override the query count (profiling runs)")
    return p.parse_args()


# ----------------------------------------------------------------------------- helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1506_08620_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel_key):
    """Per-launch DRAM bytes from a committed ncu capture, if it was taken on the
    current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    e = d.get(kernel_key)
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("bytes_per_launch")


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


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle
    from paper_1506_08620_gb300 import workloads as W
    X, Z, desc = reference_sample(args)
    oracle.lib()
    for _ in range(max(args.warmup, 0)):
        oracle.upper_bound(X, Z)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.upper_bound(X, Z)
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    value = Z.size / t
    line = {"impl": "reference", "metric": "lookups/s", "value": value, "unit": "lookups/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if X.dtype == np.float64 else "f32",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": "lookups/s", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "lookups/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reference_sample(args, n=1 << 20):
    from paper_1506_08620_gb300 import workloads as W
    if args.workload.startswith("direct_f64"):
        w = W.workload2(m=n, sort=args.workload.endswith("sorted"))
    elif args.workload == "direct_f32":
        w = W.workload1()
    else:
        w = W.workload2(m=n)
    return w["X"], w["Z"], "%d queries of workload %s (same knots), one pass per step" % (w["Z"].size, w["name"])


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
    return {"value": n / dt, "unit": "lookups/s", "cores": 1, "kind": "oracle",
            "sample": "first %d of the %d queries, one pass, %.1f s" % (n, Z.size, dt)}


def workload_config(args):
    base = {
        "direct_f64": {"workload": "direct search f64: 2^20+1 knots, lognormal(0,0.5) gaps, 2^27 uniform queries",
                       "knots": (1 << 20) + 1, "queries": 1 << 27},
        "direct_f64_sorted": {"workload": "direct search f64: 2^20+1 knots, lognormal(0,0.5) gaps, "
                                          "2^27 sorted uniform queries", "knots": (1 << 20) + 1, "queries": 1 << 27},
        "direct_f32": {"workload": "direct search f32: 1025 knots, 1,002,048 queries tiled 512x into one stream",
                       "knots": 1025, "queries": 1002048 * 512},
    }.get(args.workload, {"workload": args.workload})
    base = dict(base)
    base["variant"] = args.variant
    if args.queries:
        base["queries"] = args.queries
    base["l2"] = "inputs larger than L2 (queries and results stream from HBM every step)"
    base["step"] = "one search pass over all queries; table built before the clock (Algorithm harness)"
    return base


# ----------------------------------------------------------------------------- our arm
def main():
    args = parse()
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

    flags = {"plain": 0, "fma": ds.DS_FMA, "cache": ds.DS_CACHE_LAYOUT,
             "fma_cache": ds.DS_FMA | ds.DS_CACHE_LAYOUT}[args.variant]
    if args.workload in ("direct_f64", "direct_f64_sorted"):
        w = W.workload2(seed=W.SEED_BASE + 2 + 1000 * rank if rank else None, m=args.queries or (1 << 27),
                        sort=args.workload.endswith("sorted"))
        X, Z = w["X"], w["Z"]
        Zh = Z
        bytes_per_lookup = 8 + 4
        dtype_name = "f64"
    elif args.workload == "direct_f32":
        w = W.workload1()
        X = w["X"]
        Zh = np.tile(w["Z"], 512)
        if args.queries:
            Zh = Zh[: args.queries]
        bytes_per_lookup = 4 + 4
        dtype_name = "f32"
    else:
        raise SystemExit("workload %s: not timed by this bench" % args.workload)
    m = Zh.size
    Xd = torch.from_numpy(X).to(dev)
    Zd = torch.from_numpy(Zh).to(dev)
    out = torch.empty(m, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    # build (timed separately; the paper reports setup cost apart from throughput)
    builds = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        idx = ds.ds_build(Xd, flags)
        torch.cuda.synchronize()
        builds.append((time.perf_counter() - t0) * 1e3)
        info = idx.info()
        if _ < 2:
            idx.free()
    build_ms = float(np.median(builds))

    for _ in range(max(args.warmup, 3)):
        ds.ds_search(idx, Zd, out)
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
        ds.ds_search(idx, Zd, out)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = world * m / (ms_per_step * 1e-3)

    # dominant kernel: the search kernel, one launch per step
    peak, peak_kind = peaks()
    achieved = bytes_per_lookup * m / (float(np.mean(per)) * 1e-3) / 1e9
    kernel_key = "search_%s_%s" % (dtype_name, args.variant)
    traffic = traffic_for(kernel_key)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": bytes_per_lookup * m, "kernel": kernel_key}

    line = {"metric": "lookups/s", "value": value, "unit": "lookups/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_name, "data": "synthetic", "config": workload_config(args),
            "roofline": roofline, "gpu_launches": args.steps, "clocks": clk, "build_ms": build_ms,
            "lookups_per_s_with_build": world * m / ((ms_per_step + build_ms) * 1e-3),
            "table": {"H": info["H"], "R": info["R"], "table_bytes": info["table_bytes"],
                      "smem_resident": info["smem_resident"], "h_updates": info["h_updates"]}}

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    if rank == 0 or world > 1:
        Zp = torch.from_numpy(Zh).pin_memory()
        Ip = torch.empty(m, dtype=torch.int32).pin_memory()
        ds.ds_search_host(idx, Zp, Ip)
        torch.cuda.synchronize()
        e2e_steps = max(3, min(args.steps, 10))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ds.ds_search_host(idx, Zp, Ip)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        if world > 1:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        line["e2e"] = {"value": world * m / e2e_s, "unit": "lookups/s", "h2d_bytes_per_step": Zp.numel() * Zp.element_size(),
                       "d2h_bytes_per_step": Ip.numel() * 4}
        if rank == 0:
            ok = bool(torch.equal(Ip.to(dev), out))
            line["e2e"]["matches_device_path"] = ok
        del Zp, Ip

    if rank == 0 and not args.no_extras:
        extras = {}
        for name, fl in (("fma", ds.DS_FMA), ("cache", ds.DS_CACHE_LAYOUT), ("fma_cache", ds.DS_FMA | ds.DS_CACHE_LAYOUT),
                         ("plain", 0)):
            if name == args.variant:
                continue
            j = ds.ds_build(Xd, fl)
            for _ in range(3):
                ds.ds_search(j, Zd, out)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                ds.ds_search(j, Zd, out)
            e1.record(stream)
            torch.cuda.synchronize()
            extras[name] = m / (e0.elapsed_time(e1) / 5 * 1e-3)
            j.free()
        if args.workload == "direct_f64":
            Zs = torch.sort(Zd).values
            for _ in range(3):
                ds.ds_search(idx, Zs, out)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                ds.ds_search(idx, Zs, out)
            e1.record(stream)
            torch.cuda.synchronize()
            extras["sorted_queries_" + args.variant] = m / (e0.elapsed_time(e1) / 5 * 1e-3)
            del Zs
        line["variants_lookups_per_s"] = extras
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(X, Zh[: 1 << 26], args.cpu_seconds)
        print(json.dumps(line), flush=True)
    idx.free()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
