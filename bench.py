#!/usr/bin/env python
"""Benchmark of the level-by-level k-d tree build (subset-median splits) on GB300.

One step = one complete kdt_build of the workload's tree through the C ABI,
on inputs already resident in HBM (they are larger than L2). Prints one JSON
line on rank 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3|c2|c1]
    python bench.py --impl reference ...   # the CPU oracle on a bounded sample

N > 1 runs under torchrun: every rank builds its own tree of the same shape
(a different seed) with no exchange between ranks ("replicas"); the value is
the points x levels of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "build points×levels/s"
UNIT = "points*levels/s"


def workload(name: str, rank: int):
    from paper_2201_08288_gb300 import workloads as W
    if name == "c3":
        spec = W.config3()
    elif name == "c2":
        spec = W.config2()
    elif name == "c1":
        spec = W.config1()
    elif name == "c3s":  # profiling case: config 3's recipe at n=2^22 (larger than L2, small for ncu)
        spec = W.config3(n=1 << 22, depth=15)
    elif name == "w6":  # Sec. 5's simulation shape: trivariate normal, correlation 0.5, n=2^27, depth 10
        spec = W.paper_mvn(1 << 27, 0.5, 10)
    elif name == "w6f":  # the same shape through the normal CDF, split by the paper's estimator (J = 16)
        spec = W.paper_mvn_fourier(1 << 27, 0.5, 10, 16)
    elif name == "w6fs":  # its profiling case: n=2^22, depth 8 (larger than L2, small for ncu)
        spec = W.paper_mvn_fourier(1 << 22, 0.5, 8, 16)
    else:
        raise SystemExit(f"unknown workload {name}")
    spec.seed += 1000 * rank
    if spec.sid_seed is not None:
        spec.sid_seed += 1000 * rank
    kw = dict(r=spec.r, subset_mode=spec.subset_mode, depth=spec.depth, key_rule=spec.key_rule,
              leaf_size=spec.leaf_size, max_levels=spec.max_levels, fourier_j=spec.fourier_j)
    return spec, kw


def bytes_per_point(kernel: str, d: int, sid_bytes: int, subset_mode: int) -> float:
    """Algorithmic bytes one launch moves per point it processes."""
    return {
        "k_part_scatter": 2.0 * (4 * d + 4 + sid_bytes),   # read + write every column, perm, ids
        "k_subtree": 4.0 * d + 4 + sid_bytes + 4,           # stage everything once, write perm once
        "k_ps_move": 2.0 * (4 * d + sid_bytes) + 4,         # columns and ids in and out, perm out
        "k_part_count": 4.0,
        "k_select_small": 4.0,                              # the key column, read in place
        "k_fourier_moments": 4.0,                           # the key column, read in place
        "k_minmax": 4.0 * d,
    }.get(kernel, 0.0)


def model_bytes_per_point_level(d: int, sid_bytes: int, subset_mode: int) -> float:
    """Bytes each level must move per point (SoA ping-pong model): the key
    column read for the selection, the subset-id source (explicit ids, or the
    permutation the id is derived from), read+write of all columns and the
    permutation, read+write of an explicit id column."""
    s_sel = sid_bytes if subset_mode == 2 else 4
    return 4 + s_sel + 8 * (d + 1) + 2 * (sid_bytes if subset_mode == 2 else 0)


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's);
    x itself when there is no process group."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples (KDT_CLOCKS_DIR, default: the system's temporary directory);
        # the JSON line carries their summary
        out_dir = os.environ.get("KDT_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        """Start sampling and wait (at most 10 s) for the first sample: the
        sampler's own start-up (NVML initialisation, which on a fresh box takes
        long enough to delay the build's host thread) stays out of the timed
        region, which the caller opens later with mark()."""
        self.offset = 0
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 10.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)

    def mark(self):
        """The timed region starts: stop() summarises the samples from here on."""
        try:
            self.offset = os.path.getsize(self.path)
        except OSError:
            self.offset = 0

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            text = fh.read()
        lines = text[self.offset:].splitlines()
        if not any(len(x.split(",")) >= 9 for x in lines):  # a region shorter than one sample period
            lines = text.splitlines()
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() in ("active", "0x1") or v == "1":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_gbs() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def copy_rates(host, dev) -> tuple:
    """Pinned host <-> device copy rates (GB/s) of 1 GiB taken from `host`,
    each the best of three."""
    import torch
    n = min(host.numel(), (1 << 30) // 4)
    h = host.reshape(-1)[:n]
    d = torch.empty(n, dtype=h.dtype, device=dev)
    best = [float("inf"), float("inf")]
    for _ in range(3):
        for k, (dst, src) in enumerate(((d, h), (h, d))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            best[k] = min(best[k], time.perf_counter() - t0)
    del d
    return n * 4 / best[0] / 1e9, n * 4 / best[1] / 1e9


def recorded_traffic(kernel: str, workload_name: str):
    """DRAM bytes per point of `kernel` from the committed ncu summary, if the
    kernel sources are unchanged since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(p))[f"{kernel}:{workload_name}"]
    except Exception:
        return None
    h = hashlib.sha256()
    for f in sorted(rec.get("sources", [])):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if h.hexdigest() != rec.get("sha256"):
        return None
    return float(rec["dram_bytes_per_point"])


def oracle_build(oracle, spec, pts, sid, s, depth_s):
    """The oracle's build of a sample: the subset-median rule, or the paper's
    estimator for a workload that splits by it."""
    if spec.fourier_j > 0:
        return oracle.fourier_build_tree(pts, depth=depth_s, J=spec.fourier_j)
    return oracle.build_tree(pts, r=s.r, subset_mode=s.subset_mode, sid=sid, depth=depth_s, key_rule=s.key_rule)


def cpu_baseline(name: str, target_s: float = 12.0) -> dict:
    """The oracle as it stands, single-threaded on a host core, on a bounded
    sample of the same workload recipe (fewer points, depth reduced so the
    leaves keep the same size)."""
    import oracle
    from paper_2201_08288_gb300 import workloads as W
    spec, kw = workload(name, 0)
    full_n, full_depth = spec.n, spec.depth
    n_s = 1 << 16
    while True:
        depth_s = max(1, full_depth - int(round(np.log2(full_n / n_s))))
        s = W.TreeSpec(spec.name, n_s, spec.d, spec.dist, spec.seed, spec.r, spec.subset_mode, spec.key_rule,
                       depth=depth_s, sid_seed=spec.sid_seed, rho=spec.rho)
        pts, sid = s.points(), s.sids()
        t0 = time.perf_counter()
        t = oracle_build(oracle, spec, pts, sid, s, depth_s)
        dt = time.perf_counter() - t0
        if dt * 4 > target_s or n_s >= full_n:
            return {"value": n_s * t.levels / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                    "host_cores": os.cpu_count(),
                    "sample": f"n={n_s} depth={depth_s} of the {spec.name} recipe, one build, {dt:.2f} s"}
        n_s *= 2


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    spec, _ = workload(args.workload, 0)
    import oracle
    from paper_2201_08288_gb300 import workloads as W
    n_s = 1 << 18
    depth_s = max(1, spec.depth - int(round(np.log2(spec.n / n_s))))
    s = W.TreeSpec(spec.name, n_s, spec.d, spec.dist, spec.seed, spec.r, spec.subset_mode, spec.key_rule,
                   depth=depth_s, sid_seed=spec.sid_seed, rho=spec.rho)
    pts, sid = s.points(), s.sids()
    for _ in range(args.warmup):
        oracle_build(oracle, spec, pts, sid, s, depth_s)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        t = oracle_build(oracle, spec, pts, sid, s, depth_s)
    dt = time.perf_counter() - t0
    value = args.steps * n_s * t.levels / dt
    sample = f"n={n_s} depth={depth_s} of the {spec.name} recipe per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": {"workload": spec.name, "reference_sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))] if xs else None


def run_batched(args, dev, kdt) -> dict:
    """Independent trees of the batched recipe (n log-uniform in [2^8, 2^20],
    d in {2,3,8,16}, uniform or 8-cluster mixture, r in {4,16,64} by index mod
    r, cyclic, leaf <= 32) built together by kdt_build_batched; the same trees
    built one by one with kdt_build for comparison."""
    import torch
    from paper_2201_08288_gb300 import workloads as W
    specs = W.config4_batch(num_trees=args.trees)
    items = []
    for s in specs:
        items.append(dict(points=s.points_device(dev), r=s.r, subset_mode=0, depth=0, leaf_size=32,
                          max_levels=s.max_levels, key_rule=0))
    descs, outs = kdt.make_descs(items)
    ws = torch.empty(kdt.kdt_workspace_size_batched(descs), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    clocks = Clocks(dev.index or 0)
    clocks.start()
    for _ in range(args.warmup):
        trees, st = kdt.kdt_build_batched(items, workspace=ws, outputs=outs, descs=descs, stream=stream)
    torch.cuda.synchronize()
    assert all(x == 0 for x in st), st
    units = sum(int(s.n) * t.levels for s, t in zip(specs, trees))
    clocks.mark()
    launches0 = kdt.kdt_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        kdt.kdt_build_batched(items, workspace=ws, outputs=outs, descs=descs, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = kdt.kdt_launch_count() - launches0
    clk = clocks.stop()
    del ws
    torch.cuda.empty_cache()
    # the same trees, one kdt_build each (workspace sized for the largest)
    big = max(range(len(items)), key=lambda i: specs[i].n * (specs[i].d + 1))
    sizes = [kdt.kdt_workspace_size(kdt.make_params(int(s.n), s.d, r=s.r, subset_mode=0, depth=0, leaf_size=32,
                                                    max_levels=s.max_levels)) for s in specs]
    ws1 = torch.empty(max(sizes), dtype=torch.uint8, device=dev)
    for i in range(min(64, len(items))):
        it = items[i]
        kdt.kdt_build(it["points"], workspace=ws1, outputs=outs[i], stream=stream,
                      **{k: v for k, v in it.items() if k != "points"})
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, it in enumerate(items):
        kdt.kdt_build(it["points"], workspace=ws1, outputs=outs[i], stream=stream,
                      **{k: v for k, v in it.items() if k != "points"})
    torch.cuda.synchronize()
    solo_s = time.perf_counter() - t0
    value = args.steps * units / (ms / 1e3)
    solo = units / solo_s
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"batched_{len(items)}_trees_n2^8..2^20_d2-16_mod_r4-64_leaf32",
                       "points": int(sum(s.n for s in specs)), "points_x_levels": units,
                       "parallelism": "replicas1"},
            "solo_loop": {"value": solo, "unit": UNIT, "ms": 1e3 * solo_s,
                          "what": "the same trees, one kdt_build call each, in sequence"},
            "batched_vs_solo": value / solo, "gpu_launches": launches, "clocks": clk}


def run_serving(args, dev, kdt) -> dict:
    """A Poisson stream of build requests (n log-uniform in [2^10, 2^24],
    d in {3,16}, uniform or 8-cluster mixture, r=32 by index mod r, leaf <= 64)
    submitted to a kdt.Server with a 64 GB budget; each request's points are
    drawn on the device when it arrives. The arrival rate is `load` times the
    server's saturated capacity (the first 200 requests submitted at once).
    Reports p50/p99 latency (submit to completion) and throughput against the
    same requests built one by one."""
    import torch
    from paper_2201_08288_gb300 import workloads as W
    stream = torch.cuda.current_stream(dev)
    _, specs = W.config5_stream(num_requests=args.requests, rate=1.0)
    kw_of = lambda s: dict(r=32, subset_mode=0, depth=0, leaf_size=64, max_levels=s.max_levels, key_rule=0)
    sample = specs[:min(200, len(specs))]
    # solo: the sample built one by one
    ws1 = torch.empty(max(kdt.kdt_workspace_size(kdt.make_params(int(s.n), s.d, **kw_of(s))) for s in sample),
                      dtype=torch.uint8, device=dev)
    pts_s = [s.points_device(dev) for s in sample]
    for p_, s in zip(pts_s[:8], sample[:8]):
        kdt.kdt_build(p_, workspace=ws1, stream=stream, **kw_of(s))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    solo_units = 0
    solo_lat = []
    for p_, s in zip(pts_s, sample):
        t1 = time.perf_counter()
        t = kdt.kdt_build(p_, workspace=ws1, stream=stream, **kw_of(s))  # returns when built
        solo_lat.append(1e3 * (time.perf_counter() - t1))
        solo_units += int(s.n) * t.levels
    torch.cuda.synchronize()
    solo_s = time.perf_counter() - t0
    del ws1
    torch.cuda.empty_cache()
    with kdt.Server(64 << 30, 256) as sv:
        # saturated capacity: the sample submitted at once
        t0 = time.perf_counter()
        tks = [sv.submit(dict(points=p_, **kw_of(s))) for p_, s in zip(pts_s, sample)]
        for tk in tks:
            assert sv.poll(tk)[0] == 0
        capacity = len(sample) / (time.perf_counter() - t0)
        del pts_s, tks
        torch.cuda.empty_cache()
        rate = args.load * capacity
        arrivals, specs = W.config5_stream(num_requests=args.requests, rate=rate)
        lat, units, backlog_max = [], 0, 0
        live = {}
        t_start = time.perf_counter()

        def reap(wait):
            nonlocal units
            for tk in list(live):
                r = sv.poll(tk, -1 if wait else 0)
                if r is not None:
                    assert r[0] == 0, r[0]
                    lat.append(r[2])
                    units += int(live.pop(tk).n) * r[1].levels

        for i, s in enumerate(specs):
            reap(False)  # once per arrival: polling takes the server's lock
            ahead = arrivals[i] - (time.perf_counter() - t_start)
            if ahead > 0:
                time.sleep(ahead)
            if len(live) > 512:
                raise SystemExit("serving: more than 512 requests outstanding; the arrival rate exceeds capacity")
            live[sv.submit(dict(points=s.points_device(dev), **kw_of(s)))] = s
            backlog_max = max(backlog_max, len(live))
        reap(True)
        wall = time.perf_counter() - t_start
        info = sv.stats()
    return {"metric": METRIC, "value": units / wall, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": 1e3 * wall, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"serving_{len(specs)}_requests_poisson_n2^10..2^24_d3or16_mod_r32_leaf64",
                       "rate_per_s": rate, "load": args.load, "capacity_per_s": capacity, "mem_budget_gb": 64},
            "latency_ms": {"p50": _pct(lat, 0.5), "p99": _pct(lat, 0.99), "max": max(lat)},
            "peak_in_flight": info["peak_in_flight"], "outstanding_max": backlog_max,
            "solo": {"value": solo_units / solo_s, "unit": UNIT, "requests_per_s": len(sample) / solo_s,
                     "latency_ms": {"p50": _pct(solo_lat, 0.5), "p99": _pct(solo_lat, 0.99), "max": max(solo_lat)},
                     "what": f"the first {len(sample)} requests, one kdt_build each, back to back "
                             "(latency: each build alone, call to return)"},
            "served_vs_solo": (units / wall) / (solo_units / solo_s)}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c3", "c2", "c1", "c3s", "w6", "w6f", "w6fs", "c4", "c5"])
    ap.add_argument("--trees", type=int, default=4096, help="c4: number of trees")
    ap.add_argument("--requests", type=int, default=20000, help="c5: number of requests")
    ap.add_argument("--load", type=float, default=0.7, help="c5: arrival rate / solo capacity")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shards", type=int, default=0,
                    help="> 0: time the sharded build (kdt_build_sharded, this many logical shards; depth mode)")
    ap.add_argument("--no-extra", action="store_true",
                    help="c3: skip the batched (config 4) and served (config 5) sub-records")
    ap.add_argument("--extra-requests", type=int, default=3000,
                    help="c3: requests of the served sub-record (config 5's stream, first N arrivals)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    from paper_2201_08288_gb300 import build as cuda_build, kdt
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        cuda_build.build()
    if dist:
        dist.barrier()
    kdt.load_library()
    if args.workload in ("c4", "c5"):
        res = run_batched(args, dev, kdt) if args.workload == "c4" else run_serving(args, dev, kdt)
        if rank == 0:
            print(json.dumps(res))
        return

    spec, kw = workload(args.workload, rank)
    pts = spec.points_device(dev)
    sid = spec.sids_device(dev)
    sid_bytes = 0 if sid is None else sid.element_size()
    p = kdt.make_params(spec.n, spec.d, sid_ptr=sid.data_ptr() if sid is not None else 0,
                        sid_bytes=max(sid_bytes, 1), **kw)
    ws = torch.empty(kdt.kdt_workspace_size(p), dtype=torch.uint8, device=dev)
    out = None
    stream = torch.cuda.current_stream(dev)

    # preallocated outputs (sized for the capacity)
    cap = spec.depth if spec.depth > 0 else spec.max_levels
    out = kdt.Tree(torch.empty(spec.n, dtype=torch.int32, device=dev),
                   torch.empty((1 << cap) - 1, dtype=torch.float32, device=dev),
                   torch.empty((1 << cap) - 1, dtype=torch.int8, device=dev),
                   torch.empty((1 << cap) + 1, dtype=torch.int64, device=dev), 0)

    def build_once():
        if args.shards:
            return kdt.kdt_build_sharded(pts, args.shards, sid=sid, outputs=out, stream=stream,
                                         **{k: kw[k] for k in ("r", "subset_mode", "depth", "key_rule")})
        return kdt.kdt_build(pts, sid=sid, workspace=ws, outputs=out, stream=stream, **kw)

    clocks = Clocks(dev.index if dev.index is not None else 0)
    clocks.start()
    for _ in range(args.warmup):
        tree = build_once()
    torch.cuda.synchronize()
    levels = tree.levels

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.mark()
    launches0 = kdt.kdt_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        build_once()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = kdt.kdt_launch_count() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist, dev)
    units = world * args.steps * spec.n * levels
    value = units / (ms / 1e3)

    # per-kernel device time of the same steps, from CUDA events recorded by the library
    kdt.kdt_trace_read(reset=True)
    kdt.kdt_trace_enable(True)
    for _ in range(args.steps):
        build_once()
    torch.cuda.synchronize()
    stats = kdt.kdt_trace_read(reset=True)
    kdt.kdt_trace_enable(False)
    dominant = max(stats.items(), key=lambda kv: kv[1][1])[0]
    nl, tot_ms, pts_done = stats[dominant]
    bpp = bytes_per_point(dominant, spec.d, sid_bytes, spec.subset_mode)
    peak, peak_src = measured_peak_gbs()
    achieved = (pts_done * bpp) / (tot_ms / 1e3) / 1e9 if tot_ms > 0 else 0.0
    traffic_pp = recorded_traffic(dominant, args.workload)
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "algorithmic_bytes_per_launch": pts_done * bpp / max(nl, 1),
                "launches": nl, "avg_launch_ms": tot_ms / max(nl, 1),
                "traffic": (traffic_pp * pts_done / max(nl, 1)) if traffic_pp is not None else None,
                "share_of_step": tot_ms / (ms / args.steps * args.steps) if ms > 0 else None}
    kernel_table = {k: {"launches": v[0], "ms": round(v[1], 3), "points": v[2]} for k, v in stats.items()}
    mb = model_bytes_per_point_level(spec.d, sid_bytes, spec.subset_mode)
    build_model_gbs = spec.n * levels * mb / (ms / args.steps / 1e3) / 1e9

    e2e = None
    if not args.no_e2e:
        host_pts = torch.empty(pts.shape, dtype=torch.float32, pin_memory=True)
        host_pts.copy_(pts)
        host_sid = None
        if sid is not None:
            host_sid = torch.empty(sid.shape, dtype=sid.dtype, pin_memory=True)
            host_sid.copy_(sid)
        hp = kdt.make_params(spec.n, spec.d, sid_ptr=1 if sid is not None else 0, sid_bytes=max(sid_bytes, 1),
                             **kw)
        ws_h = torch.empty(kdt.kdt_workspace_size_host(hp), dtype=torch.uint8, device=dev)
        del ws
        torch.cuda.empty_cache()
        o_perm = torch.empty(spec.n, dtype=torch.int32, pin_memory=True)
        o_vals = torch.empty((1 << cap) - 1, dtype=torch.float32, pin_memory=True)
        o_dims = torch.empty((1 << cap) - 1, dtype=torch.int8, pin_memory=True)
        o_offs = torch.empty((1 << cap) + 1, dtype=torch.int64, pin_memory=True)
        houts = kdt.Tree(o_perm.numpy(), o_vals.numpy(), o_dims.numpy(), o_offs.numpy(), 0)
        hsid = host_sid.numpy() if host_sid is not None else None
        if hsid is not None and hsid.dtype == np.int16:
            hsid = hsid.view(np.uint16)

        def e2e_once():
            return kdt.kdt_build_host(host_pts.numpy(), sid=hsid, workspace=ws_h, stream=stream,
                                      outputs=houts, **kw)
        for _ in range(args.warmup):
            e2e_once()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        calls = []  # each call ends with its stream synchronised: per-call host times
        for _ in range(args.steps):
            tq = time.perf_counter()
            ht = e2e_once()
            calls.append(time.perf_counter() - tq)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e_s = time.perf_counter() - t0
        e_s = max_over_ranks(e_s, dist, dev)
        nleaf = 1 << ht.levels
        e2e = {"value": world * args.steps * spec.n * ht.levels / e_s, "unit": UNIT,
               "h2d_bytes_per_step": spec.d * spec.n * 4 + spec.n * sid_bytes,
               "d2h_bytes_per_step": spec.n * 4 + (nleaf - 1) * 5 + (nleaf + 1) * 8,
               "ms_per_step": 1e3 * e_s / args.steps,
               # the spread of single calls (this rank): a slow copy shows as one outlier
               "call_ms": {"min": 1e3 * min(calls), "median": 1e3 * statistics.median(calls),
                           "max": 1e3 * max(calls)}}
        # this box's pinned copy rates (the copies alone bound the end-to-end time from below)
        h2d, d2h = copy_rates(host_pts, dev)
        e2e.update({"h2d_gbs": h2d, "d2h_gbs": d2h,
                    "copies_ms": 1e3 * (e2e["h2d_bytes_per_step"] / (h2d * 1e9) +
                                        e2e["d2h_bytes_per_step"] / (d2h * 1e9))})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)

    extra = {}
    if args.workload == "c3" and world == 1 and not args.no_extra and not args.shards:
        # the batching and serving patterns on their own configurations, beside
        # the plain build: all 4096 trees of config 4 against the same trees
        # built one by one, and config 5's stream (its first N arrivals)
        # against the same requests built one by one
        del pts, sid, out
        if "ws" in locals():
            del ws
        if e2e is not None:
            del ws_h, host_pts, host_sid, houts
        torch.cuda.empty_cache()
        sub = argparse.Namespace(**vars(args))
        sub.steps, sub.warmup = 3, 3
        b = run_batched(sub, dev, kdt)
        extra["batched"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "steps", "config", "solo_loop",
                                              "batched_vs_solo", "gpu_launches", "clocks")}
        torch.cuda.empty_cache()
        sub.requests = args.extra_requests
        sv = run_serving(sub, dev, kdt)
        extra["served"] = {k: sv[k] for k in ("value", "unit", "ms_per_step", "config", "latency_ms", "solo",
                                              "served_vs_solo", "peak_in_flight", "outstanding_max")}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": spec.name, "n": spec.n, "d": spec.d, "r": spec.r,
                       "subset_mode": ["mod", "contiguous", "explicit"][spec.subset_mode],
                       "key_rule": ["cyclic", "widest_spread"][spec.key_rule], "depth": spec.depth,
                       "levels": levels, "parallelism": f"replicas{world}",
                       **({"shards": args.shards} if args.shards else {}),
                       "l2": f"inputs larger than L2 ({spec.d * spec.n * 4 / 1e9:.1f} GB per step)"},
            "roofline": roofline,
            "build_model_gbs": build_model_gbs, "build_model_frac": build_model_gbs / peak,
            "model_bytes_per_point_level": mb,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "kernels": kernel_table, **extra,
        }))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
