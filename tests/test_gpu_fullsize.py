"""GPU parity at the benchmark's full sizes, built the way bench.py times the
build (the same workload recipe and parameters, a preallocated workspace and
preallocated outputs, the caller's stream, the default tuning).

Compared bit for bit with the oracle's whole tree (perm, split values as bit
patterns, split dims, node offsets, L):
  - config 3: n = 2^27, d = 8, r = 256 explicit, widest spread, depth 20;
  - config 2: n = 2^24, d = 3, r = 64 contiguous, cyclic, depth 16;
  - Sec. 5's simulation shape at rho = 0.5: trivariate normal with common
    correlation rho, n = 2^27, r = 64 by index, cyclic, depth 10;
  - config 4: all 4096 trees of the batched recipe through kdt_build_batched;
  - config 5: a seeded sample of 200 requests of the serving stream (the 10
    largest of its 20000 requests among them) through the server, submitted
    in arrival order so that they overlap on the device.
The oracle is single-threaded per tree; independent trees run on the host's
cores at the same time (a thread pool: the oracle's C calls release the
interpreter lock), and the single-tree oracle builds start as soon as their
inputs are on the host, so that they run while the GPU-side checks do.

Every node of the single trees is also checked on the device against the
properties that fix a tree given its splits (devcheck.py); Sec. 5's other
correlations are checked that way, plus the oracle's split of sampled nodes."""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np
import pytest

import bench
import oracle
from devcheck import check_sampled_nodes, check_tree_device
from gpu_util import assert_same_tree, require_gpu
from paper_2201_08288_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

_POOL = None


def oracle_pool() -> cf.ThreadPoolExecutor:
    global _POOL
    if _POOL is None:
        _POOL = cf.ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2))
    return _POOL


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def oracle_kw(kw: dict) -> dict:
    return {k: kw[k] for k in ("r", "subset_mode", "depth", "leaf_size", "max_levels", "key_rule")}


def host_sids(sid):
    if sid is None:
        return None
    return sid.cpu().numpy().view(np.uint16 if sid.element_size() == 2 else np.uint8)


def exact_cases():
    spec3, kw3 = bench.workload("c3", 0)
    spec2, kw2 = bench.workload("c2", 0)
    spec6 = workloads.paper_mvn(1 << 27, 0.5, 10)
    kw6 = dict(r=spec6.r, subset_mode=spec6.subset_mode, depth=spec6.depth, key_rule=spec6.key_rule,
               leaf_size=spec6.leaf_size, max_levels=spec6.max_levels)
    return {"c3": (spec3, kw3), "c2": (spec2, kw2), "w6_rho0.5": (spec6, kw6)}


@pytest.fixture(scope="module")
def exact_jobs():
    """Per bit-exact single-tree case: its inputs on the device (drawn as
    bench.py draws them), and the oracle's build of the same inputs running
    in the pool."""
    dev = torch.device("cuda:0")
    jobs = {}
    for name, (spec, kw) in exact_cases().items():
        pts = spec.points_device(dev)
        sid = spec.sids_device(dev)
        pts_h, sid_h = pts.cpu().numpy(), host_sids(sid)
        fut = oracle_pool().submit(oracle.build_tree, pts_h, sid=sid_h, **oracle_kw(kw))
        jobs[name] = (spec, kw, pts, sid, fut)
    yield jobs
    jobs.clear()
    torch.cuda.empty_cache()


def bench_build(spec, kw, pts=None, sid=None):
    from paper_2201_08288_gb300 import kdt
    dev = torch.device("cuda:0")
    if pts is None:
        pts = spec.points_device(dev)
        sid = spec.sids_device(dev)
    sid_bytes = 0 if sid is None else sid.element_size()
    p = kdt.make_params(spec.n, spec.d, sid_ptr=sid.data_ptr() if sid is not None else 0,
                        sid_bytes=max(sid_bytes, 1), **kw)
    ws = torch.empty(kdt.kdt_workspace_size(p), dtype=torch.uint8, device=dev)
    cap = spec.depth
    out = kdt.Tree(torch.empty(spec.n, dtype=torch.int32, device=dev),
                   torch.empty((1 << cap) - 1, dtype=torch.float32, device=dev),
                   torch.empty((1 << cap) - 1, dtype=torch.int8, device=dev),
                   torch.empty((1 << cap) + 1, dtype=torch.int64, device=dev), 0)
    stream = torch.cuda.current_stream(dev)
    t = kdt.kdt_build(pts, sid=sid, workspace=ws, outputs=out, stream=stream, **kw)
    torch.cuda.synchronize()
    del ws
    return pts, sid, t


def host_tree(t) -> oracle.Tree:
    return oracle.Tree(t.perm.cpu().numpy().view(np.uint32), t.split_vals.cpu().numpy(),
                       t.split_dims.cpu().numpy(), t.node_offsets.cpu().numpy(), t.levels)


def run_exact(name, jobs):
    spec, kw, pts, sid, fut = jobs[name]
    pts, sid, t = bench_build(spec, kw, pts, sid)
    assert t.levels == spec.depth
    check_tree_device(pts, t.perm, t.split_vals, t.split_dims, t.node_offsets, t.levels, spec.key_rule)
    g = host_tree(t)
    del t
    torch.cuda.empty_cache()
    assert_same_tree(g, fut.result(), name)


def run_sampled(spec, kw, levels, seed):
    pts, sid, t = bench_build(spec, kw)
    assert t.levels == spec.depth
    check_tree_device(pts, t.perm, t.split_vals, t.split_dims, t.node_offsets, t.levels, spec.key_rule)
    L = t.levels
    g = host_tree(t)
    pts_h, sid_h = pts.cpu().numpy(), host_sids(sid)
    del pts, sid, t
    torch.cuda.empty_cache()
    check_sampled_nodes(spec, pts_h, sid_h, g.perm, g.split_vals, g.split_dims, g.node_offsets, L, levels, seed)


def test_config3_full_size_bit_exact(exact_jobs):
    assert exact_jobs["c3"][0].n == 1 << 27 and exact_jobs["c3"][0].depth == 20
    run_exact("c3", exact_jobs)


def test_config2_full_size_bit_exact(exact_jobs):
    assert exact_jobs["c2"][0].n == 1 << 24 and exact_jobs["c2"][0].depth == 16
    run_exact("c2", exact_jobs)


def test_paper_simulation_shape_full_size_bit_exact(exact_jobs):
    run_exact("w6_rho0.5", exact_jobs)


@pytest.mark.parametrize("rho", [0.0, 0.25, 0.75])
def test_paper_simulation_shape_full_size(rho):
    spec = workloads.paper_mvn(1 << 27, rho, 10)
    kw = dict(r=spec.r, subset_mode=spec.subset_mode, depth=spec.depth, key_rule=spec.key_rule,
              leaf_size=spec.leaf_size, max_levels=spec.max_levels)
    run_sampled(spec, kw, [3, 6, 9, 9], seed=int(rho * 100))


def compare_in_pool(cases, what):
    """cases: (host points, host ids, oracle kwargs, host Tree of the GPU).
    Builds each with the oracle in the pool and compares bit for bit."""
    futs = {oracle_pool().submit(oracle.build_tree, p, sid=s, **kw): (i, g) for i, (p, s, kw, g) in enumerate(cases)}
    for f in cf.as_completed(futs):
        i, g = futs[f]
        assert_same_tree(g, f.result(), f"{what} {i}")


def test_config4_all_trees_bit_exact():
    """The whole batched recipe (4096 trees, 5.1e8 points) in one
    kdt_build_batched call, each tree against the oracle."""
    from paper_2201_08288_gb300 import kdt
    dev = torch.device("cuda:0")
    specs = workloads.config4_batch(num_trees=4096)
    items = [dict(points=s.points_device(dev), r=s.r, subset_mode=0, depth=0, leaf_size=32,
                  max_levels=s.max_levels, key_rule=0) for s in specs]
    descs, outs = kdt.make_descs(items)
    ws = torch.empty(kdt.kdt_workspace_size_batched(descs), dtype=torch.uint8, device=dev)
    trees, st = kdt.kdt_build_batched(items, workspace=ws, outputs=outs, descs=descs,
                                      stream=torch.cuda.current_stream(dev))
    torch.cuda.synchronize()
    assert st == [0] * len(items)
    del ws
    cases = []
    for it, t in zip(items, trees):
        kw = {k: it[k] for k in ("r", "subset_mode", "depth", "leaf_size", "max_levels", "key_rule")}
        cases.append((it["points"].cpu().numpy(), None, kw, host_tree(t)))
    del items, trees, outs, descs
    torch.cuda.empty_cache()
    compare_in_pool(cases, "config-4 tree")


def test_config5_sample_through_server_bit_exact():
    """200 requests of the 20000-request serving stream (seeded: the 10
    largest and 190 drawn at random), submitted to the server in arrival
    order, a few at a time while earlier ones are still running; every result
    against the oracle."""
    from paper_2201_08288_gb300 import kdt
    dev = torch.device("cuda:0")
    _, specs = workloads.config5_stream(num_requests=20000, rate=1.0)
    sizes = np.array([s.n for s in specs])
    largest = np.argsort(-sizes, kind="stable")[:10]
    rest = np.setdiff1d(np.arange(len(specs)), largest)
    pick = np.sort(np.concatenate([largest, np.random.default_rng(5).choice(rest, 190, replace=False)]))
    kw_of = lambda s: dict(r=32, subset_mode=0, depth=0, leaf_size=64, max_levels=s.max_levels, key_rule=0)
    cases = []
    with kdt.Server(64 << 30, 256) as sv:
        live = {}
        peak = 0
        for j, i in enumerate(pick):
            s = specs[i]
            item = dict(points=s.points_device(dev), **kw_of(s))
            live[sv.submit(item)] = (s, item)
            peak = max(peak, len(live))
            if j % 8 == 7:  # reap what has finished, keep the rest running
                for tk in list(live):
                    r = sv.poll(tk, 0)
                    if r is not None:
                        s0, it0 = live.pop(tk)
                        assert r[0] == 0, (s0.name, r[0])
                        cases.append((it0["points"].cpu().numpy(), None, kw_of(s0), host_tree(r[1])))
        for tk in list(live):
            r = sv.poll(tk)
            s0, it0 = live.pop(tk)
            assert r[0] == 0, (s0.name, r[0])
            cases.append((it0["points"].cpu().numpy(), None, kw_of(s0), host_tree(r[1])))
        info = sv.stats()
    assert len(cases) == 200 and info["peak_in_flight"] > 1
    torch.cuda.empty_cache()
    compare_in_pool(cases, "config-5 request")
