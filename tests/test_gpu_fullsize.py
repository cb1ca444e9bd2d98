"""GPU parity at the benchmark's full sizes, built the way bench.py times the
build (the same workload recipe and parameters, a preallocated workspace and
preallocated outputs, the caller's stream, the default tuning): config 3
(n = 2^27, d = 8, r = 256 explicit, widest spread, depth 20), config 2
(n = 2^24, d = 3, r = 64 contiguous, cyclic, depth 16) and the simulation
shape of Sec. 5 (trivariate normal with common correlation rho, n = 2^27,
r = 64 by index, cyclic, depth 10).

The oracle cannot build trees of this size within a test, so every node is
checked on the device against the properties that fix the tree given its
splits (devcheck.py), and the splits of sampled nodes, the root among them,
are recomputed by the oracle from the points the GPU put in each node."""
from __future__ import annotations

import numpy as np
import pytest

import bench
from devcheck import check_sampled_nodes, check_tree_device
from gpu_util import require_gpu
from paper_2201_08288_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def bench_build(spec, kw):
    from paper_2201_08288_gb300 import kdt
    dev = torch.device("cuda:0")
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


def run_fullsize(spec, kw, levels, seed):
    pts, sid, t = bench_build(spec, kw)
    assert t.levels == spec.depth
    check_tree_device(pts, t.perm, t.split_vals, t.split_dims, t.node_offsets, t.levels, spec.key_rule)
    L = t.levels
    perm = t.perm.cpu().numpy().view(np.uint32)
    vals = t.split_vals.cpu().numpy()[:(1 << L) - 1]
    dims = t.split_dims.cpu().numpy()[:(1 << L) - 1]
    offs = t.node_offsets.cpu().numpy()[:(1 << L) + 1]
    pts_h = pts.cpu().numpy()
    sid_h = sid.cpu().numpy().view(np.uint16 if sid.element_size() == 2 else np.uint8) if sid is not None else None
    del pts, sid, t
    torch.cuda.empty_cache()
    check_sampled_nodes(spec, pts_h, sid_h, perm, vals, dims, offs, L, levels, seed)


def test_config3_full_size():
    spec, kw = bench.workload("c3", 0)
    assert spec.n == 1 << 27 and spec.depth == 20
    run_fullsize(spec, kw, [0, 3, 7, 11, 14, 17, 19, 19, 19], seed=3)


def test_config2_full_size():
    spec, kw = bench.workload("c2", 0)
    assert spec.n == 1 << 24 and spec.depth == 16
    run_fullsize(spec, kw, [0, 1, 2, 5, 9, 13, 15, 15, 15], seed=2)


@pytest.mark.parametrize("rho", [0.0, 0.25, 0.5, 0.75])
def test_paper_simulation_shape_full_size(rho):
    spec = workloads.paper_mvn(1 << 27, rho, 10)
    kw = dict(r=spec.r, subset_mode=spec.subset_mode, depth=spec.depth, key_rule=spec.key_rule,
              leaf_size=spec.leaf_size, max_levels=spec.max_levels)
    run_fullsize(spec, kw, [3, 6, 9, 9], seed=int(rho * 100))
