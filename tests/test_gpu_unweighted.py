"""GPU: the unweighted combine (kdt_params.combine_rule =
KDT_COMBINE_UNWEIGHTED: every non-empty subset's lower median counts once)
gives the oracle's bits through every path that forms a split: the CTA and
warp combines of the multi-CTA pipeline, the subtree kernel's warp combine,
batched builds and the sharded build; and it differs from the weighted rule
where the subsets' sizes differ."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import assert_same_tree, check_against_oracle, gpu_build, require_gpu
from paper_2201_08288_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 1  # KDT_COMBINE_UNWEIGHTED


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _host(t):
    return oracle.Tree(t.perm.cpu().numpy().view(np.uint32), t.split_vals.cpu().numpy(),
                       t.split_dims.cpu().numpy(), t.node_offsets.cpu().numpy(), t.levels)


@pytest.mark.parametrize("case", range(6))
def test_unweighted_rule_matches_oracle(case):
    rng = np.random.default_rng(600 + case)
    if case == 0:  # few cells (CTA combine), then the subtree
        pts = workloads.uniform(200000, 3, seed=61)
        kw = dict(r=16, subset_mode=0, depth=11)
    elif case == 1:  # explicit ids of very different sizes, widest
        pts = workloads.student_t_snapped(150000, 6, 3.0, 0.1, 256, seed=62)
        sid = np.minimum(rng.geometric(0.05, 150000) - 1, 99).astype(np.uint8)
        check_against_oracle(pts, sid=sid, r=100, subset_mode=2, depth=10, key_rule=1, combine_rule=U)
        return
    elif case == 2:  # many cells per step (warp combine), contiguous subsets
        pts = workloads.gaussian_mixture(1 << 22, 3, 8, 0.05, seed=63)
        kw = dict(r=64, subset_mode=1, depth=14)
    elif case == 3:  # leaf mode with ties
        pts = rng.integers(-8, 9, (2, 60000)).astype(np.float32) / 4
        kw = dict(r=7, subset_mode=0, depth=0, leaf_size=24, max_levels=24)
    elif case == 4:  # a small tree: subtree kernel only
        pts = workloads.uniform(1200, 4, seed=64)
        kw = dict(r=9, subset_mode=0, depth=7, key_rule=1)
    else:  # singleton subsets: the exact lower median either way
        pts = workloads.uniform(3000, 2, seed=65)
        check_against_oracle(pts, sid=np.arange(3000).astype(np.uint16), r=3000, subset_mode=2, depth=6,
                             combine_rule=U)
        return
    g = check_against_oracle(pts, combine_rule=U, **kw)
    if case in (0, 2):
        w = gpu_build(pts, **kw)
        assert not np.array_equal(g.split_vals.view(np.uint32), w.split_vals.view(np.uint32))


def test_unweighted_rule_batched_and_sharded():
    from paper_2201_08288_gb300 import kdt
    rng = np.random.default_rng(7)
    pts = workloads.student_t_snapped(120000, 4, 3.0, 0.1, 256, seed=66)
    sid = np.minimum(rng.geometric(0.08, 120000) - 1, 31).astype(np.uint8)
    P, S = torch.from_numpy(pts).cuda(), torch.from_numpy(sid).cuda()
    kw = dict(r=32, subset_mode=2, depth=9, key_rule=1, combine_rule=U)
    ref = oracle.build_tree(pts, sid=sid, **kw)
    items = [dict(points=P, sid=S, **kw), dict(points=torch.from_numpy(workloads.uniform(9000, 3, seed=67)).cuda(),
                                             r=5, depth=5, combine_rule=U)]
    trees, st = kdt.kdt_build_batched(items)
    assert st == [0, 0]
    assert_same_tree(_host(trees[0]), ref, "batched")
    for shards in (2, 5):
        assert_same_tree(_host(kdt.kdt_build_sharded(P, shards, sid=S, **kw)), ref, f"sharded G={shards}")
