"""GPU: many trees built together (kdt_build_batched) give, tree by tree, the
same bits as the oracle and as a solo kdt_build; a failing tree fails alone."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import assert_same_tree, require_gpu
from paper_2201_08288_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _host_tree(t):
    return oracle.Tree(t.perm.cpu().numpy().view(np.uint32), t.split_vals.cpu().numpy(),
                       t.split_dims.cpu().numpy(), t.node_offsets.cpu().numpy(), t.levels)


def _mixed_items(num, seed, n_hi=16.0):
    rng = np.random.default_rng(seed)
    specs = workloads.config4_batch(num_trees=num, n_lo=6.0, n_hi=n_hi)
    dev = torch.device("cuda:0")
    items, host = [], []
    for i, s in enumerate(specs):
        pts = s.points()
        kind = i % 4
        kw = dict(r=s.r, subset_mode=0, depth=0, leaf_size=32, max_levels=s.max_levels, key_rule=0)
        sid = None
        if kind == 1:
            kw.update(key_rule=1)
        elif kind == 2:
            kw.update(depth=int(rng.integers(1, 12)), leaf_size=1)
        elif kind == 3:
            kw.update(subset_mode=2, r=int(rng.integers(1, 300)), key_rule=int(rng.integers(0, 2)))
            sid = rng.integers(0, kw["r"], pts.shape[1]).astype(np.uint8 if kw["r"] <= 256 else np.uint16)
        item = dict(points=torch.from_numpy(pts).to(dev), **kw)
        if sid is not None:
            item["sid"] = torch.from_numpy(sid.view(np.int16) if sid.dtype == np.uint16 else sid).to(dev)
        items.append(item)
        host.append((pts, sid, kw))
    return items, host


def test_batched_matches_oracle_and_solo_per_tree():
    from paper_2201_08288_gb300 import kdt
    items, host = _mixed_items(48, 1)
    trees, stats = kdt.kdt_build_batched(items)
    torch.cuda.synchronize()
    assert stats == [0] * len(items)
    for i, ((pts, sid, kw), t) in enumerate(zip(host, trees)):
        ref = oracle.build_tree(pts, sid=sid, **kw)
        assert_same_tree(_host_tree(t), ref, f"tree {i}")
    # solo builds of a few of them give the same bits
    for i in (0, 5, 17, 33):
        it = {k: v for k, v in items[i].items() if k != "points"}
        solo = kdt.kdt_build(items[i]["points"], **it)
        torch.cuda.synchronize()
        assert_same_tree(_host_tree(solo), _host_tree(trees[i]), f"solo {i}")


def test_batched_with_large_trees_through_the_multi_cta_pipeline():
    from paper_2201_08288_gb300 import kdt
    items, host = _mixed_items(12, 2, n_hi=19.0)
    trees, stats = kdt.kdt_build_batched(items)
    torch.cuda.synchronize()
    assert stats == [0] * len(items)
    for i, ((pts, sid, kw), t) in enumerate(zip(host, trees)):
        assert_same_tree(_host_tree(t), oracle.build_tree(pts, sid=sid, **kw), f"tree {i}")


def test_a_failing_tree_fails_alone():
    from paper_2201_08288_gb300 import kdt
    items, host = _mixed_items(8, 3)
    bad = items[3]["points"].clone()
    bad[0, bad.shape[1] // 2] = float("nan")
    items[3]["points"] = bad
    trees, stats = kdt.kdt_build_batched(items)
    torch.cuda.synchronize()
    assert stats[3] == 2
    for i, ((pts, sid, kw), t) in enumerate(zip(host, trees)):
        if i == 3:
            continue
        assert stats[i] == 0
        assert_same_tree(_host_tree(t), oracle.build_tree(pts, sid=sid, **kw), f"tree {i}")
