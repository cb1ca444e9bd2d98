"""GPU: the sharded build (kdt_build_sharded: G logical shards, subset s on
shard s % G, the per-level all-gather of the (cell, subset) medians and
sizes, and for widest spread of the per-coordinate min / max; local
partitions; leaves merged by original index) gives the same bits as the
build on one GPU and as the oracle, for G = 1, 2, 3, 4, 8 and 16, every
subset mode and both key rules, with shards that own no subset (r < G), an
empty input and a single subset."""
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


def _host(t):
    return oracle.Tree(t.perm.cpu().numpy().view(np.uint32), t.split_vals.cpu().numpy(),
                       t.split_dims.cpu().numpy(), t.node_offsets.cpu().numpy(), t.levels)


CASES = {
    "uniform_mod_cyclic": (lambda: (workloads.uniform(100000, 3, seed=51), None), dict(r=8, subset_mode=0, depth=9)),
    "studentt_explicit_widest": (lambda: (workloads.student_t_snapped(150000, 8, 3.0, 0.1, 256, seed=52),
                                          workloads.explicit_sids(150000, 64, seed=53)),
                                 dict(r=64, subset_mode=2, depth=10, key_rule=1)),
    "mixture_contiguous_cyclic": (lambda: (workloads.gaussian_mixture(80000, 3, 8, 0.05, seed=54), None),
                                  dict(r=16, subset_mode=1, depth=8)),
    "few_subsets_widest": (lambda: (workloads.student_t_snapped(20000, 4, 3.0, 0.1, 256, seed=55), None),
                           dict(r=3, subset_mode=0, depth=7, key_rule=1)),
    "one_subset": (lambda: (workloads.uniform(30000, 2, seed=56), None), dict(r=1, subset_mode=0, depth=6)),
    "large_leaves": (lambda: (workloads.uniform(300000, 3, seed=57), None), dict(r=32, subset_mode=0, depth=4)),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("shards", [1, 2, 3, 4, 8, 16])
def test_sharded_equals_one_gpu_and_oracle(case, shards):
    from paper_2201_08288_gb300 import kdt
    make, kw = CASES[case]
    pts, sid = make()
    P = torch.from_numpy(pts).cuda()
    S = torch.from_numpy(sid).cuda() if sid is not None else None
    got = _host(kdt.kdt_build_sharded(P, shards, sid=S, **kw))
    ref = _host(kdt.kdt_build(P, sid=S, **kw))
    assert_same_tree(got, ref, f"{case} G={shards} vs kdt_build")
    if shards in (1, 4):
        assert_same_tree(got, oracle.build_tree(pts, sid=sid, **kw), f"{case} G={shards} vs oracle")


def test_sharded_empty_input_and_errors():
    from paper_2201_08288_gb300 import kdt
    P = torch.zeros((3, 0), dtype=torch.float32, device="cuda")
    t = _host(kdt.kdt_build_sharded(P, 4, r=8, depth=3))
    assert t.levels == 3 and np.all(t.node_offsets == 0) and np.all(t.split_dims == -1)
    Q = torch.from_numpy(workloads.uniform(1000, 3, seed=58)).cuda()
    for bad in (dict(shards=0), dict(shards=17)):
        with pytest.raises(kdt.KdtError) as e:
            kdt.kdt_build_sharded(Q, bad["shards"], r=4, depth=3)
        assert e.value.status == 1
    pts = workloads.uniform(1000, 3, seed=59)
    pts[1, 17] = np.nan
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_build_sharded(torch.from_numpy(pts).cuda(), 2, r=4, depth=3)
    assert e.value.status == 2
