"""GPU test of kdt_build_noalloc, the entry point for callers that cannot
allocate device memory (it uses the library's fixed 64 MiB device scratch
array as its workspace). Its results must equal kdt_build's on the same
inputs, on two calls in a row, and after a larger problem has left its
tables in the shared scratch array. Collected last on purpose."""
from __future__ import annotations

import numpy as np
import pytest

from gpu_util import require_gpu
from paper_2201_08288_gb300 import workloads

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _outputs(n, cap, dev):
    from paper_2201_08288_gb300 import kdt
    return kdt.Tree(torch.empty(max(n, 1), dtype=torch.int32, device=dev),
                    torch.empty(max((1 << cap) - 1, 1), dtype=torch.float32, device=dev),
                    torch.empty(max((1 << cap) - 1, 1), dtype=torch.int8, device=dev),
                    torch.empty((1 << cap) + 1, dtype=torch.int64, device=dev), 0)


def _host(t):
    return (t.perm.cpu().numpy(), t.split_vals.cpu().numpy().view(np.uint32), t.split_dims.cpu().numpy(),
            t.node_offsets.cpu().numpy(), t.levels)


@pytest.mark.parametrize("case", ["cyclic_mod", "widest_explicit", "leaf_mode"])
def test_noalloc_matches_kdt_build_twice(case):
    from paper_2201_08288_gb300 import kdt
    dev = torch.device("cuda:0")
    if case == "cyclic_mod":
        pts = workloads.uniform(60000, 3, seed=11)
        sid = None
        kw = dict(r=8, subset_mode=0, depth=9, key_rule=0)
    elif case == "widest_explicit":
        pts = workloads.student_t_snapped(90000, 4, 3.0, 0.1, 256, seed=12)
        sid = workloads.explicit_sids(90000, 64, seed=13)
        kw = dict(r=64, subset_mode=2, depth=10, key_rule=1)
    else:
        pts = workloads.gaussian_mixture(40000, 3, 8, 0.05, seed=14)
        sid = None
        kw = dict(r=16, subset_mode=0, depth=0, leaf_size=32, max_levels=16, key_rule=0)
    P = torch.from_numpy(pts).to(dev)
    S = torch.from_numpy(sid).to(dev) if sid is not None else None
    cap = kw["depth"] if kw["depth"] > 0 else kw["max_levels"]
    ref = _host(kdt.kdt_build(P, sid=S, outputs=_outputs(P.shape[1], cap, dev), **kw))
    for _ in range(2):
        got = _host(kdt.kdt_build_noalloc(P, sid=S, outputs=_outputs(P.shape[1], cap, dev), **kw))
        torch.cuda.synchronize()
        assert got[4] == ref[4]
        for a, b in zip(got[:4], ref[:4]):
            np.testing.assert_array_equal(a, b)


def test_noalloc_over_a_larger_problems_leftovers():
    """A larger widest-spread build fills more of the shared scratch array
    with its tables; a smaller leaf-mode build that follows runs over those
    leftovers and must still give kdt_build's bits (a counter that the build
    failed to clear would show here)."""
    from paper_2201_08288_gb300 import kdt
    dev = torch.device("cuda:0")
    big = workloads.student_t_snapped(400000, 6, 3.0, 0.1, 256, seed=21)
    big_sid = workloads.explicit_sids(400000, 200, seed=22)
    P = torch.from_numpy(big).to(dev)
    S = torch.from_numpy(big_sid).to(dev)
    kw_big = dict(r=200, subset_mode=2, depth=12, key_rule=1)
    got_big = _host(kdt.kdt_build_noalloc(P, sid=S, outputs=_outputs(P.shape[1], 12, dev), **kw_big))
    ref_big = _host(kdt.kdt_build(P, sid=S, outputs=_outputs(P.shape[1], 12, dev), **kw_big))
    small = workloads.gaussian_mixture(30000, 3, 8, 0.05, seed=23)
    Q = torch.from_numpy(small).to(dev)
    kw_small = dict(r=16, subset_mode=0, depth=0, leaf_size=32, max_levels=16, key_rule=0)
    got = _host(kdt.kdt_build_noalloc(Q, outputs=_outputs(Q.shape[1], 16, dev), **kw_small))
    ref = _host(kdt.kdt_build(Q, outputs=_outputs(Q.shape[1], 16, dev), **kw_small))
    torch.cuda.synchronize()
    for g, r in ((got_big, ref_big), (got, ref)):
        assert g[4] == r[4]
        for a, b in zip(g[:4], r[:4]):
            np.testing.assert_array_equal(a, b)


def test_noalloc_rejects_problems_beyond_the_scratch_size():
    from paper_2201_08288_gb300 import kdt
    dev = torch.device("cuda:0")
    n, d = 4_000_000, 3
    P = torch.zeros((d, n), dtype=torch.float32, device=dev)
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_build_noalloc(P, r=4, depth=4, outputs=_outputs(n, 4, dev))
    assert e.value.status == 5
