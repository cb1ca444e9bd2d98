"""GPU: box and k-nearest queries on built trees (kdt_query_box,
kdt_query_knn) give exactly the brute-force answers of oracle.box_members
and oracle.nearest: depth and leaf mode (terminal cells with sentinels),
both key rules, ties, duplicate points, signed zeros, boxes that are empty,
degenerate or cover everything, and fewer points than k."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import require_gpu
from paper_2201_08288_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _points(kind):
    rng = np.random.default_rng({"uniform": 1, "ties": 2, "studentt": 3}[kind])
    if kind == "uniform":
        return workloads.uniform(60000, 3, seed=71)
    if kind == "ties":  # a coarse grid: many equal coordinates and duplicate points, signed zeros
        p = rng.integers(-6, 7, (3, 40000)).astype(np.float32) / 4
        p[p == 0] = np.where(rng.random((p == 0).sum()) < 0.5, -0.0, 0.0)
        return p
    return workloads.student_t_snapped(50000, 5, 3.0, 0.1, 256, seed=72)


BUILDS = [("uniform", dict(r=8, depth=10)), ("ties", dict(r=4, depth=0, leaf_size=16, max_levels=26)),
          ("studentt", dict(r=16, depth=9, key_rule=1)), ("ties", dict(r=2, depth=6, key_rule=1))]


def _boxes(pts, nq, rng):
    d, n = pts.shape
    a = pts[:, rng.integers(0, n, nq)]
    b = pts[:, rng.integers(0, n, nq)]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    lo[:, 0], hi[:, 0] = -np.inf, np.inf  # everything
    lo[:, 1], hi[:, 1] = 1.0, -1.0        # nothing
    lo[:, 2] = hi[:, 2] = pts[:, 7]       # one point and its duplicates
    return lo.astype(np.float32), hi.astype(np.float32)


@pytest.mark.parametrize("case", range(len(BUILDS)))
def test_box_queries_equal_brute_force(case):
    from paper_2201_08288_gb300 import kdt
    kind, kw = BUILDS[case]
    pts = _points(kind)
    P = torch.from_numpy(pts).cuda()
    t = kdt.kdt_build(P, **kw)
    rng = np.random.default_rng(case)
    lo, hi = _boxes(pts, 300, rng)
    counts, lists = kdt.kdt_query_box(P, t, torch.from_numpy(lo).cuda(), torch.from_numpy(hi).cuda(),
                                      list_cap=pts.shape[1])
    counts, lists = counts.cpu().numpy(), lists.cpu().numpy()
    for q in range(lo.shape[1]):
        want = oracle.box_members(pts, lo[:, q], hi[:, q])
        assert counts[q] == want.size, f"box {q}"
        assert np.array_equal(np.sort(lists[q, :counts[q]]), want), f"box {q} members"


@pytest.mark.parametrize("case", range(len(BUILDS)))
@pytest.mark.parametrize("k", [1, 5, 17, 32])
def test_knn_equals_brute_force(case, k):
    from paper_2201_08288_gb300 import kdt
    kind, kw = BUILDS[case]
    pts = _points(kind)
    P = torch.from_numpy(pts).cuda()
    t = kdt.kdt_build(P, **kw)
    rng = np.random.default_rng(100 + case)
    q = np.concatenate([pts[:, rng.integers(0, pts.shape[1], 60)],
                        (pts[:, rng.integers(0, pts.shape[1], 60)] + rng.standard_normal((pts.shape[0], 60)) * 0.05)],
                       axis=1).astype(np.float32)
    idx, d2 = kdt.kdt_query_knn(P, t, torch.from_numpy(q).cuda(), k)
    idx, d2 = idx.cpu().numpy().view(np.uint32), d2.cpu().numpy()
    for j in range(q.shape[1]):
        wi, wd = oracle.nearest(pts, q[:, j], k)
        assert np.array_equal(idx[j], wi.astype(np.uint32)), f"query {j}"
        assert np.array_equal(d2[j], wd), f"query {j} distances"


def test_knn_with_fewer_points_than_k_and_argument_checks():
    from paper_2201_08288_gb300 import kdt
    pts = workloads.uniform(5, 2, seed=73)
    P = torch.from_numpy(pts).cuda()
    t = kdt.kdt_build(P, r=1, depth=2)
    q = torch.from_numpy(np.array([[0.5], [0.5]], np.float32)).cuda()
    idx, d2 = kdt.kdt_query_knn(P, t, q, 8)
    wi, wd = oracle.nearest(pts, np.array([0.5, 0.5], np.float32), 5)
    assert idx.cpu().numpy().view(np.uint32)[0, :5].tolist() == wi.tolist()
    assert np.all(idx.cpu().numpy().view(np.uint32)[0, 5:] == 0xFFFFFFFF) and np.all(np.isinf(d2.cpu().numpy()[0, 5:]))
    for bad_k in (0, 33):
        with pytest.raises(kdt.KdtError) as e:
            kdt.kdt_query_knn(P, t, q, bad_k)
        assert e.value.status == 1
