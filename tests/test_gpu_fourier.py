"""GPU tests of the paper's own estimator (fourier_j > 0: every split is the
root of Eq. (kd:eq:b) built from the cell's sums of Lemma 1's basis terms).
The GPU adds float32 basis terms and the oracle float64 ones, so the splits
agree within a tolerance derived from that arithmetic (devcheck.py); what
the splits fix is exact: the permutation, the leaves' order, the cyclic
keys, every point's side of every split above it, and the sentinel of empty
nodes. Each node's split is compared with the oracle's root for the points
the GPU put in that node."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from devcheck import check_fourier_nodes, check_tree_device
from gpu_util import gpu_build, require_gpu
from paper_2201_08288_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def check_tree(pts, g, J, heaps=None):
    check_tree_device(torch.from_numpy(pts), torch.from_numpy(g.perm.astype(np.int64)),
                      torch.from_numpy(g.split_vals), torch.from_numpy(g.split_dims),
                      torch.from_numpy(g.node_offsets), g.levels, 0, fourier=True)
    if heaps is None:
        heaps = range((1 << g.levels) - 1)
    return check_fourier_nodes(pts, g.perm, g.split_vals, g.split_dims, g.node_offsets, g.levels, J, heaps)


@pytest.mark.parametrize("n,d,depth,J", [(1, 1, 3, 4), (5, 2, 4, 1), (1000, 3, 6, 8), (4099, 2, 8, 16),
                                         (70001, 3, 7, 32), (300000, 3, 10, 16)])
def test_every_node_matches_the_oracle(n, d, depth, J):
    pts = workloads.uniform_open(n, d, seed=n + depth)
    g = gpu_build(pts, depth=depth, fourier_j=J)
    assert g.levels == depth
    check_tree(pts, g, J)


def test_correlated_normal_shape():
    """Sec. 5's trivariate normal (rho = 0.75) mapped into (0,1) by the normal CDF."""
    spec = workloads.paper_mvn_fourier(200000, 0.75, 9, 16, seed=4)
    pts_t = spec.points_device("cuda")
    pts = pts_t.cpu().numpy()
    g = gpu_build(pts, depth=9, fourier_j=16)
    check_tree(pts, g, 16)


def test_subsets_do_not_change_the_splits():
    """The estimator's statistics are sums, which subsets add up (Sec. 3.2):
    r and the subset ids leave the tree unchanged, bit for bit."""
    pts = workloads.uniform_open(50000, 3, seed=9)
    base = gpu_build(pts, depth=8, fourier_j=12)
    sid = np.random.default_rng(1).integers(0, 37, size=50000).astype(np.uint8)
    for kw in (dict(r=64, subset_mode=0), dict(r=37, subset_mode=2, sid=sid), dict(r=5, subset_mode=1)):
        g = gpu_build(pts, depth=8, fourier_j=12, **kw)
        np.testing.assert_array_equal(g.perm, base.perm)
        np.testing.assert_array_equal(g.split_vals.view(np.uint32), base.split_vals.view(np.uint32))
        np.testing.assert_array_equal(g.node_offsets, base.node_offsets)


@pytest.mark.parametrize("bad,status", [(1.0, 1), (0.0, 1), (-0.25, 1), (np.nan, 2)])
def test_coordinates_outside_the_open_unit_interval_are_refused(bad, status):
    from paper_2201_08288_gb300 import kdt
    pts = workloads.uniform_open(5000, 2, seed=2)
    pts[1, 4321] = bad
    with pytest.raises(kdt.KdtError) as e:
        gpu_build(pts, depth=3, fourier_j=4)
    assert e.value.status == status


@pytest.mark.parametrize("kw", [dict(fourier_j=33, depth=4), dict(fourier_j=-1, depth=4),
                                dict(fourier_j=4, depth=4, key_rule=1), dict(fourier_j=4, depth=0, leaf_size=8)])
def test_parameter_combinations_refused(kw):
    from paper_2201_08288_gb300 import kdt
    pts = workloads.uniform_open(100, 2, seed=3)
    with pytest.raises(kdt.KdtError) as e:
        gpu_build(pts, **kw)
    assert e.value.status == 1


@pytest.mark.parametrize("rho", [0.0, 0.5])
def test_full_size_paper_shape(rho):
    """n = 2^27 (Sec. 5's trivariate normal, through the normal CDF), depth 10,
    J = 16, built as bench.py's w6f workload: every node checked on the device,
    nodes of levels 5-9 against the oracle."""
    from devcheck import check_tree_device as dev_check
    spec = workloads.paper_mvn_fourier(1 << 27, rho, 10, 16)
    pts = spec.points_device("cuda")
    from paper_2201_08288_gb300 import kdt
    t = kdt.kdt_build(pts, depth=10, fourier_j=16)
    torch.cuda.synchronize()
    dev_check(pts, t.perm, t.split_vals, t.split_dims, t.node_offsets, t.levels, 0, fourier=True)
    pts_h = pts.cpu().numpy()
    perm, vals = t.perm.cpu().numpy().view(np.uint32), t.split_vals.cpu().numpy()
    dims, offs = t.split_dims.cpu().numpy(), t.node_offsets.cpu().numpy()
    rng = np.random.default_rng(int(rho * 10))
    heaps = [(1 << lv) - 1 + int(rng.integers(0, 1 << lv)) for lv in (5, 6, 7, 8, 9, 9, 9)]
    check_fourier_nodes(pts_h, perm, vals, dims, offs, 10, 16, heaps)
