"""The device-side tree checks (devcheck.py) run here with torch on the CPU:
they accept the oracle's trees, and each planted mistake in a tree's outputs
is caught."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from devcheck import check_tree_device

torch = pytest.importorskip("torch")


def _case(kind):
    rng = np.random.default_rng(11)
    if kind == "widest":
        pts = rng.standard_t(3.0, size=(4, 5000)).astype(np.float32)
        pts[:, ::7] = np.rint(pts[:, ::7] * 4) / 4  # ties
        sid = rng.integers(0, 8, size=5000).astype(np.uint8)
        kw = dict(r=8, subset_mode=2, sid=sid, depth=7, key_rule=1)
    elif kind == "cyclic":
        pts = rng.random((3, 3000)).astype(np.float32)
        kw = dict(r=5, subset_mode=0, depth=6, key_rule=0)
    else:  # more levels than points: empty cells get the terminal sentinel
        pts = rng.random((2, 40)).astype(np.float32)
        kw = dict(r=3, subset_mode=1, depth=7, key_rule=0)
    t = oracle.build_tree(pts, **kw)
    return pts, kw["key_rule"], t


def _check(pts, key_rule, perm, vals, dims, offs, L):
    check_tree_device(torch.from_numpy(pts), torch.from_numpy(perm.astype(np.int64)),
                      torch.from_numpy(vals), torch.from_numpy(dims), torch.from_numpy(offs), L, key_rule)


@pytest.mark.parametrize("kind", ["widest", "cyclic", "empty_cells"])
def test_accepts_the_oracles_trees(kind):
    pts, key_rule, t = _case(kind)
    _check(pts, key_rule, t.perm, t.split_vals, t.split_dims, t.node_offsets, t.levels)


def _first_split(t, level):
    nodes = np.arange((1 << level) - 1, (1 << (level + 1)) - 1)
    return int(nodes[t.split_dims[nodes] >= 0][0])


@pytest.mark.parametrize("kind", ["widest", "cyclic"])
@pytest.mark.parametrize("mistake", ["perm_swap_in_leaf", "perm_swap_across", "split_next_float",
                                     "split_dim", "offset", "sentinel_value"])
def test_catches_planted_mistakes(kind, mistake):
    pts, key_rule, t = _case(kind)
    perm, vals = t.perm.copy(), t.split_vals.copy()
    dims, offs = t.split_dims.copy(), t.node_offsets.copy()
    L = t.levels
    if mistake == "perm_swap_in_leaf":
        k = int(np.argmax(np.diff(offs) >= 2))
        perm[offs[k]], perm[offs[k] + 1] = perm[offs[k] + 1], perm[offs[k]]
    elif mistake == "perm_swap_across":
        perm[0], perm[-1] = perm[-1], perm[0]
    elif mistake == "split_next_float":
        h = _first_split(t, 2)
        vals[h] = np.nextafter(vals[h], np.float32(np.inf), dtype=np.float32)
    elif mistake == "split_dim":
        h = _first_split(t, 3)
        dims[h] = (dims[h] + 1) % pts.shape[0]
    elif mistake == "offset":
        k = int(np.argmax(np.diff(offs) >= 2))
        offs[k + 1] += 1
    else:
        vals[0] = np.float32(np.inf)
    with pytest.raises(AssertionError):
        _check(pts, key_rule, perm, vals, dims, offs, L)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_sampled_node_check_accepts_the_oracles_trees(mode):
    """The oracle, given one node's points with explicit ids, agrees with the
    split it made inside its own build, for every subset mode."""
    from devcheck import check_sampled_nodes
    from paper_2201_08288_gb300 import workloads
    rng = np.random.default_rng(40 + mode)
    n, r = 6000, 7
    pts = rng.standard_normal((3, n)).astype(np.float32)
    sid = rng.integers(0, r, size=n).astype(np.uint8) if mode == 2 else None
    spec = workloads.TreeSpec("t", n, 3, "mvn", 0, r, mode, 1, depth=8)
    t = oracle.build_tree(pts, r=r, subset_mode=mode, sid=sid, depth=8, key_rule=1)
    check_sampled_nodes(spec, pts, sid, t.perm, t.split_vals, t.split_dims, t.node_offsets, t.levels,
                        [0, 1, 3, 5, 7, 7], seed=1)
    vals = t.split_vals.copy()
    vals[3] = np.nextafter(vals[3], np.float32(np.inf), dtype=np.float32)
    with pytest.raises(AssertionError):
        check_sampled_nodes(spec, pts, sid, t.perm, vals, t.split_dims, t.node_offsets, t.levels,
                            [2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2], seed=1)


def _fourier_case():
    from paper_2201_08288_gb300 import workloads
    pts = workloads.uniform_open(4000, 2, seed=21)
    return pts, oracle.fourier_build_tree(pts, depth=6, J=8)


def test_fourier_checks_accept_the_oracles_tree():
    from devcheck import check_fourier_nodes
    pts, t = _fourier_case()
    _check_f(pts, t.perm, t.split_vals, t.split_dims, t.node_offsets, t.levels)
    worst = check_fourier_nodes(pts, t.perm, t.split_vals, t.split_dims, t.node_offsets, t.levels, 8, range(63))
    assert worst < 1e-6


def _check_f(pts, perm, vals, dims, offs, L):
    check_tree_device(torch.from_numpy(pts), torch.from_numpy(perm.astype(np.int64)), torch.from_numpy(vals),
                      torch.from_numpy(dims), torch.from_numpy(offs), L, 0, fourier=True)


@pytest.mark.parametrize("mistake", ["split_off_by_a_thousandth", "split_dim", "perm_swap_across", "offset"])
def test_fourier_checks_catch_planted_mistakes(mistake):
    from devcheck import check_fourier_nodes
    pts, t = _fourier_case()
    perm, vals = t.perm.copy(), t.split_vals.copy()
    dims, offs = t.split_dims.copy(), t.node_offsets.copy()
    h = 5
    if mistake == "split_off_by_a_thousandth":
        a, b = oracle.fourier_cell_bounds(vals, h, 2)
        vals[h] = np.float32(vals[h] + 1e-3 * (b - a))
    elif mistake == "split_dim":
        dims[h] = 1 - dims[h]
    elif mistake == "perm_swap_across":
        perm[0], perm[-1] = perm[-1], perm[0]
    else:
        k = int(np.argmax(np.diff(offs) >= 2))
        offs[k + 1] += 1
    with pytest.raises(AssertionError):
        _check_f(pts, perm, vals, dims, offs, t.levels)
        check_fourier_nodes(pts, perm, vals, dims, offs, t.levels, 8, range(63))
