"""Checks on a built tree that hold for any input and any size (P7 invariants).

A tree is (perm, split_vals, split_dims, node_offsets, L). Node h at level l
(heap order, children 2h+1 and 2h+2) covers the leaves
[k 2^(L-l), (k+1) 2^(L-l)) with k = h - (2^l - 1), hence the positions
[offs[k 2^(L-l)], offs[(k+1) 2^(L-l)]) of perm.
"""
from __future__ import annotations

import numpy as np


def le_total(x: np.ndarray, m: float) -> np.ndarray:
    """x <= m in the total order of floats where -0.0 < +0.0 (no NaN)."""
    x = np.asarray(x, dtype=np.float32)
    m = np.float32(m)
    eq = x == m
    return (x < m) | (eq & (np.signbit(x) | ~np.signbit(m)))


def node_range(offs: np.ndarray, L: int, heap: int):
    level = int(np.floor(np.log2(heap + 1)))
    k = heap - ((1 << level) - 1)
    span = 1 << (L - level)
    return int(offs[k * span]), int(offs[(k + 1) * span]), level


def check_invariants(points: np.ndarray, perm, vals, dims, offs, L: int):
    """Raises AssertionError on the first violated invariant."""
    points = np.asarray(points, dtype=np.float32)
    d, n = points.shape
    perm = np.asarray(perm, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float32)
    dims = np.asarray(dims, dtype=np.int64)
    offs = np.asarray(offs, dtype=np.int64)
    assert perm.shape == (n,)
    assert np.array_equal(np.sort(perm), np.arange(n)), "perm is not a permutation"
    assert offs.shape == ((1 << L) + 1,)
    assert offs[0] == 0 and offs[-1] == n, "offsets do not span [0, n)"
    assert np.all(np.diff(offs) >= 0), "offsets not monotone"
    assert vals.shape == ((1 << L) - 1,) and dims.shape == vals.shape
    for k in range(1 << L):
        leaf = perm[offs[k]:offs[k + 1]]
        assert np.all(np.diff(leaf) > 0), f"leaf {k} not in increasing original order"
    for h in range((1 << L) - 1):
        b, e, level = node_range(offs, L, h)
        lb, le, _ = node_range(offs, L, 2 * h + 1)
        rb, re, _ = node_range(offs, L, 2 * h + 2)
        assert lb == b and le == rb and re == e, f"children of {h} do not tile it"
        t = int(dims[h])
        if t < 0:
            assert t == -1 and np.isposinf(vals[h]), f"bad sentinel at {h}"
            assert rb == re, f"sentinel node {h} has a non-empty right child"
            continue
        assert 0 <= t < d
        idx = perm[b:e]
        assert idx.size > 0, f"split recorded on empty node {h}"
        col = points[t, idx]
        m = vals[h]
        left = points[t, perm[lb:le]]
        right = points[t, perm[rb:re]]
        assert np.all(le_total(left, m)), f"node {h}: a left point is above the split"
        assert not np.any(le_total(right, m)), f"node {h}: a right point is at or below the split"
        assert np.any(col.view(np.uint32) == np.float32(m).view(np.uint32)), \
            f"node {h}: split value is not a coordinate of the node"


def quartile_bound_ok(points, perm, vals, dims, offs, L) -> bool:
    """P5: #{key <= m} >= ceil(W/4) and #{key >= m} > W/4 at every split."""
    points = np.asarray(points, dtype=np.float32)
    for h in range((1 << L) - 1):
        t = int(dims[h])
        if t < 0:
            continue
        b, e, _ = node_range(offs, L, h)
        col = points[t, np.asarray(perm[b:e], dtype=np.int64)]
        W = col.size
        m = vals[h]
        le = int(np.count_nonzero(le_total(col, m)))
        lt = int(np.count_nonzero(le_total(col, m) & (col.view(np.uint32) != np.float32(m).view(np.uint32))))
        ge = W - lt
        if not (4 * le >= W and 4 * ge > W):
            return False
    return True
