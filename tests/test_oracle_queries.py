"""Pins of the query definitions in oracle/ (CPU): the box test against a
plain per-point loop with hand-checked cases (-0.0 below +0.0, inclusive
edges), the squared distance against a closed form, and the k nearest
against a full sort, ties by index."""
from __future__ import annotations

import numpy as np

import oracle


def test_box_members_hand_cases_and_loop():
    pts = np.array([[-0.0, 0.0, 1.0, 2.0, 2.0, 3.0], [5.0, 5.0, 5.0, 5.0, 6.0, 5.0]], np.float32)
    # +0 excludes -0 (key order), the upper edge is inclusive
    got = oracle.box_members(pts, np.array([0.0, 5.0], np.float32), np.array([2.0, 5.0], np.float32))
    assert got.tolist() == [1, 2, 3]
    got = oracle.box_members(pts, np.array([-0.0, 0.0], np.float32), np.array([0.0, 10.0], np.float32))
    assert got.tolist() == [0, 1]
    rng = np.random.default_rng(3)
    pts = rng.integers(-4, 5, (3, 400)).astype(np.float32) / 2
    for _ in range(20):
        lo = rng.integers(-4, 5, 3).astype(np.float32) / 2
        hi = lo + rng.integers(0, 4, 3).astype(np.float32) / 2
        want = [i for i in range(400) if all(lo[j] <= pts[j, i] <= hi[j] for j in range(3))
                and not any(pts[j, i] == 0 and lo[j] == 0 and (np.signbit(pts[j, i]) < np.signbit(lo[j]))
                            for j in range(3))]
        assert oracle.box_members(pts, lo, hi).tolist() == want


def test_squared_distance_closed_form_and_nearest_by_sort():
    pts = np.array([[0.0, 3.0, -3.0, 0.0, 1.0], [0.0, 4.0, 4.0, 5.0, 1.0]], np.float32)
    d2 = oracle.squared_distances(pts, np.array([0.0, 0.0], np.float32))
    assert d2.tolist() == [0.0, 25.0, 25.0, 25.0, 2.0]
    idx, dd = oracle.nearest(pts, np.array([0.0, 0.0], np.float32), 4)
    assert idx.tolist() == [0, 4, 1, 2] and dd.tolist() == [0.0, 2.0, 25.0, 25.0]  # ties: smaller index first
    rng = np.random.default_rng(4)
    pts = rng.standard_normal((4, 300)).astype(np.float32)
    q = rng.standard_normal(4).astype(np.float32)
    full = sorted(range(300), key=lambda i: (sum((float(pts[j, i]) - float(q[j])) ** 2 for j in range(4)), i))
    idx, _ = oracle.nearest(pts, q, 10)
    assert idx.tolist() == full[:10]
