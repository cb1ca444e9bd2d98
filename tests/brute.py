"""A second, deliberately different reference used only to pin the C oracle.

Pure Python, recursive (depth first) instead of level by level, floats
compared through the total order (value, sign bit) instead of the uint32 key
map, per-subset medians from ``sorted`` on Python lists, and the combine rule
stated as "the smallest subset median v whose subsets with median <= v hold at
least half of the cell" instead of a cumulative scan over sorted pairs.
Slow: meant for n <= a few hundred.
"""
from __future__ import annotations

import math


def order_key(x: float):
    """Total order on non-NaN floats with -0.0 below +0.0."""
    return (x, 0 if math.copysign(1.0, x) < 0 else 1)


def subset_ids(n: int, r: int, mode: int, sid=None):
    if mode == 0:
        return [i % r for i in range(n)]
    if mode == 1:
        return [(i * r) // n for i in range(n)]
    return [int(s) for s in sid]


def lower_median(values):
    s = sorted(values, key=order_key)
    return s[(len(s) - 1) // 2]


def combine(meds_and_weights):
    """Smallest median v such that the subsets whose median is <= v hold >= half."""
    total = sum(w for _, w in meds_and_weights)
    best = None
    for v, _ in meds_and_weights:
        below = sum(w for u, w in meds_and_weights if order_key(u) <= order_key(v))
        if 2 * below >= total and (best is None or order_key(v) < order_key(best)):
            best = v
    return best


def widest_dim(cols, pts):
    best, best_range = 0, -1.0
    for l, col in enumerate(cols):
        vals = [col[i] for i in pts]
        hi = max(vals, key=order_key)
        lo = min(vals, key=order_key)
        rng = 0.0 if order_key(hi) == order_key(lo) else float(hi) - float(lo)
        if rng > best_range:
            best, best_range = l, rng
    return best


def split(cols, sids, pts, level, key_rule, combine_rule=0):
    """(dim, value) of a non-empty cell given its point indices; with
    combine_rule 1 every subset weighs one."""
    d = len(cols)
    t = level % d if key_rule == 0 else widest_dim(cols, pts)
    groups = {}
    for i in pts:
        groups.setdefault(sids[i], []).append(cols[t][i])
    meds = [(lower_median(v), 1 if combine_rule else len(v)) for v in groups.values()]
    return t, combine(meds)


def build(points, *, r=1, subset_mode=0, sid=None, depth=0, leaf_size=1, max_levels=20,
          key_rule=0, combine_rule=0):
    """Returns (perm, split_vals, split_dims, node_offsets, L) as Python lists."""
    cols = [[float(v) for v in row] for row in points]
    d = len(cols)
    n = len(cols[0]) if d else 0
    sids = subset_ids(n, r, subset_mode, sid)
    leaf_mode = depth == 0
    stall_limit = d if key_rule == 0 else 1

    def terminal(pts, stall):
        if leaf_mode:
            return len(pts) <= leaf_size or stall >= stall_limit
        return len(pts) == 0

    def children(pts, level, stall):
        """(dim, value, left, right, child_stall) of one node."""
        if terminal(pts, stall):
            return -1, math.inf, pts, [], stall
        t, m = split(cols, sids, pts, level, key_rule, combine_rule)
        left = [i for i in pts if order_key(cols[t][i]) <= order_key(m)]
        right = [i for i in pts if order_key(cols[t][i]) > order_key(m)]
        return t, m, left, right, (stall + 1 if not right else 0)

    # pass 1: depth of the tree (leaf mode: deepest non-terminal node + 1)
    if leaf_mode:
        def deepest(pts, level, stall):
            if terminal(pts, stall):
                return level
            if level == max_levels:
                raise OverflowError("level cap")
            _, _, lft, rgt, st = children(pts, level, stall)
            return max(deepest(lft, level + 1, st), deepest(rgt, level + 1, st))
        L = deepest(list(range(n)), 0, 0)
    else:
        L = depth

    vals = [0.0] * ((1 << L) - 1)
    dims = [0] * ((1 << L) - 1)
    leaves = [None] * (1 << L)

    def fill(pts, level, heap, stall):
        if level == L:
            leaves[heap - ((1 << L) - 1)] = pts
            return
        t, m, lft, rgt, st = children(pts, level, stall)
        dims[heap] = t
        vals[heap] = m
        fill(lft, level + 1, 2 * heap + 1, st)
        fill(rgt, level + 1, 2 * heap + 2, st)

    fill(list(range(n)), 0, 0, 0)
    perm, offs = [], []
    for lf in leaves:
        offs.append(len(perm))
        perm.extend(sorted(lf))
    offs.append(len(perm))
    return perm, vals, dims, offs, L
