"""Checks on a built tree, vectorised with torch so that they run on the
device at the benchmark's full sizes (2^27 points), on every node.

A tree is fixed by its splits: given each node's key coordinate and split key,
a stable partition places every point. So a tree is right when (1) every
point lies on the side of every split above it that its leaf says (left keys
<= split key < right keys, in the total order of the key transform: -0 < +0),
(2) perm is a permutation, increasing inside every leaf (the partition is
stable), (3) every split is the rule's: the key coordinate is the cyclic one
or the widest range (lowest coordinate on ties), and the split key is a key of
the node that satisfies the combine's quartile bound; the exact key of sampled
nodes is then recomputed by the oracle from the node's points.

Node h at level l (heap order) covers the leaves [k 2^(L-l), (k+1) 2^(L-l)),
k = h - (2^l - 1).
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
import treecheck


def ord_key(bits: torch.Tensor) -> torch.Tensor:
    """The order key of float32 bit patterns (int32 tensor) as int64: negative
    values map to the complement of their bits, the others get the top bit set
    (Sec. 2 compares reals; this is the integer order of float32 with -0 < +0)."""
    u = bits.to(torch.int64) & 0xFFFFFFFF
    return torch.where((u >> 31) == 1, u ^ 0xFFFFFFFF, u | 0x80000000)


def check_tree_device(pts: torch.Tensor, perm: torch.Tensor, vals: torch.Tensor, dims: torch.Tensor,
                      offs: torch.Tensor, L: int, key_rule: int, depth_mode: bool = True,
                      fourier: bool = False) -> None:
    """Raises AssertionError on the first violated property. pts: float32
    [d, n] on any device; perm int32/int64 [n]; vals float32 [2^L - 1]; dims
    int8 [2^L - 1]; offs int64 [2^L + 1]. fourier: the splits are the
    Fourier estimator's roots, not keys of their nodes (no key-of-node and
    quartile checks)."""
    dev = pts.device
    d, n = pts.shape
    perm = perm[:n].to(torch.int64)
    nodes = (1 << L) - 1
    vals = vals[:nodes]
    dims = dims[:nodes].to(torch.int64)
    offs = offs[:(1 << L) + 1].to(torch.int64)

    assert torch.equal(torch.sort(perm).values, torch.arange(n, device=dev)), "perm is not a permutation"
    assert int(offs[0]) == 0 and int(offs[-1]) == n, "offsets do not span [0, n)"
    cnt = offs[1:] - offs[:-1]
    assert bool((cnt >= 0).all()), "offsets not monotone"
    leaf = torch.repeat_interleave(torch.arange(1 << L, device=dev), cnt, output_size=n)
    same = leaf[1:] == leaf[:-1]
    assert bool(((perm[1:] > perm[:-1]) | ~same).all()), "a leaf is not in increasing original order"
    sent = dims < 0
    assert bool((dims[sent] == -1).all()), "split dims below -1"
    assert bool(torch.isposinf(vals[sent]).all()), "a terminal node's value is not +inf"
    assert bool((dims < d).all()), "split dim out of range"

    vkey = ord_key(vals.contiguous().view(torch.int32))
    xs = pts[:, perm]                       # coordinates in tree order
    xk = ord_key(xs.contiguous().view(torch.int32))
    pos = torch.arange(n, device=dev)
    for l in range(L):
        nn = 1 << l
        node = leaf >> (L - l)
        heap = node + (nn - 1)
        left = ((leaf >> (L - l - 1)) & 1) == 0
        tdim = dims[heap]
        term = tdim < 0
        assert not bool((term & ~left).any()), f"level {l}: a terminal node has points on its right"
        k = xk.view(-1)[tdim.clamp(min=0) * n + pos]
        m = vkey[heap]
        ok = torch.where(left, k <= m, k > m) | term
        assert bool(ok.all()), f"level {l}: a point lies on the wrong side of a split"

        def per_node(x):
            return torch.zeros(nn, dtype=torch.int64, device=dev).index_add_(0, node, x.to(torch.int64))

        W = per_node(torch.ones_like(node))
        eq = (k == m) & ~term
        n_le = per_node(left & ~term)
        n_ge = per_node((~left | eq) & ~term)
        n_eq = per_node(eq)
        ldims = dims[nn - 1:2 * nn - 1]
        split = ldims >= 0
        if depth_mode:
            assert torch.equal(split, W > 0), f"level {l}: a non-empty node without a split, or an empty one with"
        if not fourier:
            assert bool((n_eq[split] > 0).all()), f"level {l}: a split key is not a key of its node"
            assert bool((4 * n_le[split] >= W[split]).all()), f"level {l}: fewer than ceil(W/4) keys <= split"
            assert bool((4 * n_ge[split] > W[split]).all()), f"level {l}: no more than W/4 keys >= split"
        if key_rule == 0:
            assert bool((ldims[split] == l % d).all()), f"level {l}: not the cyclic coordinate"
        else:
            lo = torch.full((d, nn), float("inf"), dtype=torch.float32, device=dev)
            hi = torch.full((d, nn), float("-inf"), dtype=torch.float32, device=dev)
            for j in range(d):
                lo[j].scatter_reduce_(0, node, xs[j], "amin")
                hi[j].scatter_reduce_(0, node, xs[j], "amax")
            rng = hi.to(torch.float64) - lo.to(torch.float64)
            rng = torch.where(lo == hi, torch.zeros_like(rng), rng)
            best = torch.argmax(rng, dim=0)  # first maximum: the lowest coordinate on ties
            assert torch.equal(ldims[split], best[split]), f"level {l}: not the widest coordinate"


def check_sampled_nodes(spec, pts_h, sid_h, perm, vals, dims, offs, L, levels, seed):
    """The oracle's split of one random node per entry of `levels`, from the
    points the tree put in that node: key coordinate, split value (bits) and
    left count. A node smaller than the whole set is passed to the oracle as
    its points alone, with their subsets (by index mod r, by contiguous index
    range, or explicit) given as explicit ids: the same grouping, the same ids
    for the combine's order on ties."""
    rng = np.random.default_rng(seed)
    n = spec.n
    for level in levels:
        h = (1 << level) - 1 + int(rng.integers(0, 1 << level))
        b, e, _ = treecheck.node_range(offs, L, h)
        idx = np.sort(perm[b:e].astype(np.int64))
        if e - b == n:
            P, S, I, mode = pts_h, sid_h, idx, spec.subset_mode
        else:
            # the node's points alone; their subsets as explicit ids
            P = np.ascontiguousarray(pts_h[:, idx])
            if spec.subset_mode == 2:
                S = np.ascontiguousarray(sid_h[idx])
            else:
                s = idx % spec.r if spec.subset_mode == 0 else (idx * spec.r) // n
                S = s.astype(np.uint8 if spec.r <= 256 else np.uint16)
            I, mode = np.arange(e - b, dtype=np.int64), 2
        dim, _, val, left = oracle.split_cell(P, I, level, r=spec.r, subset_mode=mode, sid=S,
                                              key_rule=spec.key_rule)
        lb, le, _ = treecheck.node_range(offs, L, 2 * h + 1)  # its left child (a leaf below level L - 1)
        assert dim == int(dims[h]), f"node {h} (level {level}): dim {dims[h]}, oracle {dim}"
        assert np.float32(val).view(np.uint32) == vals[h].view(np.uint32), \
            f"node {h} (level {level}): split {vals[h]!r}, oracle {val!r}"
        assert left == le - lb, f"node {h} (level {level}): left count {le - lb}, oracle {left}"


def fourier_node_tolerance(a: float, b: float) -> float:
    """Bound on |GPU root - oracle root| for one node: the GPU sums float32
    basis terms (|error| about 1e-7 per term, 5e-6 per point with the thread
    sums), which moves F by at most about W * 6e-5 while F rises by about
    2W / (b - a) per unit of m, i.e. 3e-5 (b - a); with margin 1e-4 (b - a),
    plus the float rounding of the split."""
    return 1e-4 * (b - a) + 1e-6


def check_fourier_nodes(pts_h, perm, vals, dims, offs, L, J, heaps):
    """For each node of `heaps`: the oracle's root of Eq. (kd:eq:b) from the
    points the GPU put in the node and the bounds its ancestors' splits give
    it, against the GPU's split, within fourier_node_tolerance."""
    d = pts_h.shape[0]
    worst = 0.0
    for h in heaps:
        b0, e0, level = treecheck.node_range(offs, L, h)
        if e0 == b0:
            assert int(dims[h]) == -1 and np.isposinf(vals[h]), f"node {h}: empty node without the sentinel"
            continue
        t = level % d
        assert int(dims[h]) == t, f"node {h}: dim {dims[h]}, want {t}"
        a, b = oracle.fourier_cell_bounds(vals, h, d)
        x = pts_h[t, np.asarray(perm[b0:e0], dtype=np.int64)].astype(np.float64)
        assert np.all(x > a) and np.all(x <= b), f"node {h}: points outside its bounds"
        m = oracle.fourier_split(x, a, b, J)
        err = abs(float(vals[h]) - m)
        worst = max(worst, err / (b - a))
        assert err <= fourier_node_tolerance(a, b), f"node {h} (level {level}): split {vals[h]!r}, oracle {m!r}"
    return worst
