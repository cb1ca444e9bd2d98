"""The sharded protocol run by CPU processes, one per shard (torch.distributed
with gloo), on numpy arrays: the host-side model of kdt_build_sharded.

Shard g holds the points whose subset s has s % G == g (App. C.2: the data
stays in its subsets; Sec. 3.2: their statistics combine exactly). Every
level, for every cell of the level (the same list on every rank):
  1. key coordinate: cyclic, or the widest range (double max - double min,
     lowest coordinate on ties) from the per-coordinate min / max of the
     cell's points, all-gathered and reduced over the ranks;
  2. every rank takes the lower median (rank (w-1)/2 in key order) and the
     size w of each of its (cell, subset) groups;
  3. all-gather of those (key, subset, w) triples; every rank forms the
     same split: sort by (key, subset), the first whose running size reaches
     half the cell (2c >= W);
  4. local stable partition, keys <= split to the left.
Empty cells (depth mode) carry the sentinel (-1, +inf). At the end the ranks'
leaves are gathered and each leaf is listed in increasing original index.
"""
from __future__ import annotations

import numpy as np


def order_keys(x: np.ndarray) -> np.ndarray:
    """Order-preserving map of float32 values to uint64 (-0 < +0)."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return np.where(b >> 31 == 1, b ^ 0xFFFFFFFF, b | 0x80000000)


def key_value(k: int) -> np.float32:
    b = (k ^ 0x80000000) if k >> 31 else (~k & 0xFFFFFFFF)
    return np.array([b], dtype=np.uint32).view(np.float32)[0]


def run_rank(dist, rank: int, world: int, pts: np.ndarray, sid: np.ndarray, depth: int, key_rule: int):
    """pts float32 [d, n] and sid [n] of the WHOLE input (each rank keeps only
    its own points). Returns (perm, split_vals, split_dims, node_offsets) on
    every rank."""
    d, n = pts.shape
    mine = np.nonzero(sid % world == rank)[0]          # original indices, ascending
    cells = {0: mine}                                  # heap -> this rank's points (original indices)
    vals = np.full((1 << depth) - 1, np.inf, np.float32)
    dims = np.full((1 << depth) - 1, -1, np.int8)
    keys = [order_keys(pts[j]) for j in range(d)]
    for level in range(depth):
        heaps = range((1 << level) - 1, (1 << (level + 1)) - 1)
        # 1. key coordinate of every cell
        if key_rule == 0:
            tdim = {h: level % d for h in heaps}
        else:
            local = {}
            for h in heaps:
                idx = cells[h]
                local[h] = [(int(keys[j][idx].min()), int(keys[j][idx].max())) if idx.size else None for j in range(d)]
            gathered = [None] * world
            dist.all_gather_object(gathered, local)
            tdim = {}
            for h in heaps:
                best, best_range = 0, -1.0
                for j in range(d):
                    mm = [g[h][j] for g in gathered if g[h][j] is not None]
                    if not mm:
                        continue
                    lo, hi = min(m[0] for m in mm), max(m[1] for m in mm)
                    rng = 0.0 if lo == hi else float(key_value(hi)) - float(key_value(lo))
                    if rng > best_range:
                        best, best_range = j, rng
                tdim[h] = best
        # 2. this rank's (cell, subset) lower medians and sizes
        local = {}
        for h in heaps:
            idx = cells[h]
            k = keys[tdim[h]][idx]
            s = sid[idx]
            triples = []
            for sub in np.unique(s):
                ks = np.sort(k[s == sub])
                triples.append((int(ks[(ks.size - 1) // 2]), int(sub), int(ks.size)))
            local[h] = triples
        gathered = [None] * world
        dist.all_gather_object(gathered, local)
        # 3. the same split on every rank; 4. local partition
        nxt = {}
        for h in heaps:
            triples = sorted(t for g in gathered for t in g[h])
            W = sum(t[2] for t in triples)
            if W == 0:
                nxt[2 * h + 1] = nxt[2 * h + 2] = cells[h]
                continue
            c = 0
            for key, _, w in triples:
                c += w
                if 2 * c >= W:
                    break
            vals[h], dims[h] = key_value(key), tdim[h]
            idx = cells[h]
            left = keys[tdim[h]][idx] <= key
            nxt[2 * h + 1], nxt[2 * h + 2] = idx[left], idx[~left]
        cells = nxt
    leaves = range((1 << depth) - 1, (1 << (depth + 1)) - 1)
    gathered = [None] * world
    dist.all_gather_object(gathered, {h: cells[h] for h in leaves})
    perm, offs = [], [0]
    for h in leaves:
        merged = np.sort(np.concatenate([g[h] for g in gathered]))
        perm.append(merged)
        offs.append(offs[-1] + merged.size)
    return np.concatenate(perm).astype(np.uint32), vals, dims, np.array(offs, np.int64)
