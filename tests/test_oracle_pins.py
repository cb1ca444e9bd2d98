"""Pins for the CPU oracle: each test fixes part of it against something other
than itself (hand-derived trees, a second implementation, textbook routines,
closed forms, invariants, probability facts). CPU only."""
from __future__ import annotations

import itertools
import math
import struct

import numpy as np
import pytest

import brute
import golden_io
import oracle
from treecheck import check_invariants, le_total, node_range, quartile_bound_ok


def _tree_tuple(t):
    return t.perm, t.split_vals, t.split_dims, t.node_offsets, t.levels


# ----------------------------------------------------------------- key order


SPECIAL = [0.0, -0.0, 1.0, -1.0, 1e-45, -1e-45, 1.1754942e-38, -1.1754942e-38, 1.17549435e-38,
           3.4028235e38, -3.4028235e38, math.inf, -math.inf, 0.5, -0.5, 2.0, 1e-10, -1e-10,
           123.456, -123.456, 1.0000001, 0.99999994]


def test_key_order_matches_float_order_with_signed_zero():
    """The uint32 key orders floats like `<`, with -0.0 below +0.0 (reading R4)."""
    vals = [np.float32(v).item() for v in SPECIAL]
    rng = np.random.default_rng(0)
    vals += [float(v) for v in (rng.standard_normal(200) * 10.0 ** rng.integers(-30, 30, 200)).astype(np.float32)]
    for a in vals:
        for b in vals[:40]:
            ka, kb = oracle.key(a), oracle.key(b)
            assert (ka < kb) == (brute.order_key(a) < brute.order_key(b)), (a, b)
            assert (ka == kb) == (brute.order_key(a) == brute.order_key(b)), (a, b)


def test_key_round_trip_is_bit_exact():
    for v in SPECIAL + [float(x) for x in np.random.default_rng(1).standard_normal(100).astype(np.float32)]:
        f = np.float32(v)
        back = np.float32(oracle.key_value(oracle.key(float(f))))
        assert struct.pack("<f", back) == struct.pack("<f", f)


# ------------------------------------------------------------ golden trees


@pytest.mark.parametrize("case", golden_io.all_cases(), ids=lambda c: c["name"])
def test_golden_hand_derived(case):
    t = oracle.build_tree(case["points"], r=case["r"], subset_mode=case["subset_mode"],
                          sid=case.get("sid"), depth=case["depth"], leaf_size=case["leaf_size"],
                          max_levels=case["max_levels"], key_rule=case["key_rule"])
    assert t.levels == case["levels"]
    np.testing.assert_array_equal(t.perm, case["perm"])
    np.testing.assert_array_equal(t.split_dims, case["split_dims"])
    np.testing.assert_array_equal(t.node_offsets, case["offsets"])
    assert t.split_vals.view(np.uint32).tolist() == case["split_vals"].view(np.uint32).tolist()


# ------------------------------------------------- P1: brute force, all sids


def _compare_with_brute(pts, **kw):
    t = oracle.build_tree(pts, **kw)
    bp, bv, bd, bo, bL = brute.build(pts.tolist(), **kw)
    assert t.levels == bL
    assert t.perm.tolist() == bp
    assert t.node_offsets.tolist() == bo
    assert t.split_dims.tolist() == bd
    assert t.split_vals.view(np.uint32).tolist() == np.array(bv, np.float32).view(np.uint32).tolist()


@pytest.mark.parametrize("n,r,d", [(6, 3, 1), (7, 3, 2), (8, 2, 2), (10, 2, 1)])
def test_brute_force_every_subset_assignment(n, r, d):
    """P1: every assignment of n points to r explicit subsets, both key rules,
    depth 3 and leaf mode, on small-integer data with many ties."""
    rng = np.random.default_rng(n * 100 + r * 10 + d)
    pts = rng.integers(-2, 3, size=(d, n)).astype(np.float32)
    pts[0, 0] = -0.0
    for a_i, assign in enumerate(itertools.product(range(r), repeat=n)):
        if a_i % 3 and n * r > 20:  # every third assignment for the larger spaces
            continue
        sid = np.array(assign, np.uint8)
        for key_rule in (0, 1):
            _compare_with_brute(pts, r=r, subset_mode=2, sid=sid, depth=3, key_rule=key_rule)
        if a_i % 7 == 0:
            _compare_with_brute(pts, r=r, subset_mode=2, sid=sid, depth=0, leaf_size=1,
                                max_levels=12, key_rule=a_i % 2)


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_random_cases(seed):
    """P1: random sizes, modes, rules, depths and leaf sizes against the second implementation."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(0, 120))
    d = int(rng.integers(1, 5))
    r = int(rng.integers(1, 12))
    mode = int(rng.integers(0, 3))
    key_rule = int(rng.integers(0, 2))
    if seed % 3 == 0:
        pts = rng.integers(-3, 4, size=(d, n)).astype(np.float32)  # heavy ties
    else:
        pts = rng.standard_normal((d, n)).astype(np.float32)
    sid = rng.integers(0, r, n).astype(np.uint8) if mode == 2 else None
    if seed % 2:
        _compare_with_brute(pts, r=r, subset_mode=mode, sid=sid, depth=int(rng.integers(1, 7)),
                            key_rule=key_rule)
    else:
        _compare_with_brute(pts, r=r, subset_mode=mode, sid=sid, depth=0,
                            leaf_size=int(rng.integers(1, 9)), max_levels=24, key_rule=key_rule)


# ------------------------------------------- P2/P3: textbook exact medians


def _assert_every_split_is_exact_lower_median(pts, t):
    L = t.levels
    for h in range((1 << L) - 1):
        dim = int(t.split_dims[h])
        b, e, _ = node_range(t.node_offsets, L, h)
        if dim < 0:
            assert b == e
            continue
        col = pts[dim, t.perm[b:e].astype(np.int64)]
        k = (col.size - 1) // 2
        expect = np.partition(col, k)[k]
        assert np.float32(t.split_vals[h]) == expect, h


@pytest.mark.parametrize("key_rule", [0, 1])
def test_r1_split_is_exact_lower_median(key_rule):
    """P2: with one subset the split is the cell's lower median (numpy.partition)."""
    pts = np.random.default_rng(5).standard_normal((3, 3000)).astype(np.float32)
    t = oracle.build_tree(pts, r=1, depth=8, key_rule=key_rule)
    _assert_every_split_is_exact_lower_median(pts, t)


def test_singleton_subsets_give_exact_lower_median():
    """P3: each point its own subset (explicit id = index, r = n) gives the exact
    lower median, which exercises the combine's half-weight boundary."""
    n = 4099
    pts = np.random.default_rng(6).random((2, n), dtype=np.float32)
    sid = np.arange(n, dtype=np.uint16)
    t = oracle.build_tree(pts, r=n, subset_mode=2, sid=sid, depth=7)
    _assert_every_split_is_exact_lower_median(pts, t)
    t1 = oracle.build_tree(pts, r=1, depth=7)
    np.testing.assert_array_equal(t.perm, t1.perm)


def test_exact_tree_is_perfectly_balanced():
    """P4: the r=1 tree on 65536 points with distinct coordinates (config 1's
    shape; each coordinate a random permutation of k / 2^16, exact in float32)
    to depth 10 has 64 points in every leaf, and every left child holds
    ceil(n_c/2) points."""
    n = 65536
    rng = np.random.default_rng(0)
    pts = np.stack([rng.permutation(n) for _ in range(3)]).astype(np.float32) / np.float32(n)
    assert all(np.unique(pts[j]).size == n for j in range(3))
    t = oracle.build_tree(pts, r=1, depth=10)
    assert np.all(np.diff(t.node_offsets) == 64)
    for h in range((1 << 10) - 1):
        b, e, _ = node_range(t.node_offsets, 10, h)
        lb, le, _ = node_range(t.node_offsets, 10, 2 * h + 1)
        assert le - lb == (e - b + 1) // 2


# ----------------------------------------------- P5/P7: bounds, invariants


@pytest.mark.parametrize("seed", range(12))
def test_invariants_and_quartile_bound(seed):
    """P7 invariants and the P5 quartile guarantee of the combine rule on every node."""
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(1, 6000))
    d = int(rng.integers(1, 9))
    r = int(rng.choice([1, 2, 7, 64, 256]))
    mode = seed % 3
    key_rule = seed % 2
    if seed % 4 == 0:
        pts = np.round(rng.standard_t(3, size=(d, n)) * 4).astype(np.float32) / 4
    else:
        pts = rng.standard_normal((d, n)).astype(np.float32)
    sid = rng.integers(0, r, n).astype(np.uint16 if r > 256 else np.uint8) if mode == 2 else None
    if seed % 2:
        t = oracle.build_tree(pts, r=r, subset_mode=mode, sid=sid, depth=int(rng.integers(1, 11)),
                              key_rule=key_rule)
    else:
        t = oracle.build_tree(pts, r=r, subset_mode=mode, sid=sid, depth=0,
                              leaf_size=int(rng.integers(1, 40)), max_levels=26, key_rule=key_rule)
    check_invariants(pts, *_tree_tuple(t))
    assert quartile_bound_ok(pts, *_tree_tuple(t))


def test_leaf_mode_terminates_at_leaf_size():
    pts = np.random.default_rng(9).random((3, 5000), dtype=np.float32)
    t = oracle.build_tree(pts, r=8, depth=0, leaf_size=32, max_levels=24)
    sizes = np.diff(t.node_offsets)
    assert sizes.max() <= 32
    # a cell only splits when it holds more than leaf_size points
    for h in range((1 << t.levels) - 1):
        b, e, _ = node_range(t.node_offsets, t.levels, h)
        assert (t.split_dims[h] >= 0) == (e - b > 32)


# ------------------------------------------------------ P8: metamorphic


def test_scaling_by_power_of_two_scales_splits_only():
    """M1: multiplying every coordinate by 2^k keeps the tree; split values scale exactly."""
    pts = np.random.default_rng(10).standard_normal((3, 3000)).astype(np.float32)
    for k in (-3, 5):
        for key_rule in (0, 1):
            a = oracle.build_tree(pts, r=16, depth=7, key_rule=key_rule)
            b = oracle.build_tree(pts * np.float32(2.0 ** k), r=16, depth=7, key_rule=key_rule)
            np.testing.assert_array_equal(a.perm, b.perm)
            np.testing.assert_array_equal(a.split_dims, b.split_dims)
            np.testing.assert_array_equal(a.node_offsets, b.node_offsets)
            np.testing.assert_array_equal(a.split_vals * np.float32(2.0 ** k), b.split_vals)


def test_shuffle_with_explicit_ids_keeps_splits_and_leaf_sets():
    """M2: permuting the points together with their subset ids keeps every split
    and maps every leaf to the same set of points."""
    rng = np.random.default_rng(11)
    n, r = 4000, 32
    pts = rng.standard_normal((4, n)).astype(np.float32)
    sid = (np.arange(n) % r).astype(np.uint8)
    a = oracle.build_tree(pts, r=r, subset_mode=2, sid=sid, depth=6, key_rule=1)
    p = rng.permutation(n)
    b = oracle.build_tree(pts[:, p], r=r, subset_mode=2, sid=sid[p], depth=6, key_rule=1)
    np.testing.assert_array_equal(a.split_vals, b.split_vals)
    np.testing.assert_array_equal(a.split_dims, b.split_dims)
    np.testing.assert_array_equal(a.node_offsets, b.node_offsets)
    for k in range(1 << 6):
        sa = set(a.perm[a.node_offsets[k]:a.node_offsets[k + 1]].tolist())
        sb = set(p[b.perm[b.node_offsets[k]:b.node_offsets[k + 1]]].tolist())
        assert sa == sb


def test_unused_subset_ids_change_nothing():
    """M3: declaring more subsets than are used changes nothing."""
    rng = np.random.default_rng(12)
    pts = rng.random((3, 2000), dtype=np.float32)
    sid = rng.integers(0, 10, 2000).astype(np.uint8)
    a = oracle.build_tree(pts, r=10, subset_mode=2, sid=sid, depth=6)
    b = oracle.build_tree(pts, r=200, subset_mode=2, sid=sid, depth=6)
    for x, y in zip(_tree_tuple(a), _tree_tuple(b)):
        np.testing.assert_array_equal(x, y)


def test_contiguous_and_mod_are_explicit_special_cases():
    rng = np.random.default_rng(13)
    n, r = 3001, 7
    pts = rng.random((2, n), dtype=np.float32)
    for mode, ids in ((0, np.arange(n) % r), (1, (np.arange(n) * r) // n)):
        a = oracle.build_tree(pts, r=r, subset_mode=mode, depth=6)
        b = oracle.build_tree(pts, r=r, subset_mode=2, sid=ids.astype(np.uint8), depth=6)
        for x, y in zip(_tree_tuple(a), _tree_tuple(b)):
            np.testing.assert_array_equal(x, y)


# ------------------------------------------------ P6: rank-error statistics


def test_rank_error_distribution_matches_order_statistics_model():
    """P6: the root's left-count error (n_l - n/2) over many seeds matches a
    model built only from uniform order statistics: the subset medians are the
    h-th smallest of w uniforms (Beta(h, w-h+1)), the split is the (r/2)-th
    smallest median, and each subset contributes a binomial count of its
    points between its median and the split. Discriminates the lower from the
    upper median of medians (mean error of opposite sign) and from the exact
    median (error 0). The paper's guarantee (Sec. 4) is the asymptotic
    statement |n_l - n/2| < eps |X|; here the relative error is ~47/8192."""
    n, r, seeds = 1 << 14, 16, 1000
    w = n // r
    errs = np.empty(seeds)
    for s in range(seeds):
        x = np.random.default_rng(s).random((1, n), dtype=np.float32)
        t = oracle.build_tree(x, r=r, depth=1)
        errs[s] = t.node_offsets[1] - n / 2
    rng = np.random.default_rng(7)
    M = 40000
    h = (w - 1) // 2 + 1
    med = rng.beta(h, w - h + 1, size=(M, r))
    m = np.sort(med, axis=1)[:, r // 2 - 1:r // 2]
    above, below = med > m, med < m
    up = rng.binomial(w - h, np.clip(np.where(below, (m - med) / (1 - med), 0), 0, 1))
    dn = rng.binomial(h - 1, np.clip(np.where(above, (med - m) / med, 0), 0, 1))
    model = up.sum(1) - dn.sum(1) - above.sum(1)
    se = errs.std(ddof=1) / math.sqrt(seeds)
    assert abs(errs.mean() - model.mean()) < 4 * se + 0.5, (errs.mean(), model.mean())
    assert 0.9 < errs.std(ddof=1) / model.std() < 1.1, (errs.std(ddof=1), model.std())
    assert model.mean() < -15  # the lower median of medians sits below n/2


# ------------------------------------------------------------ error paths


def test_nan_is_rejected():
    pts = np.zeros((2, 10), np.float32)
    pts[1, 7] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.build_tree(pts, depth=2)
    assert e.value.status == 2


@pytest.mark.parametrize("kw", [dict(r=0, depth=2), dict(r=1, depth=31), dict(r=1, depth=0, leaf_size=0),
                                dict(r=4, subset_mode=2, sid=np.full(10, 4, np.uint8), depth=2),
                                dict(r=1, depth=2, key_rule=5)])
def test_invalid_arguments(kw):
    with pytest.raises(oracle.OracleError) as e:
        oracle.build_tree(np.zeros((2, 10), np.float32), **kw)
    assert e.value.status == 1


def test_level_cap():
    pts = np.random.default_rng(3).random((2, 1000), dtype=np.float32)
    with pytest.raises(oracle.OracleError) as e:
        oracle.build_tree(pts, depth=0, leaf_size=1, max_levels=5)
    assert e.value.status == 7


def test_empty_and_single_point():
    t = oracle.build_tree(np.zeros((3, 0), np.float32), depth=3)
    assert t.levels == 3 and np.all(t.split_dims == -1) and np.all(t.node_offsets == 0)
    t = oracle.build_tree(np.ones((2, 1), np.float32), depth=0, leaf_size=1)
    assert t.levels == 0 and t.node_offsets.tolist() == [0, 1]
    t = oracle.build_tree(np.ones((2, 1), np.float32), depth=2)
    assert t.split_dims.tolist() == [0, 1, -1] and t.node_offsets.tolist() == [0, 1, 1, 1, 1]


def test_split_cell_agrees_with_build():
    rng = np.random.default_rng(14)
    pts = rng.standard_normal((5, 2000)).astype(np.float32)
    sid = rng.integers(0, 50, 2000).astype(np.uint8)
    t = oracle.build_tree(pts, r=50, subset_mode=2, sid=sid, depth=5, key_rule=1)
    for h in range(31):
        b, e, level = node_range(t.node_offsets, 5, h)
        idx = rng.permutation(t.perm[b:e].astype(np.int64))
        dim, k, v, left = oracle.split_cell(pts, idx, level, r=50, subset_mode=2, sid=sid, key_rule=1)
        assert dim == t.split_dims[h]
        assert np.float32(v).view(np.uint32) == t.split_vals[h].view(np.uint32)
        lb, le, _ = node_range(t.node_offsets, 5, 2 * h + 1)
        assert left == le - lb
        assert np.all(le_total(pts[dim, t.perm[lb:le].astype(np.int64)], v))


# ------------------------------------- the unweighted rule (R2u, NEXT-4)


def test_unweighted_rule_hand_example():
    """One subset of seven points (median 4) and two singletons (10, 11): the
    count-weighted rule splits at 4 (7 of 9 points reach half), the
    unweighted one at the middle of the medians 4, 10, 11, i.e. 10."""
    pts = np.array([[1, 2, 3, 4, 5, 6, 7, 10, 11]], np.float32)
    sid = np.array([0] * 7 + [1, 2], np.uint8)
    w = oracle.build_tree(pts, r=3, subset_mode=2, sid=sid, depth=1)
    u = oracle.build_tree(pts, r=3, subset_mode=2, sid=sid, depth=1, combine_rule=oracle.COMBINE_UNWEIGHTED)
    assert float(w.split_vals[0]) == 4.0 and w.node_offsets.tolist() == [0, 4, 9]
    assert float(u.split_vals[0]) == 10.0 and u.node_offsets.tolist() == [0, 8, 9]
    # an even number of medians takes the lower one: 4 and 10 -> 4
    u2 = oracle.build_tree(pts[:, :8], r=2, subset_mode=2, sid=sid[:8], depth=1,
                           combine_rule=oracle.COMBINE_UNWEIGHTED)
    assert float(u2.split_vals[0]) == 4.0


@pytest.mark.parametrize("seed", range(24))
def test_unweighted_rule_against_brute_force(seed):
    rng = np.random.default_rng(5000 + seed)
    n = int(rng.integers(0, 100))
    d = int(rng.integers(1, 4))
    r = int(rng.integers(1, 10))
    pts = (rng.integers(-3, 4, size=(d, n)).astype(np.float32) if seed % 2
           else rng.standard_normal((d, n)).astype(np.float32))
    sid = rng.integers(0, r, n).astype(np.uint8)
    kw = dict(r=r, subset_mode=2, sid=sid, key_rule=seed % 2, combine_rule=oracle.COMBINE_UNWEIGHTED)
    if seed % 3:
        _compare_with_brute(pts, depth=int(rng.integers(1, 6)), **kw)
    else:
        _compare_with_brute(pts, depth=0, leaf_size=int(rng.integers(1, 6)), max_levels=24, **kw)


def test_unweighted_rule_equals_weighted_for_one_subset_and_for_singletons():
    """With one subset, or with every point its own subset, every subset has
    the same size in every cell, and both rules take the lower median."""
    rng = np.random.default_rng(9)
    pts = rng.standard_normal((3, 3000)).astype(np.float32)
    for kw in (dict(r=1, depth=8), dict(r=3000, subset_mode=2,
                                          sid=np.arange(3000).astype(np.uint16), depth=8)):
        a = oracle.build_tree(pts, **kw)
        b = oracle.build_tree(pts, combine_rule=oracle.COMBINE_UNWEIGHTED, **kw)
        assert np.array_equal(a.perm, b.perm) and np.array_equal(a.split_vals.view(np.uint32),
                                                                  b.split_vals.view(np.uint32))
