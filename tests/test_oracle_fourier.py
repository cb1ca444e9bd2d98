"""Pins of the oracle's Fourier-moment estimator (Sec. 3.1 Lemma 1, Sec. 3.2
Eq. (kd:eq:b)) against what the mathematics fixes: the partial sums of
Lemma 1 converge to the indicator off its edges, the whole interval is
exact, the statistics add over any partition into subsets, the root of
Eq. (kd:eq:b) balances the counts on its two sides as J grows, mirroring
the data mirrors the root, and for large J the tree agrees with the
exact-median tree."""
from __future__ import annotations

import numpy as np
import pytest

import oracle


def partial_sum(x: float, a: float, b: float, J: int) -> float:
    return sum(oracle.fourier_c(j, x) * oracle.fourier_g(j, a, b) for j in range(2 * J + 1))


@pytest.mark.parametrize("a,b", [(0.0, 0.6), (0.3, 1.0), (0.2, 0.7), (0.05, 0.12)])
def test_lemma1_partial_sums_converge_to_the_indicator(a, b):
    """1_J(x, a, b) -> 1(a < x < b) uniformly away from a and b (Lemma 2 (A))."""
    xs = [x for x in np.linspace(0.01, 0.99, 50) if min(abs(x - a), abs(x - b)) >= 0.03]
    for J, tol in ((300, 0.05), (2000, 0.01)):
        for x in xs:
            want = 1.0 if a < x < b else 0.0
            assert abs(partial_sum(x, a, b, J) - want) < tol, (x, J)


def test_whole_interval_is_exact():
    """g_0(0, 1) = 1 and g_j(0, 1) = 0 for j >= 1: every partial sum is 1."""
    assert oracle.fourier_g(0, 0.0, 1.0) == 1.0
    for j in range(1, 41):
        assert oracle.fourier_g(j, 0.0, 1.0) == 0.0
    for x in (0.001, 0.3, 0.999):
        assert partial_sum(x, 0.0, 1.0, 20) == 1.0


def test_g0_takes_half_per_inner_edge():
    assert oracle.fourier_g(0, 0.3, 0.6) == 0.0
    assert oracle.fourier_g(0, 0.0, 0.6) == 0.5
    assert oracle.fourier_g(0, 0.3, 1.0) == 0.5


def test_basis_terms():
    """c_0 = 1, c_{2j-1} = cos((2j-1)x), c_{2j} = sin((2j-1)x)."""
    x = 0.37
    assert oracle.fourier_c(0, x) == 1.0
    for j in range(1, 9):
        assert oracle.fourier_c(2 * j - 1, x) == pytest.approx(np.cos((2 * j - 1) * x), abs=1e-15)
        assert oracle.fourier_c(2 * j, x) == pytest.approx(np.sin((2 * j - 1) * x), abs=1e-15)


def test_statistics_add_over_any_partition_into_subsets():
    """C_j(X) = sum_r C_j(X_r) (Sec. 3.2): the subsets' moments add up."""
    rng = np.random.default_rng(3)
    x = rng.random(5000)
    sid = rng.integers(0, 7, size=x.size)
    whole = oracle.fourier_moments(x, 16)
    parts = sum(oracle.fourier_moments(x[sid == s], 16) for s in range(7))
    np.testing.assert_allclose(parts, whole, rtol=1e-12, atol=1e-9)
    assert whole[0] == x.size


@pytest.mark.parametrize("dist", ["uniform", "beta"])
def test_root_balances_the_counts(dist):
    """As J grows the root of Eq. (kd:eq:b) splits the points in halves."""
    rng = np.random.default_rng(11)
    n = 40001
    x = rng.random(n) if dist == "uniform" else rng.beta(2.0, 5.0, size=n)
    for J, frac in ((64, 0.02), (2000, 0.004)):
        m = oracle.fourier_split(x, 0.0, 1.0, J)
        assert abs(np.count_nonzero(x <= m) - n / 2) <= frac * n, (J, m)
    # inside a cell: only its points, bounds from its ancestors
    a, b = 0.2, 0.7
    y = x[(x > a) & (x < b)]
    m = oracle.fourier_split(y, a, b, 2000)
    assert a < m < b
    assert abs(np.count_nonzero(y <= m) - y.size / 2) <= 0.004 * y.size


def test_mirroring_the_data_mirrors_the_root():
    rng = np.random.default_rng(5)
    x = rng.beta(2.0, 3.0, size=3001)
    for (a, b) in ((0.0, 1.0), (0.1, 0.8)):
        y = x[(x > a) & (x < b)]
        m = oracle.fourier_split(y, a, b, 24)
        mm = oracle.fourier_split(1.0 - y, 1.0 - b, 1.0 - a, 24)
        assert mm == pytest.approx(1.0 - m, abs=1e-9)


def test_large_J_tree_agrees_with_the_exact_median_tree():
    """For large J each split sits within a few order statistics of the
    exact lower median of its cell (same cyclic keys), so the leaves hold
    nearly equal counts, and every split lies inside its cell's bounds."""
    rng = np.random.default_rng(8)
    n, d, depth = 8192, 2, 4
    pts = ((rng.integers(0, 1 << 24, size=(d, n)) + 0.5) / (1 << 24)).astype(np.float32)
    f = oracle.fourier_build_tree(pts, depth=depth, J=1500)
    e = oracle.build_tree(pts, r=1, depth=depth)
    np.testing.assert_array_equal(f.split_dims, e.split_dims)
    counts = np.diff(f.node_offsets)
    assert np.all(np.abs(counts - n / (1 << depth)) <= 0.02 * n / (1 << depth) + 2), counts
    for h in range((1 << depth) - 1):
        a, b = oracle.fourier_cell_bounds(f.split_vals, h, d)
        assert a <= f.split_vals[h] <= b
        assert abs(float(f.split_vals[h]) - float(e.split_vals[h])) <= 0.02 * (b - a), h
    # the partition follows the splits: coordinate <= split goes left, stable
    check_partition(pts, f)


def check_partition(pts, t):
    import treecheck
    L = t.levels
    for h in range((1 << L) - 1):
        lb, le, _ = treecheck.node_range(t.node_offsets, L, 2 * h + 1)
        rb, re, _ = treecheck.node_range(t.node_offsets, L, 2 * h + 2)
        dim = int(t.split_dims[h])
        assert np.all(pts[dim, t.perm[lb:le]] <= t.split_vals[h])
        assert np.all(pts[dim, t.perm[rb:re]] > t.split_vals[h])
    for k in range(1 << L):
        assert np.all(np.diff(t.perm[t.node_offsets[k]:t.node_offsets[k + 1]].astype(np.int64)) > 0)


def test_empty_cells_get_the_sentinel():
    pts = np.array([[0.2, 0.7, 0.4]], np.float32)
    t = oracle.fourier_build_tree(pts, depth=4, J=8)
    assert np.all(np.diff(t.node_offsets) >= 0) and t.node_offsets[-1] == 3
    empty = [h for h in range(15) if t.split_dims[h] == -1]
    assert empty and all(np.isposinf(t.split_vals[h]) for h in empty)
    check_partition_nonempty(pts, t)


def check_partition_nonempty(pts, t):
    assert sorted(t.perm.tolist()) == [0, 1, 2]


@pytest.mark.parametrize("bad,status", [(0.0, 1), (1.0, 1), (-0.5, 1), (np.nan, 2)])
def test_coordinates_outside_the_open_unit_interval_are_refused(bad, status):
    pts = np.full((2, 10), 0.5, np.float32)
    pts[1, 3] = bad
    with pytest.raises(oracle.OracleError) as e:
        oracle.fourier_build_tree(pts, depth=2, J=4)
    assert e.value.status == status
