"""GPU parity: the CUDA build (through the C ABI) against the CPU oracle,
element by element and bit for bit, on seeded inputs that span both the
multi-CTA pipeline and the in-shared-memory subtree kernel, ragged tiles, and
the degenerate cases of the method."""
from __future__ import annotations

import numpy as np
import pytest

import golden_io
import oracle
from gpu_util import assert_same_tree, check_against_oracle, gpu_build, require_gpu
from paper_2201_08288_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("case", golden_io.all_cases(), ids=lambda c: c["name"])
def test_golden(case):
    g = gpu_build(case["points"], sid=case.get("sid"), r=case["r"], subset_mode=case["subset_mode"],
                  depth=case["depth"], leaf_size=case["leaf_size"], max_levels=case["max_levels"],
                  key_rule=case["key_rule"])
    assert g.levels == case["levels"]
    np.testing.assert_array_equal(g.perm, case["perm"])
    np.testing.assert_array_equal(g.split_dims, case["split_dims"])
    np.testing.assert_array_equal(g.node_offsets, case["offsets"])
    np.testing.assert_array_equal(g.split_vals.view(np.uint32), case["split_vals"].view(np.uint32))


def test_config1_plain_and_exact():
    """n=65536, d=3 uniform, r=8 by index mod 8, cyclic, depth 10; plus the r=1 exact tree."""
    spec = workloads.config1()
    pts = spec.points()
    check_against_oracle(pts, r=8, subset_mode=0, depth=10)
    check_against_oracle(pts, r=1, subset_mode=0, depth=10)


def test_config2_shape_reduced():
    """Config 2's recipe (16-Gaussian mixture, r=64 contiguous, cyclic) at n=2^20, depth 13."""
    spec = workloads.config2(n=1 << 20, depth=13)
    check_against_oracle(spec.points(), r=64, subset_mode=1, depth=13)


def test_config3_shape_reduced():
    """Config 3's recipe (Student-t with a 1/256 grid, r=256 explicit, widest) at n=2^19, depth 12."""
    spec = workloads.config3(n=1 << 19, depth=12)
    check_against_oracle(spec.points(), sid=spec.sids(), r=256, subset_mode=2, depth=12, key_rule=1)


@pytest.mark.parametrize("seed", range(60))
def test_random_small_cases(seed):
    """Random sizes (empty to several tiles, ragged), d in 1..16, r in 1..300,
    all subset modes, both key rules, depth and leaf modes, ties injected."""
    rng = np.random.default_rng(5000 + seed)
    n = int(rng.choice([0, 1, 2, 3, 31, 33, 1000, 4099, 9000, 30011, 70001]))
    d = int(rng.integers(1, 17))
    r = int(rng.integers(1, 301))
    mode = int(rng.integers(0, 3))
    key_rule = int(rng.integers(0, 2))
    kind = seed % 4
    if kind == 0:
        pts = rng.integers(-4, 5, size=(d, n)).astype(np.float32)
    elif kind == 1:
        pts = rng.standard_normal((d, n)).astype(np.float32)
        pts[:, rng.random(n) < 0.2] = 0.0
    elif kind == 2:
        pts = rng.standard_t(2, size=(d, n)).astype(np.float32)
    else:
        pts = rng.random((d, n), dtype=np.float32)
    if n and seed % 5 == 0:
        pts[0, rng.integers(0, n, size=max(1, n // 10))] = -0.0
    sid = None
    if mode == 2:
        sid = rng.integers(0, r, n).astype(np.uint8 if r <= 256 else np.uint16)
    if seed % 2:
        check_against_oracle(pts, sid=sid, r=r, subset_mode=mode, depth=int(rng.integers(1, 16)),
                             key_rule=key_rule)
    else:
        check_against_oracle(pts, sid=sid, r=r, subset_mode=mode, depth=0,
                             leaf_size=int(rng.integers(1, 70)), max_levels=26, key_rule=key_rule)


@pytest.mark.parametrize("d", [1, 2, 8, 16, 64])
def test_dims_around_subtree_capacity(d):
    """Cells just above and below the subtree kernel's capacity for this d."""
    from paper_2201_08288_gb300 import kdt
    cap = kdt.kdt_subtree_capacity(d)
    rng = np.random.default_rng(d)
    for n in (cap - 1, cap, cap + 1, 2 * cap + 3):
        pts = rng.standard_normal((d, n)).astype(np.float32)
        check_against_oracle(pts, r=5, subset_mode=0, depth=6, key_rule=d % 2)


def test_big_steps_with_many_cells():
    """d = 16 and cells of about 48 points more than the subtree capacity at
    level 10: more than a thousand big cells in one step, where the combine
    and the tile scan run a warp per cell."""
    from paper_2201_08288_gb300 import kdt
    d = 16
    n = 1024 * (kdt.kdt_subtree_capacity(d) + 48)
    pts = np.random.default_rng(11).standard_normal((d, n)).astype(np.float32)
    check_against_oracle(pts, r=8, subset_mode=0, depth=11, key_rule=1)


@pytest.mark.parametrize("d", [1, 3, 16])
def test_subtree_levels_with_many_live_cells(d):
    """One cell of the subtree kernel's full capacity split down to single
    points: its deep levels hold more live cells than the kernel's
    shared-memory cell table, so their cells are kept in global memory."""
    from paper_2201_08288_gb300 import kdt
    cap = kdt.kdt_subtree_capacity(d)
    assert cap >= 1024
    rng = np.random.default_rng(40 + d)
    pts = rng.standard_normal((d, cap)).astype(np.float32)
    check_against_oracle(pts, r=3, subset_mode=0, depth=0, leaf_size=1, max_levels=26, key_rule=1)
    check_against_oracle(pts, r=3, subset_mode=0, depth=12, key_rule=0)


def test_all_equal_points_depth_and_leaf():
    pts = np.ones((3, 20000), np.float32)
    check_against_oracle(pts, r=4, depth=5)
    check_against_oracle(pts, r=4, depth=0, leaf_size=8, max_levels=10)
    check_against_oracle(pts, r=4, depth=0, leaf_size=8, max_levels=10, key_rule=1)


def test_two_valued_and_infinities():
    rng = np.random.default_rng(3)
    pts = rng.choice(np.array([-np.inf, -1.0, 0.0, -0.0, 1.0, np.inf], np.float32), size=(4, 50000))
    check_against_oracle(pts, r=16, depth=8)
    check_against_oracle(pts, r=16, depth=8, key_rule=1)


def test_singleton_subsets_exact_median():
    """Explicit id = index (r = n = 4096): the exact lower median at every node."""
    n = 4096
    pts = np.random.default_rng(4).random((2, n), dtype=np.float32)
    sid = np.arange(n, dtype=np.uint16)
    g = check_against_oracle(pts, sid=sid, r=n, subset_mode=2, depth=9)
    ref1 = oracle.build_tree(pts, r=1, depth=9)
    np.testing.assert_array_equal(g.perm, ref1.perm)


@pytest.mark.parametrize("mode", [0, 2])
def test_small_roots_with_more_subsets_than_the_root_sort_counts(mode):
    """Roots within the subtree capacity whose r exceeds the subset counts the
    subtree kernel keeps for a root (2048): the pipeline puts them in subset
    order and splits them first."""
    from paper_2201_08288_gb300 import kdt
    rng = np.random.default_rng(70 + mode)
    n = kdt.kdt_subtree_capacity(3) - 100
    pts = rng.standard_normal((3, n)).astype(np.float32)
    sid = rng.integers(0, 3000, n).astype(np.uint16) if mode == 2 else None
    check_against_oracle(pts, sid=sid, r=3000, subset_mode=mode, depth=7)
    check_against_oracle(pts, sid=sid, r=3000, subset_mode=mode, depth=0, leaf_size=5, max_levels=20, key_rule=1)


def test_max_subsets_large_cells():
    n = 300000
    rng = np.random.default_rng(7)
    pts = rng.random((3, n), dtype=np.float32)
    sid = rng.integers(0, 4096, n).astype(np.uint16)
    check_against_oracle(pts, sid=sid, r=4096, subset_mode=2, depth=7)


def test_leaf_mode_config4_like_trees():
    specs = workloads.config4_batch(num_trees=24, n_lo=8.0, n_hi=16.0)
    for s in specs:
        pts = s.points()
        check_against_oracle(pts, r=s.r, subset_mode=0, depth=0, leaf_size=32, max_levels=s.max_levels)


# ------------------------------------------------------------- error paths

def test_nan_input_is_reported():
    from paper_2201_08288_gb300 import kdt
    for n in (100, 50000):
        pts = np.random.default_rng(1).random((3, n), dtype=np.float32)
        pts[2, n // 2] = np.nan
        with pytest.raises(kdt.KdtError) as e:
            gpu_build(pts, r=4, depth=4)
        assert e.value.status == 2


# Every place the input is checked for NaN: the presort of a root in subset
# order (by its per-column min / max keys under widest spread, value by value
# otherwise), and the first pipeline pass of a root that is not presorted
# (contiguous subsets). Quiet and signalling patterns of both signs, in a
# coordinate that is not the first key.
@pytest.mark.parametrize("mode,key_rule", [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1)])
@pytest.mark.parametrize("bits", [0x7FC00000, 0xFFC00000, 0x7F800001, 0xFF800001])
def test_nan_input_is_reported_on_every_root_path(mode, key_rule, bits):
    from paper_2201_08288_gb300 import kdt
    n, d, r = 60000, 4, 16
    rng = np.random.default_rng(7)
    pts = rng.random((d, n), dtype=np.float32)
    pts.view(np.uint32)[2, 12345] = np.uint32(bits)
    sid = rng.integers(0, r, n).astype(np.uint8) if mode == 2 else None
    with pytest.raises(kdt.KdtError) as e:
        gpu_build(pts, sid=sid, r=r, subset_mode=mode, depth=6, key_rule=key_rule)
    assert e.value.status == 2


def test_level_cap_is_reported():
    from paper_2201_08288_gb300 import kdt
    pts = np.random.default_rng(2).random((2, 5000), dtype=np.float32)
    with pytest.raises(kdt.KdtError) as e:
        gpu_build(pts, r=2, depth=0, leaf_size=1, max_levels=6)
    assert e.value.status == 7


@pytest.mark.parametrize("kw", [dict(r=0, depth=3), dict(r=4097, depth=3), dict(r=2, depth=31),
                                dict(r=2, depth=0, leaf_size=0)])
def test_invalid_arguments(kw):
    from paper_2201_08288_gb300 import kdt
    with pytest.raises(kdt.KdtError) as e:
        gpu_build(np.zeros((2, 10), np.float32), **kw)
    assert e.value.status == 1


def test_host_buffer_entry_point_matches_device_entry_point():
    from paper_2201_08288_gb300 import kdt
    spec = workloads.config3(n=200000, depth=11)
    pts, sid = spec.points(), spec.sids()
    h = kdt.kdt_build_host(pts, sid=sid, r=256, subset_mode=2, depth=11, key_rule=1)
    ref = oracle.build_tree(pts, sid=sid, r=256, subset_mode=2, depth=11, key_rule=1)
    assert_same_tree(oracle.Tree(h.perm, h.split_vals, h.split_dims, h.node_offsets, h.levels), ref)
