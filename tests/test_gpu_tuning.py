"""GPU: the tuning of the select paths changes only speed. Under every choice
of every kdt_tuning field (and all four shapes of the CTA radix select) the
build is bit-identical to the default tuning's, which is checked against the
oracle; the autotuner returns and installs one of the choices."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import assert_same_tree, gpu_build, require_gpu
from paper_2201_08288_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()
    from paper_2201_08288_gb300 import kdt
    kdt.set_tuning(None)
    yield
    kdt.set_tuning(None)


def _cases():
    """Segments of every select path: config 3's recipe (r = 256 explicit,
    widest; root segments of 4096 keys), a cyclic r = 8 tree whose root
    segments hold 2^17 keys, and a clustered one: uniform on [1, 2), where
    every key shares its sign and exponent and the CTA select's first digit
    leaves 2^15 keys in each of four bins."""
    s3 = workloads.config3(n=1 << 20, depth=13)
    pts1 = np.random.default_rng(21).standard_normal((3, 1 << 20)).astype(np.float32)
    pts2 = (1.0 + np.random.default_rng(22).random((3, 1 << 18))).astype(np.float32)
    return [("c3", s3.points(), s3.sids(), dict(r=256, subset_mode=2, depth=13, key_rule=1)),
            ("r8", pts1, None, dict(r=8, subset_mode=0, depth=12, key_rule=0)),
            ("u12", pts2, None, dict(r=2, subset_mode=0, depth=6, key_rule=0))]


def _tunings():
    from paper_2201_08288_gb300 import kdt
    d = kdt.tuning_default()
    out = []
    for f, choices in kdt.TUNING_CHOICES.items():
        for v in choices:
            if v != d[f]:
                t = dict(d)
                t[f] = v
                out.append(t)
    for th in (256, 512):  # the four shapes of the CTA select, on segments above 1024 keys
        for bits in (8, 11):
            out.append(dict(d, warp_max=1024, cta_threads=th, digit_bits=bits))
    return out


def test_every_tuning_gives_the_default_bits():
    from paper_2201_08288_gb300 import kdt
    for name, pts, sid, kw in _cases():
        kdt.set_tuning(None)
        ref = gpu_build(pts, sid=sid, **kw)
        assert_same_tree(ref, oracle.build_tree(pts, sid=sid, **kw), f"{name} default vs oracle")
        for t in _tunings():
            kdt.set_tuning(t)
            assert_same_tree(gpu_build(pts, sid=sid, **kw), ref, f"{name} {t}")
    kdt.set_tuning(None)


def test_autotune_installs_one_of_the_choices():
    from paper_2201_08288_gb300 import kdt
    dev = torch.device("cuda:0")
    specs = workloads.config4_batch(num_trees=12, n_lo=10.0, n_hi=16.0)
    items, host = [], []
    for s in specs:
        pts = s.points()
        kw = dict(r=s.r, subset_mode=0, depth=0, leaf_size=32, max_levels=s.max_levels, key_rule=0)
        items.append(dict(points=torch.from_numpy(pts).to(dev), **kw))
        host.append((pts, kw))
    best, ms = kdt.autotune(items, repeats=1)
    assert ms > 0
    assert kdt.get_tuning() == best
    for f, choices in kdt.TUNING_CHOICES.items():
        assert best[f] in choices
    trees, stats = kdt.kdt_build_batched(items)
    torch.cuda.synchronize()
    assert stats == [0] * len(items)
    for i in (0, 5, 11):
        pts, kw = host[i]
        t = trees[i]
        g = oracle.Tree(t.perm.cpu().numpy().view(np.uint32), t.split_vals.cpu().numpy(),
                        t.split_dims.cpu().numpy(), t.node_offsets.cpu().numpy(), t.levels)
        assert_same_tree(g, oracle.build_tree(pts, **kw), f"tree {i} after autotune")
    kdt.set_tuning(None)
