"""Helpers for the GPU parity tests: run the CUDA build through the C ABI and
compare its outputs with the CPU oracle element by element."""
from __future__ import annotations

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_08288_gb300 import build
    build.build()


def gpu_build(points: np.ndarray, *, sid=None, **kw):
    from paper_2201_08288_gb300 import kdt
    dev = torch.device("cuda:0")
    pts = torch.from_numpy(np.ascontiguousarray(points, dtype=np.float32)).to(dev)
    sid_t = None
    if sid is not None:
        sid = np.ascontiguousarray(sid)
        sid_t = torch.from_numpy(sid.view(np.int16) if sid.dtype == np.uint16 else sid).to(dev)
    t = kdt.kdt_build(pts, sid=sid_t, **kw)
    torch.cuda.synchronize()
    return oracle.Tree(t.perm.cpu().numpy().view(np.uint32).copy(), t.split_vals.cpu().numpy().copy(),
                       t.split_dims.cpu().numpy().copy(), t.node_offsets.cpu().numpy().copy(), t.levels)


def assert_same_tree(g, ref, what=""):
    assert g.levels == ref.levels, f"{what}: levels {g.levels} vs {ref.levels}"
    np.testing.assert_array_equal(g.node_offsets, ref.node_offsets, err_msg=f"{what}: node_offsets")
    np.testing.assert_array_equal(g.split_dims, ref.split_dims, err_msg=f"{what}: split_dims")
    np.testing.assert_array_equal(g.split_vals.view(np.uint32), ref.split_vals.view(np.uint32),
                                  err_msg=f"{what}: split_vals (bit patterns)")
    np.testing.assert_array_equal(g.perm, ref.perm, err_msg=f"{what}: perm")


def check_against_oracle(points, *, sid=None, **kw):
    g = gpu_build(points, sid=sid, **kw)
    ref = oracle.build_tree(points, sid=sid, **kw)
    assert_same_tree(g, ref, str(kw))
    return g
