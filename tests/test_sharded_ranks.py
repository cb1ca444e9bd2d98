"""The sharded protocol on the host: one process per shard (gloo on
127.0.0.1, world sizes 2 and 3), each holding only the points of its
subsets, exchanging per level only the (cell, subset) medians and sizes and
the per-coordinate min / max, gives the oracle's tree bit for bit."""
from __future__ import annotations

import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, case, out):
    sys.path[:0] = [ROOT, HERE]
    import torch.distributed as dist
    import shard_ranks
    pts, sid, depth, key_rule = case
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = shard_ranks.run_rank(dist, rank, world, pts, sid, depth, key_rule)
    finally:
        dist.destroy_process_group()


def _cases():
    from paper_2201_08288_gb300 import workloads
    rng = np.random.default_rng(7)
    a = workloads.uniform(3000, 3, seed=61)
    b = workloads.student_t_snapped(2500, 4, 3.0, 0.1, 256, seed=62)
    return {
        "mod_cyclic": (a, (np.arange(3000) % 8).astype(np.int64), 6, 0),
        "explicit_widest": (b, rng.integers(0, 16, 2500), 6, 1),
        "few_subsets": (b[:, :700], rng.integers(0, 2, 700), 5, 1),
    }


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", ["mod_cyclic", "explicit_widest", "few_subsets"])
def test_ranks_reproduce_the_oracle_tree(world, name):
    import torch.multiprocessing as mp
    import oracle
    pts, sid, depth, key_rule = _cases()[name]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), (pts, sid, depth, key_rule), out), nprocs=world,
                       start_method="spawn")
    sid8 = sid.astype(np.uint8)
    ref = oracle.build_tree(pts, r=int(sid.max()) + 1, subset_mode=2, sid=sid8, depth=depth, key_rule=key_rule)
    for rank in range(world):
        perm, vals, dims, offs = out[rank]
        np.testing.assert_array_equal(perm, ref.perm)
        np.testing.assert_array_equal(vals.view(np.uint32), ref.split_vals.view(np.uint32))
        np.testing.assert_array_equal(dims, ref.split_dims)
        np.testing.assert_array_equal(offs, ref.node_offsets)
