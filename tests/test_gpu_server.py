"""GPU: the continuous-batching server. A request's result is the same alone,
inside a mix, and under memory pressure (and equals the oracle's); requests
that arrive while others run are admitted into the running batch; requests
that can never fit are refused."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import assert_same_tree, require_gpu
from paper_2201_08288_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _host_tree(t):
    return oracle.Tree(t.perm.cpu().numpy().view(np.uint32), t.split_vals.cpu().numpy(),
                       t.split_dims.cpu().numpy(), t.node_offsets.cpu().numpy(), t.levels)


def _requests(num, seed, n_lo=10.0, n_hi=17.0):
    dev = torch.device("cuda:0")
    _, specs = workloads.config5_stream(num_requests=num, rate=1000.0, n_lo=n_lo, n_hi=n_hi, seed=seed)
    items, host = [], []
    for s in specs:
        pts = s.points()
        kw = dict(r=32, subset_mode=0, depth=0, leaf_size=64, max_levels=s.max_levels, key_rule=0)
        items.append(dict(points=torch.from_numpy(pts).to(dev), **kw))
        host.append((pts, kw))
    return items, host


def test_alone_equals_in_mix_equals_oracle():
    from paper_2201_08288_gb300 import kdt
    items, host = _requests(51, 7)
    probe = 0
    with kdt.Server(8 << 30, 64) as sv:
        t = sv.submit(items[probe])
        st, alone, _ = sv.poll(t)
        assert st == 0
        alone = _host_tree(alone)
        tickets = [sv.submit(it) for it in items]
        results = [sv.poll(tk) for tk in tickets]
        info = sv.stats()
    assert all(r[0] == 0 for r in results)
    assert info["peak_in_flight"] > 1
    assert_same_tree(_host_tree(results[probe][1]), alone, "probe in mix")
    assert_same_tree(alone, oracle.build_tree(host[probe][0], **host[probe][1]), "probe vs oracle")
    for i in (3, 17, 29, 50):
        assert_same_tree(_host_tree(results[i][1]), oracle.build_tree(host[i][0], **host[i][1]), f"req {i}")


def test_late_arrivals_join_a_running_batch():
    from paper_2201_08288_gb300 import kdt
    dev = torch.device("cuda:0")
    big = workloads.config2(n=1 << 23, depth=15)
    big_item = dict(points=big.points_device(dev), r=64, subset_mode=1, depth=15)
    small_items, host = _requests(20, 8, n_lo=10.0, n_hi=13.0)
    import time
    with kdt.Server(16 << 30, 64) as sv:
        tb = sv.submit(big_item)
        t0 = time.time()
        while sv.stats()["ticks"] < 2 and time.time() - t0 < 30:
            time.sleep(0.0005)
        ticks_at_submit = sv.stats()["ticks"]
        ts = [sv.submit(it) for it in small_items]
        small = [sv.poll(t) for t in ts]
        st_big, tree_big, lat_big = sv.poll(tb)
        info = sv.stats()
    assert st_big == 0 and all(s[0] == 0 for s in small)
    # the small requests arrived after the big build had started and were
    # admitted while it was still being built
    assert ticks_at_submit >= 2
    assert info["peak_in_flight"] >= 2
    assert max(s[2] for s in small) < lat_big
    for i in (0, 7, 19):
        assert_same_tree(_host_tree(small[i][1]), oracle.build_tree(host[i][0], **host[i][1]), f"small {i}")


def test_memory_pressure_still_completes_everything():
    from paper_2201_08288_gb300 import kdt
    items, host = _requests(30, 9, n_lo=14.0, n_hi=17.5)
    with kdt.Server(512 << 20, 64) as sv:
        tickets = [sv.submit(it) for it in items]
        results = [sv.poll(t) for t in tickets]
        info = sv.stats()
    assert all(r[0] == 0 for r in results)
    for i in range(0, 30, 6):
        assert_same_tree(_host_tree(results[i][1]), oracle.build_tree(host[i][0], **host[i][1]), f"req {i}")
    assert info["completed"] == 30


def test_request_larger_than_budget_is_refused_and_unknown_ticket():
    from paper_2201_08288_gb300 import kdt
    dev = torch.device("cuda:0")
    with kdt.Server(256 << 20, 8) as sv:
        pts = torch.zeros((8, 1 << 24), dtype=torch.float32, device=dev)
        with pytest.raises(kdt.KdtError) as e:
            sv.submit(dict(points=pts, r=4, depth=4))
        assert e.value.status == 5
        with pytest.raises(kdt.KdtError) as e:
            sv.poll(12345, 0)
        assert e.value.status == 9


def test_inputs_drawn_on_the_device_just_before_submit():
    """Requests whose points are produced by kernels on the caller's stream
    right before submit (the server reads them on its own stream)."""
    from paper_2201_08288_gb300 import kdt
    dev = torch.device("cuda:0")
    _, specs = workloads.config5_stream(num_requests=24, rate=1000.0, n_lo=11.0, n_hi=16.0, seed=11)
    with kdt.Server(8 << 30, 64) as sv:
        items = [dict(points=s.points_device(dev), r=32, subset_mode=0, depth=0, leaf_size=64,
                      max_levels=s.max_levels, key_rule=0) for s in specs]
        tickets = [sv.submit(it) for it in items]
        results = [sv.poll(t) for t in tickets]
    assert all(r[0] == 0 for r in results)
    for i in (0, 5, 11, 23):
        pts = items[i]["points"].cpu().numpy()
        kw = {k: v for k, v in items[i].items() if k != "points"}
        assert_same_tree(_host_tree(results[i][1]), oracle.build_tree(pts, **kw), f"req {i}")
