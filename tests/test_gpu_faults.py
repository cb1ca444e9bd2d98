"""GPU: failures made on purpose on the host (kdt_fault_inject; nothing
faults, traps or hangs the GPU) end the way the header says, leak nothing,
and leave the library usable:
  - an allocation failure gives KDT_ERR_OOM with the device's free memory
    unchanged, and the next build is correct;
  - a bounded wait of the subtree kernel that runs out (an mbarrier phase
    that nothing completes, no copy in flight) gives KDT_ERR_TIMEOUT, and the
    next build is correct;
  - a failed level step of the server ends the requests on the GPU with its
    status while queued and later requests are built correctly; if the engine
    cannot be cleared, queued requests end too and pollers are woken;
  - a queued request can be cancelled; one on the GPU cannot."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import assert_same_tree, check_against_oracle, require_gpu
from paper_2201_08288_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(autouse=True)
def _clear_faults():
    from paper_2201_08288_gb300 import kdt
    kdt.fault_clear()
    yield
    kdt.fault_clear()


def _host_tree(t):
    return oracle.Tree(t.perm.cpu().numpy().view(np.uint32), t.split_vals.cpu().numpy(),
                       t.split_dims.cpu().numpy(), t.node_offsets.cpu().numpy(), t.levels)


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _outputs(n, cap):
    from paper_2201_08288_gb300 import kdt
    return kdt.Tree(torch.empty(max(n, 1), dtype=torch.int32, device="cuda:0"),
                    torch.empty(max((1 << cap) - 1, 1), dtype=torch.float32, device="cuda:0"),
                    torch.empty(max((1 << cap) - 1, 1), dtype=torch.int8, device="cuda:0"),
                    torch.empty((1 << cap) + 1, dtype=torch.int64, device="cuda:0"), 0)


def test_allocation_failure_is_oom_without_a_leak():
    """Every entry point that allocates (kdt_build, kdt_build_host and
    kdt_build_batched without a workspace; the server's arena) returns
    KDT_ERR_OOM when its allocation fails, and the device's free memory is
    the same afterwards (all outputs are preallocated, every path has run
    once before, so nothing else allocates in between)."""
    import gc
    from paper_2201_08288_gb300 import kdt
    pts = workloads.uniform(50000, 3, seed=31)
    P = torch.from_numpy(pts).to("cuda:0")
    kw = dict(r=8, subset_mode=0, depth=8)
    out = _outputs(50000, 8)
    items = [dict(points=P, **kw), dict(points=P, r=4, depth=5)]
    bouts = [_outputs(50000, 8), _outputs(50000, 5)]

    def each_path():
        yield lambda: kdt.kdt_build(P, outputs=out, **kw)
        yield lambda: kdt.kdt_build_host(pts, **kw)
        yield lambda: kdt.kdt_build_batched(items, outputs=bouts)
        yield lambda: kdt.Server(256 << 20, 4).close()

    for call in each_path():  # warm: module loading and caches
        call()
    gc.collect()
    before = _free_bytes()
    for call in each_path():
        kdt.fault_inject(kdt.KDT_FAULT_ALLOC, 1)
        with pytest.raises(kdt.KdtError) as e:
            call()
        assert e.value.status == 3
        del e
    gc.collect()
    assert _free_bytes() == before
    check_against_oracle(pts, **kw)


def test_subtree_wait_that_runs_out_is_a_timeout_and_the_next_build_is_right():
    from paper_2201_08288_gb300 import kdt
    pts = workloads.student_t_snapped(70000, 8, 3.0, 0.1, 256, seed=32)
    sid = workloads.explicit_sids(70000, 64, seed=33)
    kw = dict(r=64, subset_mode=2, depth=9, key_rule=1)
    P = torch.from_numpy(pts).to("cuda:0")
    S = torch.from_numpy(sid).to("cuda:0")
    kdt.fault_inject(kdt.KDT_FAULT_WAIT, 1)
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_build(P, sid=S, **kw)
    assert e.value.status == 6
    check_against_oracle(pts, sid=sid, **kw)
    # the same in a batched build (whose later steps are recorded once into a
    # graph: both recorded subtree launches probe): the tree with cells in
    # those launches fails; a depth-1 tree that never reaches the subtree
    # kernel is built right beside it, and both are right in the next batch
    other = workloads.uniform(5000, 3, seed=34)
    items = [dict(points=P, sid=S, **kw), dict(points=torch.from_numpy(other).to("cuda:0"), r=4, depth=1)]
    kdt.fault_inject(kdt.KDT_FAULT_WAIT, 2)
    trees, st = kdt.kdt_build_batched(items)
    assert st == [6, 0]
    assert_same_tree(_host_tree(trees[1]), oracle.build_tree(other, r=4, depth=1), "beside the timeout")
    kdt.fault_clear()
    trees, st = kdt.kdt_build_batched(items)
    assert st == [0, 0]
    assert_same_tree(_host_tree(trees[0]), oracle.build_tree(pts, sid=sid, **kw), "after the timeout")


def _requests(num, seed):
    _, specs = workloads.config5_stream(num_requests=num, rate=1000.0, n_lo=12.0, n_hi=16.0, seed=seed)
    items, host = [], []
    for s in specs:
        pts = s.points()
        kw = dict(r=32, subset_mode=0, depth=0, leaf_size=64, max_levels=s.max_levels, key_rule=0)
        items.append(dict(points=torch.from_numpy(pts).to("cuda:0"), **kw))
        host.append((pts, kw))
    return items, host


def test_server_step_failure_ends_the_requests_on_the_gpu_only():
    from paper_2201_08288_gb300 import kdt
    items, host = _requests(12, 41)
    with kdt.Server(2 << 30, 4) as sv:  # 4 slots: 8 requests wait in the queue
        kdt.fault_inject(kdt.KDT_FAULT_SERVER_STEP, 1)
        tickets = [sv.submit(it) for it in items]
        res = [sv.poll(tk) for tk in tickets]
        info = sv.stats()
        later = sv.poll(sv.submit(items[0]))
    failed = [i for i, r in enumerate(res) if r[0] != 0]
    assert info["engine_failures"] == 1
    assert 1 <= len(failed) <= 4 and all(res[i][0] == 4 for i in failed)
    for i, r in enumerate(res):
        if r[0] == 0:
            assert_same_tree(_host_tree(r[1]), oracle.build_tree(host[i][0], **host[i][1]), f"request {i}")
    assert later[0] == 0
    assert_same_tree(_host_tree(later[1]), oracle.build_tree(host[0][0], **host[0][1]), "after the failure")


def test_server_unrecoverable_failure_ends_queued_requests_and_wakes_pollers():
    """Every request is queued first (two slots for ten requests), then the
    next level step fails and the engine cannot be cleared: each request ends
    (built before the failure, or with its status), no poller is left
    waiting, and a later submit is refused with the status."""
    from paper_2201_08288_gb300 import kdt
    items, host = _requests(10, 42)
    with kdt.Server(2 << 30, 2) as sv:
        tickets = [sv.submit(it) for it in items]
        kdt.fault_inject(kdt.KDT_FAULT_SERVER_STEP, 1)
        kdt.fault_inject(kdt.KDT_FAULT_SERVER_RESET, 1)
        res = [sv.poll(tk) for tk in tickets]  # would wait forever for a stranded request
        info = sv.stats()
        with pytest.raises(kdt.KdtError) as e:
            sv.submit(items[0])
        assert e.value.status == 4
    assert info["engine_failures"] == 1 and info["completed"] == len(items)
    assert all(r[0] in (0, 4) for r in res) and any(r[0] == 4 for r in res)
    for i, r in enumerate(res):
        if r[0] == 0:
            assert_same_tree(_host_tree(r[1]), oracle.build_tree(host[i][0], **host[i][1]), f"request {i}")


def test_server_cancels_queued_requests_only():
    import time
    from paper_2201_08288_gb300 import kdt
    items, host = _requests(10, 43)
    with kdt.Server(2 << 30, 1) as sv:  # one slot: the first request runs, the rest queue behind it
        tickets = [sv.submit(it) for it in items]
        t0 = time.time()
        while sv.stats()["admitted"] < 1 and time.time() - t0 < 30:
            time.sleep(0.001)
        assert not sv.cancel(tickets[0])  # on the GPU (or finished): not cancelled
        cancelled = [tk for tk in tickets[5:] if sv.cancel(tk)]
        res = {tk: sv.poll(tk) for tk in tickets}
        info = sv.stats()
        with pytest.raises(kdt.KdtError) as e:  # released by poll
            sv.cancel(tickets[0])
        assert e.value.status == 9
    assert len(cancelled) >= 1 and info["cancelled"] == len(cancelled)
    for i, tk in enumerate(tickets):
        st, t, _ = res[tk]
        if tk in cancelled:
            assert st == kdt.KDT_ERR_CANCELLED and t is None
        else:
            assert st == 0
            assert_same_tree(_host_tree(t), oracle.build_tree(host[i][0], **host[i][1]), f"request {i}")


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")  # nothing was recorded, by design
def test_calls_on_a_capturing_stream_are_refused():
    """A build or query waits on its stream, so one issued while the stream is
    being captured into a CUDA graph is refused with an invalid-argument
    status before it touches the stream: the capture stays valid and a later
    build on the same stream is right."""
    from paper_2201_08288_gb300 import kdt
    dev = torch.device("cuda:0")
    pts_np = workloads.uniform(5000, 3, seed=71)
    pts = torch.from_numpy(pts_np).to(dev)
    kw = dict(r=4, subset_mode=0, depth=6)
    ws = torch.empty(kdt.kdt_workspace_size(kdt.make_params(5000, 3, **kw)), dtype=torch.uint8, device=dev)
    outs = _outputs(5000, 6)
    tree = kdt.kdt_build(pts, workspace=ws, outputs=_outputs(5000, 6), **kw)
    lo = torch.zeros((3, 4), device=dev)
    hi = torch.ones((3, 4), device=dev)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    calls = [lambda: kdt.kdt_build(pts, workspace=ws, outputs=outs, stream=s, **kw),
             lambda: kdt.kdt_build_noalloc(pts, outputs=outs, stream=s, **kw),
             lambda: kdt.kdt_query_box(pts, tree, lo, hi, stream=s)]
    statuses = []
    with torch.cuda.graph(g, stream=s):
        for call in calls:
            try:
                call()
                statuses.append(0)
            except kdt.KdtError as e:
                statuses.append(e.status)
    assert statuses == [1, 1, 1]
    again = kdt.kdt_build(pts, workspace=ws, outputs=outs, stream=s, **kw)
    torch.cuda.synchronize()
    assert_same_tree(_host_tree(again), oracle.build_tree(pts_np, **kw), "after a refused capture")
