"""CPU checks of the C ABI: the library builds, loads without a GPU and exports
every function include/kdt.h declares; the binding's struct matches the
header's field order; host-side validation needs no device."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(kdt_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_08288_gb300 import build, kdt
    build.build()
    return kdt.load_library()


def test_every_declared_symbol_is_exported(lib):
    from paper_2201_08288_gb300 import kdt
    declared = _declared_functions()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(kdt.EXPORTED) <= set(declared) | set(getattr(kdt, "EXPORTED_EXTRA", []))


def test_params_struct_layout_matches_header():
    from paper_2201_08288_gb300 import kdt
    src = open(os.path.join(ROOT, "include", "kdt.h")).read()
    body = re.search(r"typedef struct kdt_params \{(.*?)\} kdt_params;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\*?\s*([a-z0-9_]+)\s*;", body)
    assert fields == [f[0] for f in kdt.kdt_params._fields_]
    assert ctypes.sizeof(kdt.kdt_params) == 64


def test_status_strings_and_capacity_need_no_gpu(lib):
    from paper_2201_08288_gb300 import kdt
    assert kdt.kdt_status_str(0) == "ok"
    assert "NaN" in kdt.kdt_status_str(2)
    caps = [kdt.kdt_subtree_capacity(d) for d in (1, 3, 8, 16, 64)]
    assert all(c > 0 and c % 32 == 0 for c in caps) and caps == sorted(caps, reverse=True)
    assert kdt.kdt_subtree_capacity(0) == 0


@pytest.mark.parametrize("kw", [dict(r=0), dict(r=4097), dict(depth=31), dict(depth=0, leaf_size=0),
                                dict(key_rule=3), dict(fourier_j=33), dict(fourier_j=-1),
                                dict(fourier_j=4, key_rule=1), dict(fourier_j=4, depth=0, leaf_size=8)])
def test_invalid_params_rejected_on_host(lib, kw):
    from paper_2201_08288_gb300 import kdt
    args = dict(r=2, depth=3)
    args.update(kw)
    p = kdt.make_params(100, 3, **args)
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_workspace_size(p)
    assert e.value.status == 1


def test_tuning_struct_layout_matches_header():
    from paper_2201_08288_gb300 import kdt
    src = open(os.path.join(ROOT, "include", "kdt.h")).read()
    body = re.search(r"typedef struct kdt_tuning \{(.*?)\} kdt_tuning;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\s([a-z0-9_]+)(?:\[\d+\])?\s*;", body)
    assert fields == [f[0] for f in kdt.kdt_tuning._fields_]
    assert ctypes.sizeof(kdt.kdt_tuning) == 32


def test_tuning_set_get_and_validation_need_no_gpu(lib):
    """The tuning is host state: defaults, a round trip through every choice of
    every field, and rejection of anything else (the tuning in force kept)."""
    from paper_2201_08288_gb300 import kdt
    d = kdt.tuning_default()
    assert d == {"tiny_max": 64, "bitonic_max": 256, "warp_max": 4096, "cta_threads": 256, "digit_bits": 11}
    kdt.set_tuning(None)
    assert kdt.get_tuning() == d
    try:
        for f, choices in kdt.TUNING_CHOICES.items():
            for v in choices:
                t = dict(d)
                t[f] = v
                kdt.set_tuning(t)
                assert kdt.get_tuning() == t
        kept = kdt.get_tuning()
        for f, bad in [("tiny_max", 0), ("tiny_max", 128), ("bitonic_max", 32), ("warp_max", 8192),
                       ("cta_threads", 128), ("digit_bits", 4)]:
            t = dict(d)
            t[f] = bad
            with pytest.raises(kdt.KdtError) as e:
                kdt.set_tuning(t)
            assert e.value.status == 1
            assert kdt.get_tuning() == kept
        raw = kdt.kdt_tuning(**d)
        raw.reserved[1] = 7
        assert lib.kdt_set_tuning(ctypes.byref(raw)) == 1
        assert lib.kdt_get_tuning(None) == 1
    finally:
        kdt.set_tuning(None)


def test_estimator_workspace_ignores_the_subsets(lib):
    """With fourier_j > 0 the build runs with one subset and no ids (the
    estimator's statistics are sums), so r and the ids do not change the
    workspace it needs; the median rule's workspace does depend on r."""
    from paper_2201_08288_gb300 import kdt
    base = kdt.kdt_workspace_size(kdt.make_params(100000, 3, depth=8, fourier_j=8))
    for kw in (dict(r=64), dict(r=300, subset_mode=1), dict(r=16, subset_mode=2, sid_ptr=4096, sid_bytes=1)):
        assert kdt.kdt_workspace_size(kdt.make_params(100000, 3, depth=8, fourier_j=8, **kw)) == base
    assert kdt.kdt_workspace_size(kdt.make_params(100000, 3, depth=8, r=64)) > base



def test_batched_builds_refuse_the_estimator(lib):
    """The trees of a batched (or served) build share one select path, so the
    estimator is a plain-build option; the refusal happens on the host."""
    from paper_2201_08288_gb300 import kdt
    descs = (kdt.kdt_tree_desc * 2)()
    for i, j in enumerate((0, 6)):
        descs[i].params = kdt.make_params(5000, 3, depth=6, fourier_j=j)
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_workspace_size_batched(descs)
    assert e.value.status == 1
    descs[1].params = kdt.make_params(5000, 3, depth=6)
    assert kdt.kdt_workspace_size_batched(descs) > 0


def test_fault_injection_is_host_state(lib):
    """kdt_fault_inject validates its arguments on the host; kdt_fault_clear
    turns every kind off (nothing here touches a device)."""
    from paper_2201_08288_gb300 import kdt
    for kind in (kdt.KDT_FAULT_ALLOC, kdt.KDT_FAULT_SERVER_STEP, kdt.KDT_FAULT_SERVER_RESET, kdt.KDT_FAULT_WAIT):
        assert lib.kdt_fault_inject(kind, 0) == 0
    assert lib.kdt_fault_inject(0, 1) == 1
    assert lib.kdt_fault_inject(99, 1) == 1
    assert lib.kdt_fault_inject(kdt.KDT_FAULT_ALLOC, -1) == 1
    kdt.fault_inject(kdt.KDT_FAULT_ALLOC, 3)
    kdt.fault_clear()
    assert kdt.kdt_status_str(kdt.KDT_ERR_CANCELLED) == "request cancelled"


def test_server_info_struct_layout_matches_header():
    from paper_2201_08288_gb300 import kdt
    src = open(os.path.join(ROOT, "include", "kdt.h")).read()
    body = re.search(r"typedef struct kdt_server_info \{(.*?)\} kdt_server_info;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            fields += [f.strip() for f in decl.split(None, 1)[1].split(",")]
    assert fields == [f[0] for f in kdt.kdt_server_info._fields_]


def test_sharded_build_refuses_leaf_mode_and_bad_shard_counts_on_the_host(lib):
    """kdt_build_sharded validates before it touches a device: leaf mode, the
    estimator and shard counts outside 1..16 are invalid arguments."""
    from paper_2201_08288_gb300 import kdt
    i32 = ctypes.c_int32(0)
    fake = ctypes.c_void_p(4096)  # never dereferenced: the call returns first
    for kw, shards in ((dict(depth=0, leaf_size=8), 2), (dict(depth=4, fourier_j=4), 2), (dict(depth=4), 0),
                       (dict(depth=4), 17)):
        p = kdt.make_params(1000, 3, r=4, **kw)
        assert lib.kdt_build_sharded(fake, ctypes.byref(p), shards, fake, fake, fake, fake, ctypes.byref(i32),
                                     None) == 1
