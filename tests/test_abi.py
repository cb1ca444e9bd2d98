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
    assert ctypes.sizeof(kdt.kdt_params) == 56


def test_status_strings_and_capacity_need_no_gpu(lib):
    from paper_2201_08288_gb300 import kdt
    assert kdt.kdt_status_str(0) == "ok"
    assert "NaN" in kdt.kdt_status_str(2)
    caps = [kdt.kdt_subtree_capacity(d) for d in (1, 3, 8, 16, 64)]
    assert all(c > 0 and c % 32 == 0 for c in caps) and caps == sorted(caps, reverse=True)
    assert kdt.kdt_subtree_capacity(0) == 0


@pytest.mark.parametrize("kw", [dict(r=0), dict(r=4097), dict(depth=31), dict(depth=0, leaf_size=0),
                                dict(key_rule=3)])
def test_invalid_params_rejected_on_host(lib, kw):
    from paper_2201_08288_gb300 import kdt
    args = dict(r=2, depth=3)
    args.update(kw)
    p = kdt.make_params(100, 3, **args)
    with pytest.raises(kdt.KdtError) as e:
        kdt.kdt_workspace_size(p)
    assert e.value.status == 1
