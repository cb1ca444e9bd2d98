"""Thin Python binding of the C ABI in include/kdt.h (ctypes).

Only argument marshalling happens here: torch allocates device memory and
provides the stream; every step of the build runs in the CUDA library
(`_build/libkdt.so`). Importing works without a GPU; calling a build without
the compiled library raises immediately (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libkdt.so")

KDT_KEY_CYCLIC = 0
KDT_KEY_WIDEST_SPREAD = 1
KDT_SUBSET_MOD = 0
KDT_SUBSET_CONTIGUOUS = 1
KDT_SUBSET_EXPLICIT = 2
KDT_COMBINE_WEIGHTED = 0
KDT_COMBINE_UNWEIGHTED = 1
KDT_MAX_LEVELS = 30
KDT_MAX_SUBSETS = 4096

STATUS_NAMES = {0: "KDT_OK", 1: "KDT_ERR_INVALID_ARG", 2: "KDT_ERR_NAN_INPUT", 3: "KDT_ERR_OOM",
                4: "KDT_ERR_CUDA", 5: "KDT_ERR_CAPACITY", 6: "KDT_ERR_TIMEOUT", 7: "KDT_ERR_LEVEL_CAP",
                8: "KDT_ERR_BUSY", 9: "KDT_ERR_NOT_FOUND", 10: "KDT_ERR_CANCELLED"}
KDT_ERR_CANCELLED = 10

# fault kinds of kdt_fault_inject
KDT_FAULT_ALLOC = 1
KDT_FAULT_SERVER_STEP = 2
KDT_FAULT_SERVER_RESET = 3
KDT_FAULT_WAIT = 4

# Every symbol include/kdt.h declares (checked by the CPU test suite).
EXPORTED = ["kdt_workspace_size", "kdt_build", "kdt_workspace_size_host", "kdt_build_host",
            "kdt_subtree_capacity", "kdt_status_str", "kdt_trace_enable", "kdt_launch_count",
            "kdt_trace_read", "kdt_build_noalloc", "kdt_workspace_size_batched", "kdt_build_batched",
            "kdt_server_create", "kdt_server_submit", "kdt_server_poll", "kdt_server_stats",
            "kdt_server_destroy", "kdt_server_cancel", "kdt_tuning_default", "kdt_set_tuning", "kdt_get_tuning",
            "kdt_autotune", "kdt_fault_inject", "kdt_fault_clear", "kdt_build_sharded", "kdt_query_box",
            "kdt_query_knn"]
KDT_KNN_MAX_K = 32


class KdtError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")
        self.status = status


class kdt_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("units", ctypes.c_uint64)]


class kdt_params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("d", ctypes.c_int32),
        ("subset_mode", ctypes.c_int32),
        ("r", ctypes.c_int32),
        ("key_rule", ctypes.c_int32),
        ("subset_id8", ctypes.c_void_p),
        ("subset_id16", ctypes.c_void_p),
        ("depth", ctypes.c_int32),
        ("leaf_size", ctypes.c_int32),
        ("max_levels", ctypes.c_int32),
        ("fourier_j", ctypes.c_int32),
        ("combine_rule", ctypes.c_int32),
    ]


class kdt_tree_desc(ctypes.Structure):
    _fields_ = [
        ("points", ctypes.c_void_p),
        ("params", kdt_params),
        ("out_perm", ctypes.c_void_p),
        ("out_split_vals", ctypes.c_void_p),
        ("out_split_dims", ctypes.c_void_p),
        ("out_node_offsets", ctypes.c_void_p),
    ]


class kdt_server_info(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("ticks", ctypes.c_uint64), ("in_flight", ctypes.c_int32), ("peak_in_flight", ctypes.c_int32),
                ("arena_bytes", ctypes.c_uint64), ("arena_bytes_in_use", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("engine_failures", ctypes.c_uint64)]


class kdt_tuning(ctypes.Structure):
    _fields_ = [("tiny_max", ctypes.c_int32), ("bitonic_max", ctypes.c_int32), ("warp_max", ctypes.c_int32),
                ("cta_threads", ctypes.c_int32), ("digit_bits", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


KDT_FOURIER_MAX_J = 32  # largest fourier_j

TUNING_FIELDS = ("tiny_max", "bitonic_max", "warp_max", "cta_threads", "digit_bits")
# the choices kdt_set_tuning accepts, per field
TUNING_CHOICES = {"tiny_max": (8, 16, 32, 64), "bitonic_max": (64, 128, 256), "warp_max": (1024, 2048, 4096),
                  "cta_threads": (256, 512), "digit_bits": (8, 11)}


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libkdt.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library missing: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER(kdt_params)
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    lib.kdt_workspace_size.argtypes = [P, ctypes.POINTER(sz)]
    lib.kdt_workspace_size.restype = ctypes.c_int
    lib.kdt_workspace_size_host.argtypes = [P, ctypes.POINTER(sz)]
    lib.kdt_workspace_size_host.restype = ctypes.c_int
    lib.kdt_build.argtypes = [vp, P, vp, sz, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int32), vp]
    lib.kdt_build.restype = ctypes.c_int
    lib.kdt_build_host.argtypes = [vp, P, vp, sz, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int32), vp]
    lib.kdt_build_host.restype = ctypes.c_int
    lib.kdt_subtree_capacity.argtypes = [ctypes.c_int32]
    lib.kdt_subtree_capacity.restype = ctypes.c_int32
    lib.kdt_status_str.argtypes = [ctypes.c_int]
    lib.kdt_status_str.restype = ctypes.c_char_p
    D = ctypes.POINTER(kdt_tree_desc)
    lib.kdt_workspace_size_batched.argtypes = [D, ctypes.c_int32, ctypes.POINTER(sz)]
    lib.kdt_workspace_size_batched.restype = ctypes.c_int
    lib.kdt_build_batched.argtypes = [D, ctypes.c_int32, vp, sz, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int), vp]
    lib.kdt_build_batched.restype = ctypes.c_int
    lib.kdt_server_create.argtypes = [sz, ctypes.c_int32, ctypes.POINTER(vp)]
    lib.kdt_server_create.restype = ctypes.c_int
    lib.kdt_server_submit.argtypes = [vp, D, ctypes.POINTER(ctypes.c_uint64)]
    lib.kdt_server_submit.restype = ctypes.c_int
    lib.kdt_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
    lib.kdt_server_poll.restype = ctypes.c_int
    lib.kdt_server_stats.argtypes = [vp, ctypes.POINTER(kdt_server_info)]
    lib.kdt_server_stats.restype = ctypes.c_int
    lib.kdt_server_destroy.argtypes = [vp]
    lib.kdt_server_destroy.restype = ctypes.c_int
    lib.kdt_server_cancel.argtypes = [vp, ctypes.c_uint64]
    lib.kdt_server_cancel.restype = ctypes.c_int
    lib.kdt_fault_inject.argtypes = [ctypes.c_int, ctypes.c_int32]
    lib.kdt_fault_inject.restype = ctypes.c_int
    lib.kdt_build_sharded.argtypes = [vp, P, ctypes.c_int32, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int32), vp]
    lib.kdt_build_sharded.restype = ctypes.c_int
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    lib.kdt_query_box.argtypes = [vp, i64, i32, vp, vp, vp, vp, i32, vp, vp, i32, vp, vp, ctypes.c_uint32, vp]
    lib.kdt_query_box.restype = ctypes.c_int
    lib.kdt_query_knn.argtypes = [vp, i64, i32, vp, vp, vp, vp, i32, vp, i32, i32, vp, vp, vp]
    lib.kdt_query_knn.restype = ctypes.c_int
    lib.kdt_fault_clear.argtypes = []
    lib.kdt_fault_clear.restype = None
    lib.kdt_build_noalloc.argtypes = [vp, P, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int32), vp]
    lib.kdt_build_noalloc.restype = ctypes.c_int
    lib.kdt_trace_enable.argtypes = [ctypes.c_int32]
    lib.kdt_trace_enable.restype = None
    lib.kdt_launch_count.argtypes = []
    lib.kdt_launch_count.restype = ctypes.c_uint64
    lib.kdt_trace_read.argtypes = [ctypes.POINTER(kdt_kernel_stat), ctypes.c_int32, ctypes.c_int32]
    lib.kdt_trace_read.restype = ctypes.c_int32
    T = ctypes.POINTER(kdt_tuning)
    lib.kdt_tuning_default.argtypes = [T]
    lib.kdt_tuning_default.restype = None
    lib.kdt_set_tuning.argtypes = [T]
    lib.kdt_set_tuning.restype = ctypes.c_int
    lib.kdt_get_tuning.argtypes = [T]
    lib.kdt_get_tuning.restype = ctypes.c_int
    lib.kdt_autotune.argtypes = [D, ctypes.c_int32, vp, sz, ctypes.c_int32, T, ctypes.POINTER(ctypes.c_float), vp]
    lib.kdt_autotune.restype = ctypes.c_int
    _lib = lib
    return lib


def make_params(n: int, d: int, *, r: int = 1, subset_mode: int = KDT_SUBSET_MOD, sid_ptr: int = 0,
                sid_bytes: int = 1, depth: int = 0, leaf_size: int = 1, max_levels: int = 20,
                key_rule: int = KDT_KEY_CYCLIC, fourier_j: int = 0,
                combine_rule: int = KDT_COMBINE_WEIGHTED) -> kdt_params:
    p = kdt_params()
    p.n, p.d, p.subset_mode, p.r, p.key_rule = n, d, subset_mode, r, key_rule
    p.subset_id8 = sid_ptr if (sid_ptr and sid_bytes == 1) else None
    p.subset_id16 = sid_ptr if (sid_ptr and sid_bytes == 2) else None
    p.depth, p.leaf_size, p.max_levels, p.fourier_j = depth, leaf_size, max_levels, fourier_j
    p.combine_rule = combine_rule
    return p


def kdt_workspace_size(p: kdt_params) -> int:
    out = ctypes.c_size_t(0)
    st = load_library().kdt_workspace_size(ctypes.byref(p), ctypes.byref(out))
    if st:
        raise KdtError(st, "kdt_workspace_size")
    return out.value


def kdt_workspace_size_host(p: kdt_params) -> int:
    out = ctypes.c_size_t(0)
    st = load_library().kdt_workspace_size_host(ctypes.byref(p), ctypes.byref(out))
    if st:
        raise KdtError(st, "kdt_workspace_size_host")
    return out.value


def kdt_subtree_capacity(d: int) -> int:
    return int(load_library().kdt_subtree_capacity(d))


def kdt_status_str(st: int) -> str:
    return load_library().kdt_status_str(st).decode()


def kdt_trace_enable(on: bool) -> None:
    load_library().kdt_trace_enable(1 if on else 0)


def kdt_launch_count() -> int:
    return int(load_library().kdt_launch_count())


def kdt_trace_read(reset: bool = True) -> dict:
    """Per-kernel {name: (launches, total_ms, points)} of the traced launches."""
    lib = load_library()
    buf = (kdt_kernel_stat * 64)()
    k = lib.kdt_trace_read(buf, 64, 1 if reset else 0)
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms), int(buf[i].units))
            for i in range(min(k, 64))}


@dataclass
class Tree:
    perm: "object"
    split_vals: "object"
    split_dims: "object"
    node_offsets: "object"
    levels: int


def _capacity(depth: int, max_levels: int) -> int:
    return depth if depth > 0 else max_levels


def _sid_info(sid):
    if sid is None:
        return 0, 1
    import torch
    if sid.dtype == torch.uint8:
        return sid.data_ptr(), 1
    if sid.dtype in (torch.int16, getattr(torch, "uint16", torch.int16)):
        return sid.data_ptr(), 2
    raise TypeError("subset ids must be uint8 or 16-bit")


def kdt_build(points, *, r: int = 1, subset_mode: int = KDT_SUBSET_MOD, sid=None, depth: int = 0,
              leaf_size: int = 1, max_levels: int = 20, key_rule: int = KDT_KEY_CYCLIC,
              workspace=None, stream=None, outputs: Optional[Tree] = None, fourier_j: int = 0,
              combine_rule: int = KDT_COMBINE_WEIGHTED) -> Tree:
    """Build on the device. points: torch float32 CUDA tensor [d, n], contiguous.
    sid: uint8 (or int16 holding uint16) CUDA tensor [n] for explicit subsets.
    workspace: optional uint8 CUDA tensor of >= kdt_workspace_size bytes.
    outputs: optional preallocated Tree of tensors (sized for the capacity).
    fourier_j > 0: splits by the paper's Fourier-moment estimator with J
    harmonics (cyclic keys, depth mode, coordinates in (0,1)).
    combine_rule: KDT_COMBINE_WEIGHTED (the default) or KDT_COMBINE_UNWEIGHTED
    (every non-empty subset's median counts once)."""
    import torch
    if not (points.is_cuda and points.dtype == torch.float32 and points.is_contiguous() and points.dim() == 2):
        raise ValueError("points must be a contiguous float32 CUDA tensor [d, n]")
    d, n = points.shape
    sid_ptr, sid_bytes = _sid_info(sid)
    p = make_params(n, d, r=r, subset_mode=subset_mode, sid_ptr=sid_ptr, sid_bytes=sid_bytes, depth=depth,
                    leaf_size=leaf_size, max_levels=max_levels, key_rule=key_rule, fourier_j=fourier_j,
                    combine_rule=combine_rule)
    lib = load_library()
    cap = _capacity(depth, max_levels)
    dev = points.device
    if outputs is None:
        outputs = Tree(torch.empty(max(n, 1), dtype=torch.int32, device=dev),
                       torch.empty(max((1 << cap) - 1, 1), dtype=torch.float32, device=dev),
                       torch.empty(max((1 << cap) - 1, 1), dtype=torch.int8, device=dev),
                       torch.empty((1 << cap) + 1, dtype=torch.int64, device=dev), 0)
    ws_ptr, ws_bytes = 0, 0
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    levels = ctypes.c_int32(0)
    with torch.cuda.device(dev):  # the library works on the current device: the one holding the points
        st = lib.kdt_build(points.data_ptr(), ctypes.byref(p), ws_ptr or None, ws_bytes,
                           outputs.perm.data_ptr(), outputs.split_vals.data_ptr(), outputs.split_dims.data_ptr(),
                           outputs.node_offsets.data_ptr(), ctypes.byref(levels), stream.cuda_stream)
    if st:
        raise KdtError(st, "kdt_build")
    L = levels.value
    m = (1 << L) - 1
    return Tree(outputs.perm[:n], outputs.split_vals[:m], outputs.split_dims[:m],
                outputs.node_offsets[:(1 << L) + 1], L)


def kdt_build_host(points: np.ndarray, *, r: int = 1, subset_mode: int = KDT_SUBSET_MOD, sid=None,
                   depth: int = 0, leaf_size: int = 1, max_levels: int = 20, key_rule: int = KDT_KEY_CYCLIC,
                   workspace=None, stream=None, outputs=None, fourier_j: int = 0,
                   combine_rule: int = KDT_COMBINE_WEIGHTED) -> Tree:
    """Build from HOST arrays (numpy, ideally pinned): copies in, builds, copies
    the outputs back into numpy arrays, all inside the library call."""
    import torch
    points = np.ascontiguousarray(points, dtype=np.float32)
    d, n = points.shape
    sid_ptr, sid_bytes = 0, 1
    if sid is not None:
        sid = np.ascontiguousarray(sid)
        sid_ptr, sid_bytes = sid.ctypes.data, sid.dtype.itemsize
    p = make_params(n, d, r=r, subset_mode=subset_mode, sid_ptr=sid_ptr, sid_bytes=sid_bytes, depth=depth,
                    leaf_size=leaf_size, max_levels=max_levels, key_rule=key_rule, fourier_j=fourier_j,
                    combine_rule=combine_rule)
    cap = _capacity(depth, max_levels)
    if outputs is None:
        outputs = Tree(np.empty(max(n, 1), np.uint32), np.empty(max((1 << cap) - 1, 1), np.float32),
                       np.empty(max((1 << cap) - 1, 1), np.int8), np.empty((1 << cap) + 1, np.int64), 0)
    ws_ptr, ws_bytes = 0, 0
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    if stream is None:
        stream = torch.cuda.current_stream()
    levels = ctypes.c_int32(0)
    st = load_library().kdt_build_host(points.ctypes.data, ctypes.byref(p), ws_ptr or None, ws_bytes,
                                       outputs.perm.ctypes.data, outputs.split_vals.ctypes.data,
                                       outputs.split_dims.ctypes.data, outputs.node_offsets.ctypes.data,
                                       ctypes.byref(levels), stream.cuda_stream)
    if st:
        raise KdtError(st, "kdt_build_host")
    L = levels.value
    m = (1 << L) - 1
    return Tree(outputs.perm[:n], outputs.split_vals[:m], outputs.split_dims[:m],
                outputs.node_offsets[:(1 << L) + 1], L)


def kdt_build_noalloc(points, *, r: int = 1, subset_mode: int = KDT_SUBSET_MOD, sid=None, depth: int = 0,
                      leaf_size: int = 1, max_levels: int = 20, key_rule: int = KDT_KEY_CYCLIC, stream=None,
                      combine_rule: int = KDT_COMBINE_WEIGHTED,
                      outputs: Tree) -> Tree:
    """kdt_build that allocates nothing: the library's fixed 64 MiB device
    scratch array is the workspace. outputs: preallocated Tree of tensors
    (sized for the capacity), as for kdt_build."""
    import torch
    if not (points.is_cuda and points.dtype == torch.float32 and points.is_contiguous() and points.dim() == 2):
        raise ValueError("points must be a contiguous float32 CUDA tensor [d, n]")
    d, n = points.shape
    sid_ptr, sid_bytes = _sid_info(sid)
    p = make_params(n, d, r=r, subset_mode=subset_mode, sid_ptr=sid_ptr, sid_bytes=sid_bytes, depth=depth,
                    leaf_size=leaf_size, max_levels=max_levels, key_rule=key_rule, combine_rule=combine_rule)
    if stream is None:
        stream = torch.cuda.current_stream(points.device)
    levels = ctypes.c_int32(0)
    with torch.cuda.device(points.device):  # the scratch array used is the current device's
        st = load_library().kdt_build_noalloc(points.data_ptr(), ctypes.byref(p), outputs.perm.data_ptr(),
                                              outputs.split_vals.data_ptr(), outputs.split_dims.data_ptr(),
                                              outputs.node_offsets.data_ptr(), ctypes.byref(levels),
                                              stream.cuda_stream)
    if st:
        raise KdtError(st, "kdt_build_noalloc")
    L = levels.value
    m = (1 << L) - 1
    return Tree(outputs.perm[:n], outputs.split_vals[:m], outputs.split_dims[:m],
                outputs.node_offsets[:(1 << L) + 1], L)


def kdt_build_sharded(points, shards: int, *, r: int = 1, subset_mode: int = KDT_SUBSET_MOD, sid=None,
                      depth: int, key_rule: int = KDT_KEY_CYCLIC, stream=None,
                      combine_rule: int = KDT_COMBINE_WEIGHTED,
                      outputs: Optional[Tree] = None) -> Tree:
    """The build emulated on `shards` logical shards (subset s on shard
    s % shards; per-level all-gather of the segment statistics), depth mode.
    Same arguments and outputs as kdt_build."""
    import torch
    if not (points.is_cuda and points.dtype == torch.float32 and points.is_contiguous() and points.dim() == 2):
        raise ValueError("points must be a contiguous float32 CUDA tensor [d, n]")
    d, n = points.shape
    sid_ptr, sid_bytes = _sid_info(sid)
    p = make_params(n, d, r=r, subset_mode=subset_mode, sid_ptr=sid_ptr, sid_bytes=sid_bytes, depth=depth,
                    key_rule=key_rule, combine_rule=combine_rule)
    dev = points.device
    if outputs is None:
        outputs = _alloc_outputs(n, depth, dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    levels = ctypes.c_int32(0)
    with torch.cuda.device(dev):
        st = load_library().kdt_build_sharded(points.data_ptr(), ctypes.byref(p), shards, outputs.perm.data_ptr(),
                                              outputs.split_vals.data_ptr(), outputs.split_dims.data_ptr(),
                                              outputs.node_offsets.data_ptr(), ctypes.byref(levels),
                                              stream.cuda_stream)
    if st:
        raise KdtError(st, "kdt_build_sharded")
    L = levels.value
    m = (1 << L) - 1
    return Tree(outputs.perm[:n], outputs.split_vals[:m], outputs.split_dims[:m],
                outputs.node_offsets[:(1 << L) + 1], L)


def _alloc_outputs(n: int, cap: int, dev):
    import torch
    return Tree(torch.empty(max(n, 1), dtype=torch.int32, device=dev),
                torch.empty(max((1 << cap) - 1, 1), dtype=torch.float32, device=dev),
                torch.empty(max((1 << cap) - 1, 1), dtype=torch.int8, device=dev),
                torch.empty((1 << cap) + 1, dtype=torch.int64, device=dev), 0)


def make_descs(items, outputs=None):
    """items: sequence of dicts with keys points (CUDA float32 [d, n]), and optionally
    sid, r, subset_mode, depth, leaf_size, max_levels, key_rule. Returns the
    ctypes descriptor array and the output Trees (allocated if not given)."""
    descs = (kdt_tree_desc * len(items))()
    outs = []
    for i, it in enumerate(items):
        pts = it["points"]
        d, n = pts.shape
        sid_ptr, sid_bytes = _sid_info(it.get("sid"))
        depth = it.get("depth", 0)
        max_levels = it.get("max_levels", 20)
        p = make_params(n, d, r=it.get("r", 1), subset_mode=it.get("subset_mode", KDT_SUBSET_MOD),
                        sid_ptr=sid_ptr, sid_bytes=sid_bytes, depth=depth, leaf_size=it.get("leaf_size", 1),
                        max_levels=max_levels, key_rule=it.get("key_rule", KDT_KEY_CYCLIC),
                        combine_rule=it.get("combine_rule", KDT_COMBINE_WEIGHTED))
        o = outputs[i] if outputs is not None else _alloc_outputs(n, _capacity(depth, max_levels), pts.device)
        outs.append(o)
        descs[i].points = pts.data_ptr()
        descs[i].params = p
        descs[i].out_perm = o.perm.data_ptr()
        descs[i].out_split_vals = o.split_vals.data_ptr()
        descs[i].out_split_dims = o.split_dims.data_ptr()
        descs[i].out_node_offsets = o.node_offsets.data_ptr()
    return descs, outs


def kdt_workspace_size_batched(descs) -> int:
    out = ctypes.c_size_t(0)
    st = load_library().kdt_workspace_size_batched(descs, len(descs), ctypes.byref(out))
    if st:
        raise KdtError(st, "kdt_workspace_size_batched")
    return out.value


def kdt_build_batched(items, *, workspace=None, stream=None, outputs=None, descs=None):
    """Build many trees together. Returns (trees, statuses): per item a Tree of
    output tensors sliced to its L (None where its status is not 0) and the
    per-tree status codes."""
    import torch
    if descs is None:
        descs, outs = make_descs(items, outputs)
    else:
        outs = outputs
    num = len(descs)
    levels = (ctypes.c_int32 * num)()
    stats = (ctypes.c_int * num)()
    ws_ptr, ws_bytes = 0, 0
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    if stream is None:
        stream = torch.cuda.current_stream()
    st = load_library().kdt_build_batched(descs, num, ws_ptr or None, ws_bytes, levels, stats, stream.cuda_stream)
    if st and not any(stats[i] for i in range(num)):
        raise KdtError(st, "kdt_build_batched")
    trees = []
    for i in range(num):
        if stats[i]:
            trees.append(None)
            continue
        L = levels[i]
        n = descs[i].params.n
        m = (1 << L) - 1
        o = outs[i]
        trees.append(Tree(o.perm[:n], o.split_vals[:m], o.split_dims[:m], o.node_offsets[:(1 << L) + 1], L))
    return trees, [int(stats[i]) for i in range(num)]


def _tuning_dict(t: kdt_tuning) -> dict:
    return {f: int(getattr(t, f)) for f in TUNING_FIELDS}


def tuning_default() -> dict:
    """The library's default tuning of the select paths (kdt_tuning_default)."""
    t = kdt_tuning()
    load_library().kdt_tuning_default(ctypes.byref(t))
    return _tuning_dict(t)


def get_tuning() -> dict:
    """The tuning in force (kdt_get_tuning)."""
    t = kdt_tuning()
    st = load_library().kdt_get_tuning(ctypes.byref(t))
    if st:
        raise KdtError(st, "kdt_get_tuning")
    return _tuning_dict(t)


def set_tuning(tuning=None) -> None:
    """Install a tuning (dict of TUNING_FIELDS; None: the defaults)."""
    lib = load_library()
    if tuning is None:
        st = lib.kdt_set_tuning(None)
    else:
        t = kdt_tuning(**{f: int(tuning[f]) for f in TUNING_FIELDS})
        st = lib.kdt_set_tuning(ctypes.byref(t))
    if st:
        raise KdtError(st, "kdt_set_tuning")


def autotune(items, *, repeats: int = 2, workspace=None, stream=None, outputs=None):
    """Time candidate tunings on these trees (items as for kdt_build_batched),
    install the fastest and return (tuning dict, ms per build)."""
    import torch
    descs, outs = make_descs(items, outputs)
    ws_ptr, ws_bytes = 0, 0
    if workspace is not None:
        ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    if stream is None:
        stream = torch.cuda.current_stream()
    best = kdt_tuning()
    ms = ctypes.c_float()
    st = load_library().kdt_autotune(descs, len(descs), ws_ptr or None, ws_bytes, repeats, ctypes.byref(best),
                                     ctypes.byref(ms), stream.cuda_stream)
    if st:
        raise KdtError(st, "kdt_autotune")
    del outs
    return _tuning_dict(best), float(ms.value)


class Server:
    """Continuous-batching build server (kdt_server_*). Requests are dicts as
    for kdt_build_batched; the caller keeps the tensors alive until poll
    returns."""

    def __init__(self, mem_budget_bytes: int, max_trees_in_flight: int = 256):
        self._lib = load_library()
        self._h = ctypes.c_void_p()
        st = self._lib.kdt_server_create(mem_budget_bytes, max_trees_in_flight, ctypes.byref(self._h))
        if st:
            raise KdtError(st, "kdt_server_create")
        self._keep = {}

    def submit(self, item, outputs=None) -> int:
        """Queue a build. The server reads the inputs on its own stream, so the
        stream that produced them is synchronised first."""
        import torch
        descs, outs = make_descs([item], [outputs] if outputs is not None else None)
        torch.cuda.current_stream(item["points"].device).synchronize()
        t = ctypes.c_uint64(0)
        st = self._lib.kdt_server_submit(self._h, descs, ctypes.byref(t))
        if st:
            raise KdtError(st, "kdt_server_submit")
        self._keep[t.value] = (item, outs[0], descs)
        return t.value

    def poll(self, ticket: int, wait_ms: int = -1):
        """(status, Tree or None, latency_ms), or None if not finished yet."""
        res, lv, lat = ctypes.c_int(0), ctypes.c_int32(0), ctypes.c_double(0)
        st = self._lib.kdt_server_poll(self._h, ticket, wait_ms, ctypes.byref(res), ctypes.byref(lv),
                                       ctypes.byref(lat))
        if st == 8:
            return None
        if st:
            raise KdtError(st, "kdt_server_poll")
        item, o, descs = self._keep.pop(ticket)
        tree = None
        if res.value == 0:
            L = lv.value
            n = descs[0].params.n
            m = (1 << L) - 1
            tree = Tree(o.perm[:n], o.split_vals[:m], o.split_dims[:m], o.node_offsets[:(1 << L) + 1], L)
        return res.value, tree, lat.value

    def cancel(self, ticket: int) -> bool:
        """Cancel a queued request (kdt_server_cancel). True if it was
        cancelled (poll then reports KDT_ERR_CANCELLED); False if it is
        already on the GPU or finished."""
        st = self._lib.kdt_server_cancel(self._h, ticket)
        if st == 8:
            return False
        if st:
            raise KdtError(st, "kdt_server_cancel")
        return True

    def stats(self) -> dict:
        info = kdt_server_info()
        st = self._lib.kdt_server_stats(self._h, ctypes.byref(info))
        if st:
            raise KdtError(st, "kdt_server_stats")
        return {k: getattr(info, k) for k, _ in kdt_server_info._fields_}

    def close(self):
        if self._h:
            self._lib.kdt_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fault_inject(kind: int, count: int) -> None:
    """Fail the next `count` events of this kind on purpose (kdt_fault_inject;
    host-side only: nothing faults the GPU)."""
    st = load_library().kdt_fault_inject(kind, count)
    if st:
        raise KdtError(st, "kdt_fault_inject")


def fault_clear() -> None:
    """Turn every injected fault off (kdt_fault_clear)."""
    load_library().kdt_fault_clear()


def _tree_args(points, tree):
    import torch
    if not (points.is_cuda and points.dtype == torch.float32 and points.is_contiguous() and points.dim() == 2):
        raise ValueError("points must be the build's contiguous float32 CUDA tensor [d, n]")
    d, n = points.shape
    return (points.data_ptr(), n, d, tree.perm.data_ptr(), tree.split_vals.data_ptr(), tree.split_dims.data_ptr(),
            tree.node_offsets.data_ptr(), tree.levels)


def kdt_query_box(points, tree: Tree, lo, hi, *, list_cap: int = 0, stream=None):
    """Points of a built tree inside each box (kdt_query_box). points: the
    build's input (CUDA float32 [d, n]); tree: its Tree; lo, hi: CUDA float32
    [d, nq]. Returns (counts int32 [nq], lists int32 [nq, list_cap] or None)."""
    import torch
    nq = lo.shape[1]
    dev = points.device
    counts = torch.empty(max(nq, 1), dtype=torch.int32, device=dev)
    lists = torch.full((max(nq, 1), list_cap), -1, dtype=torch.int32, device=dev) if list_cap else None
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    lo, hi = lo.contiguous(), hi.contiguous()  # held until the call returns
    with torch.cuda.device(dev):
        st = load_library().kdt_query_box(*_tree_args(points, tree), lo.data_ptr(),
                                          hi.data_ptr(), nq, counts.data_ptr(),
                                          lists.data_ptr() if lists is not None else None, list_cap,
                                          stream.cuda_stream)
    if st:
        raise KdtError(st, "kdt_query_box")
    return counts[:nq], (lists[:nq] if lists is not None else None)


def kdt_query_knn(points, tree: Tree, queries, k: int, *, stream=None):
    """k nearest neighbours (kdt_query_knn). queries: CUDA float32 [d, nq].
    Returns (indices int32 [nq, k], squared distances float64 [nq, k])."""
    import torch
    nq = queries.shape[1]
    dev = points.device
    idx = torch.empty((max(nq, 1), k), dtype=torch.int32, device=dev)
    d2 = torch.empty((max(nq, 1), k), dtype=torch.float64, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    queries = queries.contiguous()  # held until the call returns
    with torch.cuda.device(dev):
        st = load_library().kdt_query_knn(*_tree_args(points, tree), queries.data_ptr(), nq, k,
                                          idx.data_ptr(), d2.data_ptr(), stream.cuda_stream)
    if st:
        raise KdtError(st, "kdt_query_knn")
    return idx[:nq], d2[:nq]
