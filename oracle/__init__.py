"""CPU oracle for the subset-median k-d tree build.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The CUDA library never imports it and the two share no code.

The arithmetic lives in ``kdt_oracle.c`` (plain C, single-threaded); this
module compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kdt_oracle.c")
_SRC_FOURIER = os.path.join(_HERE, "kdt_oracle_fourier.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libkdt_oracle.so")

KEY_CYCLIC = 0
KEY_WIDEST_SPREAD = 1
SUBSET_MOD = 0
SUBSET_CONTIGUOUS = 1
SUBSET_EXPLICIT = 2
COMBINE_WEIGHTED = 0
COMBINE_UNWEIGHTED = 1

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NAN_INPUT", 3: "OOM", 7: "LEVEL_CAP"}


class OracleError(RuntimeError):
    def __init__(self, status: int):
        super().__init__(f"oracle status {status} ({STATUS.get(status, '?')})")
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("d", ctypes.c_int32),
        ("subset_mode", ctypes.c_int32),
        ("r", ctypes.c_int32),
        ("sid8", ctypes.c_void_p),
        ("sid16", ctypes.c_void_p),
        ("depth", ctypes.c_int32),
        ("leaf_size", ctypes.c_int32),
        ("max_levels", ctypes.c_int32),
        ("key_rule", ctypes.c_int32),
        ("combine", ctypes.c_int32),
    ]


def build_library(force: bool = False) -> str:
    """Compile kdt_oracle.c into a shared library (gcc, portable flags)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_FOURIER),
                                                   os.path.getmtime(os.path.join(_HERE, "kdt_oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
                           "-o", tmp, _SRC, _SRC_FOURIER, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_library())
        lib.kdto_key.restype = ctypes.c_uint32
        lib.kdto_key.argtypes = [ctypes.c_float]
        lib.kdto_key_value.restype = ctypes.c_float
        lib.kdto_key_value.argtypes = [ctypes.c_uint32]
        lib.kdto_build.restype = ctypes.c_int
        lib.kdto_build.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Params), ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_int32)]
        lib.kdto_split_cell.restype = ctypes.c_int
        lib.kdto_split_cell.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Params), ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_int64)]
        dbl = ctypes.c_double
        lib.kdto_fourier_c.restype = dbl
        lib.kdto_fourier_c.argtypes = [ctypes.c_int32, dbl]
        lib.kdto_fourier_g.restype = dbl
        lib.kdto_fourier_g.argtypes = [ctypes.c_int32, dbl, dbl]
        lib.kdto_fourier_moments.restype = ctypes.c_int
        lib.kdto_fourier_moments.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p]
        lib.kdto_fourier_split.restype = ctypes.c_int
        lib.kdto_fourier_split.argtypes = [ctypes.c_void_p, ctypes.c_int64, dbl, dbl, ctypes.c_int32,
                                           ctypes.POINTER(dbl)]
        lib.kdto_fourier_build.restype = ctypes.c_int
        lib.kdto_fourier_build.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]
        _lib = lib
    return _lib


def key(x: float) -> int:
    return int(_load().kdto_key(ctypes.c_float(x)))


def key_value(k: int) -> float:
    return float(_load().kdto_key_value(ctypes.c_uint32(k)))


@dataclass
class Tree:
    perm: np.ndarray          # uint32 [n]
    split_vals: np.ndarray    # float32 [2^L - 1]
    split_dims: np.ndarray    # int8 [2^L - 1]
    node_offsets: np.ndarray  # int64 [2^L + 1]
    levels: int


def _params(points: np.ndarray, r: int, subset_mode: int, sid, depth: int, leaf_size: int,
            max_levels: int, key_rule: int, combine_rule: int = 0):
    d, n = points.shape
    p = _Params()
    p.n, p.d, p.subset_mode, p.r = n, d, subset_mode, r
    p.sid8 = p.sid16 = None
    keep = []
    if sid is not None:
        sid = np.ascontiguousarray(sid)
        keep.append(sid)
        if sid.dtype == np.uint8:
            p.sid8 = sid.ctypes.data
        elif sid.dtype == np.uint16:
            p.sid16 = sid.ctypes.data
        else:
            raise TypeError("subset ids must be uint8 or uint16")
    p.depth, p.leaf_size, p.max_levels, p.key_rule = depth, leaf_size, max_levels, key_rule
    p.combine = combine_rule
    return p, keep


def build_tree(points: np.ndarray, *, r: int = 1, subset_mode: int = SUBSET_MOD, sid=None,
               depth: int = 0, leaf_size: int = 1, max_levels: int = 20,
               key_rule: int = KEY_CYCLIC, combine_rule: int = COMBINE_WEIGHTED) -> Tree:
    """Build with the plain CPU reference. points: float32 [d, n] (SoA)."""
    points = np.ascontiguousarray(points, dtype=np.float32)
    if points.ndim != 2:
        raise ValueError("points must be [d, n]")
    d, n = points.shape
    p, keep = _params(points, r, subset_mode, sid, depth, leaf_size, max_levels, key_rule, combine_rule)
    cap = depth if depth > 0 else max_levels
    cap = max(0, min(cap, 30))
    perm = np.zeros(max(n, 1), np.uint32)
    vals = np.zeros(max((1 << cap) - 1, 1), np.float32)
    dims = np.zeros(max((1 << cap) - 1, 1), np.int8)
    offs = np.zeros((1 << cap) + 1, np.int64)
    levels = ctypes.c_int32(0)
    st = _load().kdto_build(points.ctypes.data, ctypes.byref(p), perm.ctypes.data, vals.ctypes.data,
                            dims.ctypes.data, offs.ctypes.data, ctypes.byref(levels))
    del keep
    if st != 0:
        raise OracleError(st)
    L = levels.value
    m = (1 << L) - 1
    return Tree(perm[:n].copy(), vals[:m].copy(), dims[:m].copy(), offs[:(1 << L) + 1].copy(), L)


def split_cell(points: np.ndarray, idx: np.ndarray, level: int, *, r: int = 1,
               subset_mode: int = SUBSET_MOD, sid=None, key_rule: int = KEY_CYCLIC,
               combine_rule: int = COMBINE_WEIGHTED):
    """Split of one cell whose points have original indices ``idx``.

    Returns (dim, key, value, left_count)."""
    points = np.ascontiguousarray(points, dtype=np.float32)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    p, keep = _params(points, r, subset_mode, sid, 1, 1, 1, key_rule, combine_rule)
    dim, k, v, left = ctypes.c_int32(), ctypes.c_uint32(), ctypes.c_float(), ctypes.c_int64()
    st = _load().kdto_split_cell(points.ctypes.data, ctypes.byref(p), idx.ctypes.data,
                                 idx.size, level, ctypes.byref(dim), ctypes.byref(k),
                                 ctypes.byref(v), ctypes.byref(left))
    del keep
    if st != 0:
        raise OracleError(st)
    return dim.value, k.value, v.value, left.value


# ------------------------------------------------- the paper's estimator
# (Sec. 3.1 Lemma 1, Sec. 3.2 Eq. (kd:eq:b); readings in kdt_oracle_fourier.c)

FOURIER_MAX_J = 4096


def fourier_c(j: int, x: float) -> float:
    """Basis term c_j(x) of Lemma 1."""
    return float(_load().kdto_fourier_c(j, x))


def fourier_g(j: int, a: float, b: float) -> float:
    """Coefficient g_j(a, b) of Lemma 1."""
    return float(_load().kdto_fourier_g(j, a, b))


def fourier_moments(x: np.ndarray, J: int) -> np.ndarray:
    """C_j = sum_i c_j(x_i), j = 0..2J (float64)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(2 * J + 1, np.float64)
    st = _load().kdto_fourier_moments(x.ctypes.data, x.size, J, out.ctypes.data)
    if st != 0:
        raise OracleError(st)
    return out


def fourier_split(x: np.ndarray, a: float, b: float, J: int) -> float:
    """Root of Eq. (kd:eq:b) on (a, b) for the key values x (float64 bisection)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = ctypes.c_double()
    st = _load().kdto_fourier_split(x.ctypes.data, x.size, a, b, J, ctypes.byref(m))
    if st != 0:
        raise OracleError(st)
    return m.value


def fourier_build_tree(points: np.ndarray, *, depth: int, J: int) -> Tree:
    """Depth-D tree whose splits are the estimator's roots (cyclic keys). points: float32 [d, n] in (0,1)."""
    points = np.ascontiguousarray(points, dtype=np.float32)
    d, n = points.shape
    perm = np.zeros(max(n, 1), np.uint32)
    vals = np.zeros((1 << depth) - 1, np.float32)
    dims = np.zeros((1 << depth) - 1, np.int8)
    offs = np.zeros((1 << depth) + 1, np.int64)
    st = _load().kdto_fourier_build(points.ctypes.data, n, d, depth, J, perm.ctypes.data, vals.ctypes.data,
                                    dims.ctypes.data, offs.ctypes.data)
    if st != 0:
        raise OracleError(st)
    return Tree(perm[:n].copy(), vals, dims, offs, depth)


def fourier_cell_bounds(split_vals: np.ndarray, heap: int, d: int) -> tuple[float, float]:
    """Bounds (a, b) of node `heap` on its cyclic key coordinate: the float
    splits of its ancestors on that coordinate, (0, 1) at the root."""
    level = int(np.floor(np.log2(heap + 1)))
    t = level % d
    a, b, h = 0.0, 1.0, heap
    while h > 0:
        par = (h - 1) // 2
        plevel = int(np.floor(np.log2(par + 1)))
        if plevel % d == t:
            v = float(split_vals[par])
            if h == 2 * par + 1:
                b = min(b, v)
            else:
                a = max(a, v)
        h = par
    return a, b


# ------------------------------------------- queries on the point set
# (Sec. 1: the searches the tree serves). Their definitions written out by
# brute force over every point; the tree plays no part.

def order_keys(x: np.ndarray) -> np.ndarray:
    """The order-preserving key of float32 values (-0.0 below +0.0), as uint64."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return np.where(b >> 31 == 1, b ^ 0xFFFFFFFF, b | 0x80000000)


def box_members(points: np.ndarray, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Original indices of the points with key(lo_j) <= key(x_j) <= key(hi_j)
    for every coordinate j (points [d, n], lo and hi [d])."""
    k = order_keys(points)
    inside = np.all((order_keys(lo)[:, None] <= k) & (k <= order_keys(hi)[:, None]), axis=0)
    return np.nonzero(inside)[0]


def squared_distances(points: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Per point: sum over j = 0..d-1, in that order, of the float64 square of
    the float64 difference of coordinate j (each step rounded to double)."""
    d2 = np.zeros(points.shape[1], np.float64)
    for j in range(points.shape[0]):
        diff = points[j].astype(np.float64) - np.float64(q[j])
        d2 = d2 + diff * diff
    return d2


def nearest(points: np.ndarray, q: np.ndarray, k: int):
    """The k nearest points to q: (indices, squared distances), nearest first,
    ties by the smaller index."""
    d2 = squared_distances(points, q)
    order = np.lexsort((np.arange(d2.size), d2))[:k]
    return order, d2[order]
