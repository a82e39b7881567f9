"""FP64 CPU oracle for EMST / HDBSCAN* (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and reference legs
may import this package.  The CUDA library never calls it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, compiled with ``-ffp-contract=off``); this file
only compiles it on first use, loads it with ctypes and marshals numpy arrays.  See the header
of ``oracle.c`` for what each function computes and which part of the paper it follows.

Functions whose parity is not pinned by an independent check are marked "parity unpinned" in
their docstring; at present every exported function has at least one independent pin in
``tests/test_oracle.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            lib.wmo_sqdist.restype = dbl
            lib.wmo_sqdist.argtypes = [P, i32, i64, i64]
            lib.wmo_core_dist2.restype = ctypes.c_int
            lib.wmo_core_dist2.argtypes = [P, i64, i32, i32, P]
            lib.wmo_core_dist2_subset.restype = ctypes.c_int
            lib.wmo_core_dist2_subset.argtypes = [P, i64, i32, i32, P, i64, P]
            lib.wmo_nearest_edge.restype = ctypes.c_int
            lib.wmo_nearest_edge.argtypes = [P, i64, i32, i64, P, P]
            lib.wmo_prim.restype = ctypes.c_int
            lib.wmo_prim.argtypes = [P, i64, i32, P, P, P, P, P]
            lib.wmo_sort_edges.restype = ctypes.c_int
            lib.wmo_sort_edges.argtypes = [i64, P, P, P]
            lib.wmo_total_weight.restype = dbl
            lib.wmo_total_weight.argtypes = [i64, P]
            lib.wmo_hop_distance.restype = ctypes.c_int
            lib.wmo_hop_distance.argtypes = [i64, P, P, i32, P]
            lib.wmo_dendrogram.restype = ctypes.c_int
            lib.wmo_dendrogram.argtypes = [i64, P, P, P, i32, P, P, P, P]
            lib.wmo_inorder_leaves.restype = ctypes.c_int
            lib.wmo_inorder_leaves.argtypes = [i64, P, P, P]
            lib.wmo_reachability.restype = ctypes.c_int
            lib.wmo_reachability.argtypes = [i64, P, P, P, i32, P, P]
            lib.wmo_core_dist2_kdtree.restype = ctypes.c_int
            lib.wmo_core_dist2_kdtree.argtypes = [P, i64, i32, i32, P]
            lib.wmo_boruvka.restype = ctypes.c_int
            lib.wmo_boruvka.argtypes = [P, i64, i32, P, P, P, P]
            lib.wmo_set_kd_stack_cap.restype = ctypes.c_int
            lib.wmo_set_kd_stack_cap.argtypes = [i32]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _pts(x) -> np.ndarray:
    x = np.asarray(x)
    if x.ndim != 2:
        raise ValueError("points must have shape (n, d)")
    # FP32-stored inputs are widened exactly to FP64.
    return np.ascontiguousarray(x, dtype=np.float64)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def set_kd_stack_cap(cap: int = 256):
    """Capacity of the k-d tree solvers' search stacks (default 256, never reached by a median
    split tree).  Tests lower it to check that a search that would overflow fails loudly."""
    _check(_load().wmo_set_kd_stack_cap(int(cap)), "set_kd_stack_cap")


def sqdist(x, i: int, j: int) -> float:
    """FP64 squared distance, dimension order, no FMA (Sec. 2.1)."""
    x = _pts(x)
    return _load().wmo_sqdist(_p(x), x.shape[1], i, j)


def core_dist2(x, min_pts: int) -> np.ndarray:
    """Squared core distances: the min_pts-th smallest D(p, .) counting p itself (Sec. 2.1)."""
    x = _pts(x)
    n, d = x.shape
    out = np.empty(n, dtype=np.float64)
    _check(_load().wmo_core_dist2(_p(x), n, d, int(min_pts), _p(out)), "core_dist2")
    return out


def core_dist2_subset(x, min_pts: int, idx) -> np.ndarray:
    """Squared core distances of the points idx only (brute force over all points)."""
    x = _pts(x)
    n, d = x.shape
    q = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(len(q), dtype=np.float64)
    _check(_load().wmo_core_dist2_subset(_p(x), n, d, int(min_pts), _p(q), len(q), _p(out)), "core_dist2_subset")
    return out


def nearest_edge(x, p: int):
    """The K-minimum EMST edge incident to point p: (other endpoint, w2)."""
    x = _pts(x)
    n, d = x.shape
    other = np.zeros(1, dtype=np.int32)
    w2 = np.zeros(1, dtype=np.float64)
    _check(_load().wmo_nearest_edge(_p(x), n, d, int(p), _p(other), _p(w2)), "nearest_edge")
    return int(other[0]), float(w2[0])


def prim_complete(x, cd2=None):
    """Prim on the complete graph under K (EMST, or G_MR when cd2 is given).

    Returns (u, v, w2, tie) with the edges in Prim insertion order, u < v.
    """
    x = _pts(x)
    n, d = x.shape
    m = max(n - 1, 0)
    u = np.empty(max(m, 1), dtype=np.int32)
    v = np.empty(max(m, 1), dtype=np.int32)
    w2 = np.empty(max(m, 1), dtype=np.float64)
    tie = np.zeros(1, dtype=np.int32)
    cdp = None
    if cd2 is not None:
        cd2 = np.ascontiguousarray(cd2, dtype=np.float64)
        cdp = _p(cd2)
    _check(_load().wmo_prim(_p(x), n, d, cdp, _p(u), _p(v), _p(w2), _p(tie)), "prim")
    return u[:m], v[:m], w2[:m], bool(tie[0])


def sort_edges(u, v, w2):
    """Return copies of (u, v, w2) sorted by K = (w2, min id, max id), normalised u < v."""
    u = np.ascontiguousarray(u, dtype=np.int32).copy()
    v = np.ascontiguousarray(v, dtype=np.int32).copy()
    w2 = np.ascontiguousarray(w2, dtype=np.float64).copy()
    _check(_load().wmo_sort_edges(len(u), _p(u), _p(v), _p(w2)), "sort_edges")
    return u, v, w2


def total_weight(w2) -> float:
    """Neumaier-compensated sum of sqrt(w2) in the given order."""
    w2 = np.ascontiguousarray(w2, dtype=np.float64)
    return _load().wmo_total_weight(len(w2), _p(w2))


def hop_distance(n: int, u, v, s: int = 0) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    hop = np.empty(n, dtype=np.int32)
    _check(_load().wmo_hop_distance(n, _p(u), _p(v), int(s), _p(hop)), "hop_distance")
    return hop


def dendrogram(n: int, u, v, w2, s: int = 0):
    """Ordered dendrogram from K-ordered tree edges (Sec. 4).  Returns (left, right, height, size)."""
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    w2 = np.ascontiguousarray(w2, dtype=np.float64)
    m = max(n - 1, 1)
    left = np.empty(m, dtype=np.int32)
    right = np.empty(m, dtype=np.int32)
    height = np.empty(m, dtype=np.float64)
    size = np.empty(m, dtype=np.int32)
    _check(_load().wmo_dendrogram(n, _p(u), _p(v), _p(w2), int(s), _p(left), _p(right), _p(height),
                                  _p(size)), "dendrogram")
    k = n - 1
    return left[:k], right[:k], height[:k], size[:k]


def inorder_leaves(n: int, left, right) -> np.ndarray:
    left = np.ascontiguousarray(left, dtype=np.int32)
    right = np.ascontiguousarray(right, dtype=np.int32)
    out = np.empty(n, dtype=np.int32)
    _check(_load().wmo_inorder_leaves(n, _p(left), _p(right), _p(out)), "inorder_leaves")
    return out


def reachability(n: int, u, v, w2, s: int = 0):
    """Prim order on the tree from s under K, and bar heights (Sec. 2.1).  Returns (order, reach)."""
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    w2 = np.ascontiguousarray(w2, dtype=np.float64)
    order = np.empty(n, dtype=np.int32)
    reach = np.empty(n, dtype=np.float64)
    _check(_load().wmo_reachability(n, _p(u), _p(v), _p(w2), int(s), _p(order), _p(reach)),
           "reachability")
    return order, reach


def core_dist2_kdtree(x, min_pts: int) -> np.ndarray:
    """core_dist2 computed by an exact k-d tree search (for sizes brute force cannot reach)."""
    x = _pts(x)
    n, d = x.shape
    out = np.empty(n, dtype=np.float64)
    _check(_load().wmo_core_dist2_kdtree(_p(x), n, d, int(min_pts), _p(out)), "core_dist2_kdtree")
    return out


def boruvka(x, cd2=None):
    """The K-minimum spanning tree (EMST, or G_MR when cd2 is given) by Boruvka's algorithm over an
    exact k-d tree: the tree prim_complete + sort_edges gives, for sizes brute force cannot reach.
    Returns (u, v, w2) in K order, u < v."""
    x = _pts(x)
    n, d = x.shape
    m = max(n - 1, 0)
    u = np.empty(max(m, 1), dtype=np.int32)
    v = np.empty(max(m, 1), dtype=np.int32)
    w2 = np.empty(max(m, 1), dtype=np.float64)
    cdp = None
    if cd2 is not None:
        cd2 = np.ascontiguousarray(cd2, dtype=np.float64)
        cdp = _p(cd2)
    _check(_load().wmo_boruvka(_p(x), n, d, cdp, _p(u), _p(v), _p(w2)), "boruvka")
    return u[:m], v[:m], w2[:m]


def emst_at_scale(x):
    """emst() by the k-d tree Boruvka solver (same result, any size the host can hold)."""
    x = _pts(x)
    u, v, w2 = boruvka(x)
    return {"u": u, "v": v, "w2": w2, "w": np.sqrt(w2), "total": total_weight(w2)}


def hdbscan_at_scale(x, min_pts: int, s: int = 0):
    """hdbscan() with the k-d tree core distances and Boruvka MST (same results, any size)."""
    x = _pts(x)
    n = x.shape[0]
    cd2 = core_dist2_kdtree(x, min_pts)
    u, v, w2 = boruvka(x, cd2)
    out = {"cd2": cd2, "cd": np.sqrt(cd2), "u": u, "v": v, "w2": w2, "w": np.sqrt(w2), "total": total_weight(w2)}
    if n >= 2:
        left, right, height, size = dendrogram(n, u, v, w2, s)
        order, reach = reachability(n, u, v, w2, s)
        out.update(left=left, right=right, height=height, size=size, order=order, reach=reach)
    return out


# ------------------------------------------------------------------ composed problem calls

def emst(x):
    """EMST of the points (Sec. 2.1): edges in K order, squared weights, total weight, tie flag."""
    x = _pts(x)
    u, v, w2, tie = prim_complete(x)
    u, v, w2 = sort_edges(u, v, w2)
    return {"u": u, "v": v, "w2": w2, "w": np.sqrt(w2), "total": total_weight(w2), "tie": tie}


def hdbscan(x, min_pts: int, s: int = 0):
    """HDBSCAN* (Sec. 2.1, Sec. 4): core distances, MST of G_MR in K order, ordered dendrogram
    of start point s, reachability plot from s (Prim order) and the dendrogram's in-order leaves."""
    x = _pts(x)
    n = x.shape[0]
    cd2 = core_dist2(x, min_pts)
    u, v, w2, tie = prim_complete(x, cd2)
    u, v, w2 = sort_edges(u, v, w2)
    out = {"cd2": cd2, "cd": np.sqrt(cd2), "u": u, "v": v, "w2": w2, "w": np.sqrt(w2),
           "total": total_weight(w2), "tie": tie}
    if n >= 2:
        left, right, height, size = dendrogram(n, u, v, w2, s)
        order, reach = reachability(n, u, v, w2, s)
        out.update(left=left, right=right, height=height, size=size, order=order, reach=reach,
                   inorder=inorder_leaves(n, left, right))
    else:
        out.update(left=np.empty(0, np.int32), right=np.empty(0, np.int32),
                   height=np.empty(0), size=np.empty(0, np.int32),
                   order=np.zeros(1, np.int32), reach=np.array([np.inf]),
                   inorder=np.zeros(1, np.int32))
    return out


def single_linkage(n: int, u, v, w2, s: int = 0):
    """Ordered single-linkage dendrogram + plot from any spanning tree (edges re-sorted by K)."""
    u, v, w2 = sort_edges(u, v, w2)
    left, right, height, size = dendrogram(n, u, v, w2, s)
    order, reach = reachability(n, u, v, w2, s)
    return {"left": left, "right": right, "height": height, "size": size, "order": order,
            "reach": reach, "inorder": inorder_leaves(n, left, right)}
