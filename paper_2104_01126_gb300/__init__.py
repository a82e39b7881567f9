"""Python binding of libwspdmst: EMST and HDBSCAN* on one GB300 GPU.

Thin ctypes marshalling over the C ABI in ``include/wspdmst.h``; every step of the computation
runs in the library's CUDA kernels.  Inputs may be numpy arrays (host) or torch tensors (host
or CUDA); results come back on the same side as the input (numpy for host inputs, torch CUDA
tensors for device inputs).  PyTorch supplies device memory (outputs and the optional
workspace arena) and the current CUDA stream.

The library must have been built (``python -m paper_2104_01126_gb300.build``); importing the
binding does not fall back to anything else: a missing or unloadable library raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

__all__ = ["emst", "hdbscan", "single_linkage", "query_footprint", "library_path", "load",
           "WMError", "Stats", "version", "batch", "get_tuning", "set_tuning", "tuning"]

WM_F32, WM_F64 = 0, 1
WM_AOS, WM_SOA = 0, 1
PREC = {"fp32": 0, "fp32_screen": 0, "fp64": 1}
METHODS = {"memogfk": 0, "gfk": 1, "naive": 2, "gantao": 0x100, "gfk-geometric": 0x101, "naive-geometric": 0x102}


class WMError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {detail or 'error'} (code {code})")
        self.code = code


class _Edge(ctypes.Structure):
    _fields_ = [("u", ctypes.c_int32), ("v", ctypes.c_int32), ("w", ctypes.c_double)]


class _DNode(ctypes.Structure):
    _fields_ = [("left", ctypes.c_int32), ("right", ctypes.c_int32), ("height", ctypes.c_double),
                ("size", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("ms_total", ctypes.c_double), ("ms_ingest", ctypes.c_double),
                ("ms_build_tree", ctypes.c_double), ("ms_core_dist", ctypes.c_double),
                ("ms_wspd", ctypes.c_double), ("ms_bccp", ctypes.c_double),
                ("ms_kruskal", ctypes.c_double), ("ms_dendrogram", ctypes.c_double),
                ("rounds", ctypes.c_int64), ("pairs_retrieved", ctypes.c_int64),
                ("bccp_evals", ctypes.c_int64), ("bccp_tile_evals", ctypes.c_int64),
                ("knn_evals", ctypes.c_int64), ("fp64_rechecks", ctypes.c_int64),
                ("candidate_edges", ctypes.c_int64), ("tree_nodes", ctypes.c_int64),
                ("tree_depth", ctypes.c_int64), ("workspace_bytes_used", ctypes.c_size_t),
                ("max_rel_screen_err", ctypes.c_double), ("tie_overflow", ctypes.c_int32),
                ("edge_batch_grown", ctypes.c_int32), ("ms_knn_kernel", ctypes.c_double),
                ("ms_tile_kernel", ctypes.c_double), ("tile_launches", ctypes.c_int64),
                ("ms_getpairs", ctypes.c_double), ("getpairs_launches", ctypes.c_int64),
                ("getpairs_visits", ctypes.c_int64), ("getrho_visits", ctypes.c_int64),
                ("bccp_dual_evals", ctypes.c_int64), ("rho_shrinks", ctypes.c_int64),
                ("max_pending_pairs", ctypes.c_int64), ("bccp_pairs_below", ctypes.c_int64),
                ("bccp_pairs_above", ctypes.c_int64), ("bccp_evals_outside", ctypes.c_int64),
                ("bccp_tile_evals_skipped", ctypes.c_int64), ("ms_getrho", ctypes.c_double),
                ("ms_bccp_group", ctypes.c_double), ("ms_bccp_dual", ctypes.c_double),
                ("wspd_pairs", ctypes.c_int64)]


class _Opts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("precision", ctypes.c_int32),
                ("method", ctypes.c_int32), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("stats", ctypes.POINTER(_Stats))]


class _Tuning(ctypes.Structure):
    _fields_ = [("tight_diameters", ctypes.c_int32), ("chunk_log2", ctypes.c_int32), ("dfs_budget", ctypes.c_int32),
                ("route_big", ctypes.c_int32), ("medium_max", ctypes.c_int32), ("big_max", ctypes.c_int32),
                ("combined", ctypes.c_int32), ("getrho_sample", ctypes.c_int32), ("edges_per_point", ctypes.c_int32),
                ("range_ratio", ctypes.c_int32), ("range_gate", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


TUNING_FIELDS = ("tight_diameters", "chunk_log2", "dfs_budget", "route_big", "medium_max", "big_max", "combined",
                 "getrho_sample", "edges_per_point", "range_ratio", "range_gate")


class _Instance(ctypes.Structure):
    _fields_ = [("pts", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("min_pts", ctypes.c_int32),
                ("start", ctypes.c_int32), ("reserved", ctypes.c_int32), ("out_edges", ctypes.c_void_p),
                ("out_total_weight", ctypes.c_void_p), ("out_core_dist", ctypes.c_void_p),
                ("out_dendro", ctypes.c_void_p), ("out_order", ctypes.c_void_p), ("out_reach", ctypes.c_void_p)]


class _Job(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dtype", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("d", ctypes.c_int32), ("n", ctypes.c_int64), ("pts", ctypes.c_void_p),
                ("min_pts", ctypes.c_int32), ("start", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("out_edges", ctypes.c_void_p),
                ("out_total_weight", ctypes.c_void_p), ("out_core_dist", ctypes.c_void_p),
                ("out_dendro", ctypes.c_void_p), ("out_order", ctypes.c_void_p), ("out_reach", ctypes.c_void_p)]


EDGE_DTYPE = np.dtype([("u", np.int32), ("v", np.int32), ("w", np.float64)])
DNODE_DTYPE = np.dtype([("left", np.int32), ("right", np.int32), ("height", np.float64),
                        ("size", np.int32), ("reserved", np.int32)])
assert EDGE_DTYPE.itemsize == ctypes.sizeof(_Edge) == 16
assert DNODE_DTYPE.itemsize == ctypes.sizeof(_DNode) == 24


@dataclass
class Stats:
    ms_total: float = 0.0
    ms_ingest: float = 0.0
    ms_build_tree: float = 0.0
    ms_core_dist: float = 0.0
    ms_wspd: float = 0.0
    ms_bccp: float = 0.0
    ms_kruskal: float = 0.0
    ms_dendrogram: float = 0.0
    rounds: int = 0
    pairs_retrieved: int = 0
    bccp_evals: int = 0
    bccp_tile_evals: int = 0
    knn_evals: int = 0
    fp64_rechecks: int = 0
    candidate_edges: int = 0
    tree_nodes: int = 0
    tree_depth: int = 0
    workspace_bytes_used: int = 0
    max_rel_screen_err: float = 0.0
    tie_overflow: int = 0
    edge_batch_grown: int = 0
    ms_knn_kernel: float = 0.0
    ms_tile_kernel: float = 0.0
    tile_launches: int = 0
    ms_getpairs: float = 0.0
    getpairs_launches: int = 0
    getpairs_visits: int = 0
    getrho_visits: int = 0
    bccp_dual_evals: int = 0
    rho_shrinks: int = 0
    max_pending_pairs: int = 0
    bccp_pairs_below: int = 0
    bccp_pairs_above: int = 0
    bccp_evals_outside: int = 0
    bccp_tile_evals_skipped: int = 0
    ms_getrho: float = 0.0
    ms_bccp_group: float = 0.0
    ms_bccp_dual: float = 0.0
    wspd_pairs: int = 0

    @classmethod
    def _from(cls, s: _Stats) -> "Stats":
        return cls(**{f: getattr(s, f) for f in cls.__dataclass_fields__})


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libwspdmst.so (building it first if it is missing and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libwspdmst not built: {path} is missing")
            _build.build()
        lib = ctypes.CDLL(path)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.wm_emst.restype = ctypes.c_int
        lib.wm_emst.argtypes = [P, i64, i32, i32, i32, P, P, ctypes.POINTER(_Opts)]
        lib.wm_hdbscan.restype = ctypes.c_int
        lib.wm_hdbscan.argtypes = [P, i64, i32, i32, i32, i32, P, P, P, P, P, i32, ctypes.POINTER(_Opts)]
        lib.wm_single_linkage.restype = ctypes.c_int
        lib.wm_single_linkage.argtypes = [P, i64, i32, P, P, P, ctypes.POINTER(_Opts)]
        lib.wm_query_footprint.restype = ctypes.c_int
        lib.wm_query_footprint.argtypes = [i64, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
        lib.wm_release_cache.restype = ctypes.c_int
        lib.wm_strerror.restype = ctypes.c_char_p
        lib.wm_strerror.argtypes = [ctypes.c_int]
        lib.wm_last_error_detail.restype = ctypes.c_char_p
        lib.wm_version.restype = ctypes.c_char_p
        lib.wm_kernel_launch_count.restype = ctypes.c_int64
        lib.wm_server_create.restype = ctypes.c_int
        lib.wm_server_create.argtypes = [i32, ctypes.c_size_t, i32, ctypes.POINTER(ctypes.c_void_p)]
        lib.wm_server_destroy.restype = ctypes.c_int
        lib.wm_server_destroy.argtypes = [P]
        lib.wm_submit.restype = ctypes.c_int
        lib.wm_submit.argtypes = [P, ctypes.POINTER(_Job), ctypes.POINTER(ctypes.c_int64)]
        lib.wm_poll.restype = ctypes.c_int
        lib.wm_poll.argtypes = [P, i64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
        lib.wm_wait.restype = ctypes.c_int
        lib.wm_wait.argtypes = [P, i64, ctypes.POINTER(ctypes.c_double)]
        lib.wm_server_counters.restype = ctypes.c_int
        lib.wm_server_counters.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_size_t),
                                           ctypes.POINTER(ctypes.c_int32)]
        lib.wm_batch.restype = ctypes.c_int
        lib.wm_batch.argtypes = [ctypes.POINTER(_Instance), i32, i32, i32, ctypes.POINTER(_Opts)]
        lib.wm_emst_noalloc.restype = ctypes.c_int
        lib.wm_emst_noalloc.argtypes = [P, i64, i32, i32, i32, P, P, ctypes.POINTER(_Opts)]
        lib.wm_fp32_fma_peak.restype = ctypes.c_int
        lib.wm_fp32_fma_peak.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.wm_get_tuning.restype = ctypes.c_int
        lib.wm_get_tuning.argtypes = [i64, i32, i32, ctypes.POINTER(_Tuning)]
        lib.wm_set_tuning.restype = ctypes.c_int
        lib.wm_set_tuning.argtypes = [ctypes.POINTER(_Tuning)]
        _lib = lib
        return lib


def version() -> str:
    return load().wm_version().decode()


def _check(rc: int, where: str):
    if rc != 0:
        lib = load()
        raise WMError(rc, where, (lib.wm_last_error_detail() or b"").decode() or lib.wm_strerror(rc).decode())


# ----------------------------------------------------------------------------- marshalling
def _torch():
    try:
        import torch  # noqa: F401
        return torch
    except Exception:  # pragma: no cover - torch is present in this project
        return None


def _is_cuda_tensor(x) -> bool:
    t = _torch()
    return t is not None and isinstance(x, t.Tensor) and x.is_cuda


def _points(x, layout: str = "aos"):
    """Returns (keepalive, pointer, n, d, dtype code, on_device, torch device or None).

    layout "aos": x has shape (n, d), a row per point; "soa": x has shape (d, n), a row per
    coordinate (the C ABI's WM_SOA)."""
    if layout not in ("aos", "soa"):
        raise ValueError("layout must be 'aos' or 'soa'")
    r = _points_aos(x)
    if layout == "soa":
        return r[0], r[1], r[3], r[2], r[4], r[5], r[6]
    return r


def _points_aos(x):
    t = _torch()
    if t is not None and isinstance(x, t.Tensor):
        if x.dim() != 2:
            raise ValueError("points must be a 2-D array")
        if x.dtype not in (t.float32, t.float64):
            x = x.to(t.float64)
        x = x.contiguous()
        code = WM_F32 if x.dtype == t.float32 else WM_F64
        return x, x.data_ptr(), x.shape[0], x.shape[1], code, x.is_cuda, (x.device if x.is_cuda else None)
    a = np.asarray(x)
    if a.ndim != 2:
        raise ValueError("points must be a 2-D array")
    if a.dtype not in (np.float32, np.float64):
        a = a.astype(np.float64)
    a = np.ascontiguousarray(a)
    code = WM_F32 if a.dtype == np.float32 else WM_F64
    return a, a.ctypes.data, a.shape[0], a.shape[1], code, False, None


def _opts(precision: str, stream, stats: _Stats, workspace=None, method: str = "memogfk"):
    o = _Opts()
    o.precision = PREC[precision]
    o.method = METHODS[method]
    o.stream = stream or None
    o.stats = ctypes.pointer(stats)
    if workspace is not None:
        o.workspace = workspace[0]
        o.workspace_bytes = workspace[1]
    return o


def _current_stream(device):
    t = _torch()
    if device is None or t is None:
        return None
    return t.cuda.current_stream(device).cuda_stream


def _out_buffer(nbytes: int, device):
    """A caller-owned output buffer: a torch uint8 CUDA tensor, or a numpy byte array."""
    t = _torch()
    if device is not None:
        buf = t.empty(max(nbytes, 16), dtype=t.uint8, device=device)
        return buf, buf.data_ptr()
    buf = np.empty(max(nbytes, 16), dtype=np.uint8)
    return buf, buf.ctypes.data


def _edges_result(buf, m: int, device):
    t = _torch()
    if device is not None:
        raw = buf[: 16 * m].view(t.int32).view(m, 4) if m > 0 else t.empty((0, 4), dtype=t.int32, device=device)
        u = raw[:, 0].clone()
        v = raw[:, 1].clone()
        w = buf[: 16 * m].view(t.float64).view(m, 2)[:, 1].clone() if m > 0 else t.empty(0, dtype=t.float64, device=device)
        return u, v, w
    e = np.frombuffer(buf, dtype=EDGE_DTYPE, count=m)
    return e["u"].copy(), e["v"].copy(), e["w"].copy()


def _dnode_result(buf, m: int, device):
    t = _torch()
    if device is not None:
        if m == 0:
            z = t.empty(0, dtype=t.int32, device=device)
            return z, z.clone(), t.empty(0, dtype=t.float64, device=device), z.clone()
        i32 = buf[: 24 * m].view(t.int32).view(m, 6)
        f64 = buf[: 24 * m].view(t.float64).view(m, 3)
        return i32[:, 0].clone(), i32[:, 1].clone(), f64[:, 1].clone(), i32[:, 4].clone()
    e = np.frombuffer(buf, dtype=DNODE_DTYPE, count=m)
    return e["left"].copy(), e["right"].copy(), e["height"].copy(), e["size"].copy()


# ---------------------------------------------------------------------------------- API
def emst(points, precision: str = "fp32", stream=None, return_stats: bool = False, workspace=None,
         layout: str = "aos", method: str = "memogfk"):
    """Euclidean MST (wm_emst).  Returns dict(u, v, w, total[, stats]); edges in K order.
    workspace: optional (device pointer, bytes) of a caller-owned arena; layout: "aos" for an
    (n, d) array, "soa" for a (d, n) array; method: "memogfk" (default), "gfk" (the full WSPD
    materialised, Algorithm 2) or "naive" (EMST-Naive)."""
    lib = load()
    keep, ptr, n, d, code, on_dev, dev = _points(points, layout)
    m = max(n - 1, 0)
    buf, bptr = _out_buffer(16 * m, dev)
    total = ctypes.c_double(0.0)
    st = _Stats()
    if stream is None and on_dev:
        stream = _current_stream(dev)
    o = _opts(precision, stream, st, workspace, method)
    rc = lib.wm_emst(ptr, n, d, code, WM_SOA if layout == "soa" else WM_AOS, bptr if m > 0 else None,
                     ctypes.byref(total), ctypes.byref(o))
    _check(rc, "wm_emst")
    u, v, w = _edges_result(buf, m, dev)
    out = {"u": u, "v": v, "w": w, "total": total.value}
    if return_stats:
        out["stats"] = Stats._from(st)
    del keep
    return out


def emst_noalloc(points, precision: str = "fp32", stream=None):
    """wm_emst_noalloc: the EMST with all device scratch taken from the library's static array
    (n <= 32768), for callers that must not allocate device memory.  Outputs are allocated here
    by the caller side of the binding, as the C entry point expects caller-owned outputs."""
    lib = load()
    keep, ptr, n, d, code, on_dev, dev = _points(points)
    m = max(n - 1, 0)
    buf, bptr = _out_buffer(16 * m, dev)
    total = ctypes.c_double(0.0)
    st = _Stats()
    if stream is None and on_dev:
        stream = _current_stream(dev)
    o = _opts(precision, stream, st)
    rc = lib.wm_emst_noalloc(ptr, n, d, code, WM_AOS, bptr if m > 0 else None, ctypes.byref(total), ctypes.byref(o))
    _check(rc, "wm_emst_noalloc")
    u, v, w = _edges_result(buf, m, dev)
    del keep
    return {"u": u, "v": v, "w": w, "total": total.value}


def hdbscan(points, min_pts: int = 10, start: int = 0, precision: str = "fp32", stream=None,
            return_stats: bool = False, workspace=None, layout: str = "aos", method: str = "memogfk"):
    """HDBSCAN* (wm_hdbscan): MST of G_MR, core distances, ordered dendrogram, reachability plot.
    workspace and layout as for emst(); method: "memogfk", "gfk", "naive" or "gantao" (the
    baseline with geometric separation only; "gfk-geometric" / "naive-geometric" combine it with
    the materialised WSPD)."""
    lib = load()
    keep, ptr, n, d, code, on_dev, dev = _points(points, layout)
    m = max(n - 1, 0)
    ebuf, eptr = _out_buffer(16 * m, dev)
    cbuf, cptr = _out_buffer(8 * n, dev)
    dbuf, dptr = _out_buffer(24 * m, dev)
    obuf, optr = _out_buffer(4 * n, dev)
    rbuf, rptr = _out_buffer(8 * n, dev)
    st = _Stats()
    if stream is None and on_dev:
        stream = _current_stream(dev)
    o = _opts(precision, stream, st, workspace, method)
    rc = lib.wm_hdbscan(ptr, n, d, code, WM_SOA if layout == "soa" else WM_AOS, int(min_pts), eptr if m else None,
                        cptr, dptr if m else None,
                        optr, rptr, int(start), ctypes.byref(o))
    _check(rc, "wm_hdbscan")
    u, v, w = _edges_result(ebuf, m, dev)
    left, right, height, size = _dnode_result(dbuf, m, dev)
    t = _torch()
    if dev is not None:
        cd = cbuf[: 8 * n].view(t.float64).clone()
        order = obuf[: 4 * n].view(t.int32).clone()
        reach = rbuf[: 8 * n].view(t.float64).clone()
    else:
        cd = np.frombuffer(cbuf, dtype=np.float64, count=n).copy()
        order = np.frombuffer(obuf, dtype=np.int32, count=n).copy()
        reach = np.frombuffer(rbuf, dtype=np.float64, count=n).copy()
    out = {"u": u, "v": v, "w": w, "cd": cd, "left": left, "right": right, "height": height,
           "size": size, "order": order, "reach": reach}
    if return_stats:
        out["stats"] = Stats._from(st)
    del keep
    return out


def batch(instances, precision: str = "fp32", stream=None, return_stats: bool = False, raw: bool = False):
    """Many independent instances in one call (wm_batch).

    instances: a list of (points, min_pts, start) with min_pts <= 1 for an EMST; all points torch
    CUDA tensors or all host arrays, of one dtype.  Returns a list of dicts: (u, v, w, total) for
    an EMST, the wm_hdbscan fields for an HDBSCAN* instance; the results of each instance are those
    of its own emst() / hdbscan() call."""
    lib = load()
    t = _torch()
    pts = [_points(p) for p, _, _ in instances]
    codes = {q[4] for q in pts}
    if len(codes) != 1:
        # one dtype per call: widen to FP64 (exact for FP32 values)
        pts = [_points(q[0].to(t.float64) if q[5] else np.asarray(q[0], dtype=np.float64)) for q in pts]
    code = pts[0][4]
    dev = next((q[6] for q in pts if q[6] is not None), None)
    k = len(instances)
    arr = (_Instance * k)()
    ns = [q[2] for q in pts]
    ms = [max(n - 1, 0) for n in ns]
    hd = [int(mp) >= 2 for _, mp, _ in instances]
    eoff = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
    poff = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    ebuf, eptr = _out_buffer(16 * int(eoff[-1]), dev)
    cbuf, cptr = _out_buffer(8 * int(poff[-1]), dev)
    dbuf, dptr = _out_buffer(24 * int(eoff[-1]), dev)
    obuf, optr = _out_buffer(4 * int(poff[-1]), dev)
    rbuf, rptr = _out_buffer(8 * int(poff[-1]), dev)
    totals = (ctypes.c_double * k)()
    for j, (q, (_, mp, s)) in enumerate(zip(pts, instances)):
        a = arr[j]
        a.pts, a.n, a.d, a.min_pts, a.start = q[1], q[2], q[3], int(mp), int(s)
        a.out_edges = eptr + 16 * int(eoff[j]) if ms[j] else None
        if hd[j]:
            a.out_core_dist = cptr + 8 * int(poff[j])
            a.out_dendro = dptr + 24 * int(eoff[j]) if ms[j] else None
            a.out_order = optr + 4 * int(poff[j])
            a.out_reach = rptr + 8 * int(poff[j])
        else:
            a.out_total_weight = ctypes.addressof(totals) + 8 * j
    st = _Stats()
    if stream is None and dev is not None:
        stream = _current_stream(dev)
    o = _opts(precision, stream, st)
    rc = lib.wm_batch(arr, k, code, WM_AOS, ctypes.byref(o))
    _check(rc, "wm_batch")
    if raw:
        # concatenated outputs (instance j's slices start at edge_offsets[j] / point_offsets[j])
        res = {"edges": ebuf, "core_dist": cbuf, "dendro": dbuf, "order": obuf, "reach": rbuf,
               "edge_offsets": eoff, "point_offsets": poff, "totals": list(totals)}
        return (res, Stats._from(st)) if return_stats else res
    out = []
    for j in range(k):
        m, n = ms[j], ns[j]
        e0, p0 = int(eoff[j]), int(poff[j])
        u, v, w = _edges_result(ebuf[16 * e0:], m, dev)
        r = {"u": u, "v": v, "w": w}
        if hd[j]:
            left, right, height, size = _dnode_result(dbuf[24 * e0:], m, dev)
            if dev is not None:
                cd = cbuf[8 * p0: 8 * (p0 + n)].view(t.float64).clone()
                order = obuf[4 * p0: 4 * (p0 + n)].view(t.int32).clone()
                reach = rbuf[8 * p0: 8 * (p0 + n)].view(t.float64).clone()
            else:
                cd = np.frombuffer(cbuf, dtype=np.float64, count=n, offset=8 * p0).copy()
                order = np.frombuffer(obuf, dtype=np.int32, count=n, offset=4 * p0).copy()
                reach = np.frombuffer(rbuf, dtype=np.float64, count=n, offset=8 * p0).copy()
            r.update(cd=cd, left=left, right=right, height=height, size=size, order=order, reach=reach)
        else:
            r["total"] = totals[j]
        out.append(r)
    del pts
    if return_stats:
        return out, Stats._from(st)
    return out


def single_linkage(n: int, u, v, w, start: int = 0, stream=None):
    """Ordered dendrogram + reachability plot of a weighted spanning tree (wm_single_linkage)."""
    lib = load()
    m = max(n - 1, 0)
    rec = np.zeros(max(m, 1), dtype=EDGE_DTYPE)
    rec["u"][:m] = np.asarray(u)[:m]
    rec["v"][:m] = np.asarray(v)[:m]
    rec["w"][:m] = np.asarray(w)[:m]
    dbuf = np.empty(max(24 * m, 24), np.uint8)
    order = np.empty(n, np.int32)
    reach = np.empty(n, np.float64)
    st = _Stats()
    o = _opts("fp32", stream, st)
    rc = lib.wm_single_linkage(rec.ctypes.data if m else None, n, int(start), dbuf.ctypes.data if m else None,
                               order.ctypes.data, reach.ctypes.data, ctypes.byref(o))
    _check(rc, "wm_single_linkage")
    left, right, height, size = _dnode_result(dbuf, m, None)
    return {"left": left, "right": right, "height": height, "size": size, "order": order, "reach": reach}


def query_footprint(n: int, d: int, min_pts: int = 0) -> int:
    lib = load()
    b = ctypes.c_size_t(0)
    _check(lib.wm_query_footprint(n, d, min_pts, ctypes.byref(b)), "wm_query_footprint")
    return b.value


def get_tuning(n: int, d: int, min_pts: int = 0) -> dict:
    """The speed parameters a call with these sizes uses (wm_get_tuning)."""
    t = _Tuning()
    _check(load().wm_get_tuning(int(n), int(d), int(min_pts), ctypes.byref(t)), "wm_get_tuning")
    return {f: getattr(t, f) for f in TUNING_FIELDS}


def set_tuning(params=None):
    """Overrides the built-in tuning table for every later call (wm_set_tuning); None restores it.
    params: a dict of TUNING_FIELDS (missing fields take the built-in defaults)."""
    lib = load()
    if params is None:
        _check(lib.wm_set_tuning(None), "wm_set_tuning")
        return
    base = get_tuning(0, 1, 0)
    base.update(params)
    t = _Tuning()
    for f in TUNING_FIELDS:
        setattr(t, f, int(base[f]))
    _check(lib.wm_set_tuning(ctypes.byref(t)), "wm_set_tuning")


class tuning:
    """Context manager: `with tuning(dfs_budget=4): ...` runs calls with an override."""

    def __init__(self, **params):
        self.params = params

    def __enter__(self):
        set_tuning(self.params)
        return self

    def __exit__(self, *exc):
        set_tuning(None)


def fp32_fma_peak():
    """Measured FP32 FMA throughput of the current device: (TFLOP/s, ms of the best run)."""
    t = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    _check(load().wm_fp32_fma_peak(ctypes.byref(t), ctypes.byref(ms)), "wm_fp32_fma_peak")
    return t.value, ms.value


def kernel_launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().wm_kernel_launch_count())


def release_cache():
    _check(load().wm_release_cache(), "wm_release_cache")


# ------------------------------------------------------------------------------- serving
class Server:
    """Continuous-batching server (wm_server_*): jobs run concurrently on one device, admitted
    against an HBM budget.  Host inputs and outputs only (numpy); each submitted job keeps its
    buffers alive until it is waited for."""

    def __init__(self, hbm_budget_bytes: int, workers: int = 4, device: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.wm_server_create(device, int(hbm_budget_bytes), int(workers), ctypes.byref(h)),
               "wm_server_create")
        self._h = h
        self._lib = lib
        self._keep = {}

    def submit(self, points, kind: str = "emst", min_pts: int = 10, start: int = 0, precision: str = "fp32") -> int:
        x = np.ascontiguousarray(points)
        if x.dtype not in (np.float32, np.float64):
            x = x.astype(np.float64)
        n, d = x.shape
        m = max(n - 1, 0)
        job = _Job()
        job.kind = 0 if kind == "emst" else 1
        job.dtype = WM_F32 if x.dtype == np.float32 else WM_F64
        job.layout = WM_AOS
        job.d = d
        job.n = n
        job.pts = x.ctypes.data
        job.min_pts = int(min_pts)
        job.start = int(start)
        job.precision = PREC[precision]
        bufs = {"x": x, "edges": np.zeros(max(m, 1), dtype=EDGE_DTYPE), "total": np.zeros(1)}
        job.out_edges = bufs["edges"].ctypes.data if m else None
        if job.kind == 0:
            job.out_total_weight = bufs["total"].ctypes.data
        else:
            bufs.update(cd=np.zeros(n), dendro=np.zeros(max(m, 1), dtype=DNODE_DTYPE),
                        order=np.zeros(n, np.int32), reach=np.zeros(n))
            job.out_core_dist = bufs["cd"].ctypes.data
            job.out_dendro = bufs["dendro"].ctypes.data if m else None
            job.out_order = bufs["order"].ctypes.data
            job.out_reach = bufs["reach"].ctypes.data
        t = ctypes.c_int64(0)
        _check(self._lib.wm_submit(self._h, ctypes.byref(job), ctypes.byref(t)), "wm_submit")
        self._keep[t.value] = (job, bufs, kind, n)
        return t.value

    def poll(self, ticket: int):
        st = ctypes.c_int32(0)
        lat = ctypes.c_double(0.0)
        _check(self._lib.wm_poll(self._h, ticket, ctypes.byref(st), ctypes.byref(lat)), "wm_poll")
        return st.value, lat.value

    def wait(self, ticket: int):
        """Blocks until the job is done; returns (result dict, latency in ms)."""
        lat = ctypes.c_double(0.0)
        rc = self._lib.wm_wait(self._h, ticket, ctypes.byref(lat))
        job, bufs, kind, n = self._keep.pop(ticket)
        _check(rc, "wm_wait")
        m = max(n - 1, 0)
        e = bufs["edges"][:m]
        out = {"u": e["u"].copy(), "v": e["v"].copy(), "w": e["w"].copy()}
        if kind == "emst":
            out["total"] = float(bufs["total"][0])
        else:
            dn = bufs["dendro"][:m]
            out.update(cd=bufs["cd"], left=dn["left"].copy(), right=dn["right"].copy(),
                       height=dn["height"].copy(), size=dn["size"].copy(), order=bufs["order"],
                       reach=bufs["reach"])
        return out, lat.value

    def counters(self):
        f = ctypes.c_int64(0)
        b = ctypes.c_size_t(0)
        r = ctypes.c_int32(0)
        _check(self._lib.wm_server_counters(self._h, ctypes.byref(f), ctypes.byref(b), ctypes.byref(r)),
               "wm_server_counters")
        return {"finished": f.value, "peak_bytes": b.value, "peak_running": r.value}

    def close(self):
        if self._h:
            _check(self._lib.wm_server_destroy(self._h), "wm_server_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
