"""GB300 LSH query-workload library: Python binding of ``libqwlsh.so``.

Argument marshalling only.  Every step of the method (hashing, index build,
bucket-range search, collision counting, candidate selection, distances,
top-k) runs in the library's CUDA kernels; this module passes pointers, sizes
and the current CUDA stream through the C ABI declared in
``include/qwlsh.h``.  There is no fallback: if the library is missing, loading
it raises.

Raw entry points keep the C names (``qw_build_index``, ``qw_run_workload``,
``qw_hash`` ...).  ``Index`` and ``hash`` wrap them for torch tensors: CUDA
tensors are passed as device pointers (``QW_MEM_DEVICE``), CPU tensors as host
pointers (``QW_MEM_HOST``, the library copies in and out).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG_DIR, "libqwlsh.so")

QW_OK, QW_ERR_ARG, QW_ERR_OOM, QW_ERR_CUDA, QW_ERR_TIMEOUT, QW_ERR_RANGE = range(6)
QW_MEM_DEVICE, QW_MEM_HOST = 0, 1
QW_NSTAT = 8
QW_MAX_M = 127
QW_MAX_CAND = 4096
STAT_FIELDS = ("levels", "final_R", "n_cand_raw", "n_cand", "term", "scanned_last",
               "scanned_full", "n_prev")

# Every symbol include/qwlsh.h declares.
EXPORTED = ("qw_version", "qw_last_error", "qw_collision_probability",
            "qw_collision_threshold", "qw_hash", "qw_build_index", "qw_run_workload",
            "qw_workload_candidates", "qw_run_workload_noalloc", "qw_index_profile",
            "qw_index_get_info", "qw_index_export", "qw_index_free")


class qw_index_params(C.Structure):
    _fields_ = [("m", C.c_int32), ("w", C.c_float), ("c", C.c_int32), ("v", C.c_int32),
                ("l", C.c_int32), ("delta", C.c_float)]


class qw_query_params(C.Structure):
    _fields_ = [("batch", C.c_int32), ("profile", C.c_int32), ("path", C.c_int32),
                ("clusters", C.c_int32), ("order", C.c_int32), ("reserved", C.c_int32 * 3)]


QW_PATH_AUTO, QW_PATH_CLUSTER, QW_PATH_LEVELS = 0, 1, 2
PATHS = {"auto": QW_PATH_AUTO, "cluster": QW_PATH_CLUSTER, "levels": QW_PATH_LEVELS}
QW_ORDER_AUTO, QW_ORDER_SIGNATURE, QW_ORDER_GIVEN = 0, 1, 2
ORDERS = {"auto": QW_ORDER_AUTO, "signature": QW_ORDER_SIGNATURE, "given": QW_ORDER_GIVEN}
(QW_K_PROJECT, QW_K_SETUP, QW_K_LEVEL, QW_K_DECIDE, QW_K_SELECT, QW_K_RERANK, QW_K_CLUSTER,
 QW_K_ORDER) = range(8)
QW_K_COUNT = 8
KERNEL_CLASSES = ("project", "setup", "level", "decide", "select", "rerank", "cluster", "order")


class qw_profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * QW_K_COUNT), ("ms", C.c_double * QW_K_COUNT),
                ("timed_launches", C.c_int64 * QW_K_COUNT), ("queries", C.c_int64)]


class qw_index_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("m", C.c_int32), ("w", C.c_float),
                ("c", C.c_int32), ("v", C.c_int32), ("l", C.c_int32), ("tile", C.c_int32),
                ("n_tiles", C.c_int32), ("span_max", C.c_int32), ("n_fixups", C.c_int64),
                ("device_bytes", C.c_int64)]


class QwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[qw status {status}] {msg}")
        self.status = status


_lib: Optional[C.CDLL] = None


def load(path: Optional[str] = None) -> C.CDLL:
    """Load libqwlsh.so (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(p)
    vp = C.c_void_p
    L.qw_version.restype = C.c_char_p
    L.qw_version.argtypes = []
    L.qw_last_error.restype = C.c_char_p
    L.qw_last_error.argtypes = []
    L.qw_collision_probability.restype = C.c_double
    L.qw_collision_probability.argtypes = [C.c_double, C.c_double]
    L.qw_collision_threshold.restype = C.c_int32
    L.qw_collision_threshold.argtypes = [C.c_int32, C.c_float, C.c_int32, C.c_int64, C.c_int32,
                                         C.c_float]
    L.qw_hash.restype = C.c_int32
    L.qw_hash.argtypes = [vp, C.c_int64, C.c_int32, vp, vp, C.c_int32, C.c_float, vp,
                          C.POINTER(C.c_int64), vp]
    L.qw_build_index.restype = C.c_int32
    L.qw_build_index.argtypes = [vp, C.c_int64, C.c_int32, vp, vp, C.POINTER(qw_index_params),
                                 C.c_int32, vp, C.POINTER(vp)]
    L.qw_run_workload.restype = C.c_int32
    L.qw_run_workload.argtypes = [vp, vp, C.c_int64, C.c_int32, C.POINTER(qw_query_params), vp,
                                  vp, vp, C.c_int32, vp]
    L.qw_workload_candidates.restype = C.c_int32
    L.qw_workload_candidates.argtypes = [vp, vp, C.c_int64, C.c_int32, C.POINTER(qw_query_params),
                                         vp, vp, vp, C.c_int32, vp]
    L.qw_run_workload_noalloc.restype = C.c_int32
    L.qw_run_workload_noalloc.argtypes = [vp, vp, C.c_int64, C.c_int32, vp, vp, vp, vp]
    L.qw_index_profile.restype = C.c_int32
    L.qw_index_profile.argtypes = [vp, C.POINTER(qw_profile), C.c_int32]
    L.qw_index_get_info.restype = C.c_int32
    L.qw_index_get_info.argtypes = [vp, C.POINTER(qw_index_info)]
    L.qw_index_export.restype = C.c_int32
    L.qw_index_export.argtypes = [vp, vp, vp, vp, vp, vp]
    L.qw_index_free.restype = None
    L.qw_index_free.argtypes = [vp]
    if path is None:
        _lib = L
    return L


def _check(status: int):
    if status != QW_OK:
        msg = load().qw_last_error().decode(errors="replace")
        raise QwError(status, msg)


# ---------------------------------------------------------------- raw C names
def qw_version() -> str:
    return load().qw_version().decode()


def qw_collision_probability(r: float, w: float) -> float:
    return float(load().qw_collision_probability(r, w))


def qw_collision_threshold(m: int, w: float, c: int, n: int, v: int, delta: float = 0.0) -> int:
    return int(load().qw_collision_threshold(m, w, c, n, v, delta))


def qw_hash(V: int, nv: int, d: int, A: int, b: int, m: int, w: float, H: int, stream: int = 0):
    """Device pointers in, returns the number of FP64 recomputations."""
    fix = C.c_int64(0)
    _check(load().qw_hash(V, nv, d, A, b, m, w, H, C.byref(fix), stream or None))
    return int(fix.value)


def qw_build_index(data: int, n: int, d: int, A: int, b: int, params: qw_index_params, mem: int,
                   stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load().qw_build_index(data, n, d, A, b, C.byref(params), mem, stream or None,
                                 C.byref(h)))
    return int(h.value)


def qw_run_workload(index: int, queries: int, nq: int, k: int, qparams: qw_query_params,
                    ids: int, dists: int, stats: int, mem: int, stream: int = 0):
    _check(load().qw_run_workload(index, queries, nq, k, C.byref(qparams), ids, dists,
                                  stats or None, mem, stream or None))


def qw_workload_candidates(index: int, queries: int, nq: int, k: int, qparams: qw_query_params,
                           cand_ids: int, cand_col: int, stats: int, mem: int, stream: int = 0):
    _check(load().qw_workload_candidates(index, queries, nq, k, C.byref(qparams), cand_ids,
                                         cand_col or None, stats or None, mem, stream or None))


def qw_run_workload_noalloc(index: int, queries: int, nq: int, k: int, ids: int, dists: int,
                            stats: int, stream: int = 0):
    """Device pointers only; uses the library's static scratch, allocates nothing."""
    _check(load().qw_run_workload_noalloc(index, queries, nq, k, ids, dists, stats or None,
                                          stream or None))


def qw_index_profile(index: int, reset: bool = False) -> qw_profile:
    prof = qw_profile()
    _check(load().qw_index_profile(index, C.byref(prof), 1 if reset else 0))
    return prof


def qw_index_get_info(index: int) -> qw_index_info:
    info = qw_index_info()
    _check(load().qw_index_get_info(index, C.byref(info)))
    return info


def qw_index_export(index: int, o: int, span: int, entry_bid: int, entry_id: int,
                    stream: int = 0):
    _check(load().qw_index_export(index, o or None, span or None, entry_bid or None,
                                  entry_id or None, stream or None))


def qw_index_free(index: int):
    if index:
        load().qw_index_free(index)


# ---------------------------------------------------------------- torch helpers
def _torch():
    import torch
    return torch


def _stream_of(t) -> int:
    torch = _torch()
    if t.is_cuda:
        return int(torch.cuda.current_stream(t.device).cuda_stream)
    return 0


def _mem_of(*tensors) -> int:
    dev = {bool(t.is_cuda) for t in tensors if t is not None}
    if len(dev) != 1:
        raise ValueError("all tensors of one call must be on the GPU, or all on the host")
    return QW_MEM_DEVICE if dev.pop() else QW_MEM_HOST


def _f32(t, name):
    torch = _torch()
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 tensor")
    return t


def hash(V, A, b, w: float):
    """Bucket ids floor((A V^T + b) / w) of CUDA float32 tensors.

    Returns (H int32 nv x m on V's device, number of FP64 recomputations)."""
    torch = _torch()
    _f32(V, "V"), _f32(A, "A"), _f32(b, "b")
    if not (V.is_cuda and A.is_cuda and b.is_cuda):
        raise ValueError("hash() takes CUDA tensors")
    nv, d = V.shape
    m = A.shape[0]
    H = torch.empty((nv, m), dtype=torch.int32, device=V.device)
    fix = qw_hash(V.data_ptr(), nv, d, A.data_ptr(), b.data_ptr(), m, float(w), H.data_ptr(),
                  _stream_of(V))
    return H, fix


class Index:
    """An LSH index over ``data`` (n x d float32), owning device memory.

    ``A`` (m x d) and ``b`` (m) are the hash family's random draws (Section 3),
    passed in so callers control the seed.  ``l = 0`` derives the collision
    threshold from Eq. 1 (see ``qw_collision_threshold``)."""

    def __init__(self, data, A, b, *, w: float, c: int = 2, v: int = 100, l: int = 0,
                 delta: float = 0.0):
        _f32(data, "data"), _f32(A, "A"), _f32(b, "b")
        mem = _mem_of(data, A, b)
        n, d = data.shape
        m, d2 = A.shape
        if d2 != d or b.shape != (m,):
            raise ValueError("shape mismatch between data, A and b")
        p = qw_index_params(m=m, w=float(w), c=int(c), v=int(v), l=int(l), delta=float(delta))
        self._h = 0
        self._h = qw_build_index(data.data_ptr(), n, d, A.data_ptr(), b.data_ptr(), p, mem,
                                 _stream_of(data))
        self.n, self.d, self.m = n, d, m
        self.info = qw_index_get_info(self._h)

    @property
    def handle(self) -> int:
        return self._h

    @property
    def l(self) -> int:
        return int(self.info.l)

    @property
    def v(self) -> int:
        return int(self.info.v)

    def profile(self, reset: bool = False) -> dict:
        """Launch counts and (profile mode) summed kernel milliseconds per kernel
        class since the last reset."""
        p = qw_index_profile(self._h, reset)
        return {"launches": dict(zip(KERNEL_CLASSES, list(p.launches))),
                "ms": dict(zip(KERNEL_CLASSES, list(p.ms))),
                "timed_launches": dict(zip(KERNEL_CLASSES, list(p.timed_launches))),
                "queries": int(p.queries)}

    def query(self, Q, k: int, *, batch: int = 0, stats: bool = False, out=None,
              profile: bool = False, path: str = "auto", clusters: int = 0,
              order: str = "auto"):
        """Top-k of every query row.  Returns (ids int64 nq x k, dists float32
        nq x k[, stats int64 nq x QW_NSTAT]) on Q's device (host tensors in,
        host tensors out).  ``out`` may give preallocated (ids, dists[, stats])."""
        torch = _torch()
        _f32(Q, "Q")
        nq, d = Q.shape
        if d != self.d:
            raise ValueError("query dimension differs from the index")
        if out is not None:
            ids, dists = out[0], out[1]
            st = out[2] if (stats and len(out) > 2) else None
        else:
            pin = (not Q.is_cuda) and Q.is_pinned()
            ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device, pin_memory=pin)
            dists = torch.empty((nq, k), dtype=torch.float32, device=Q.device, pin_memory=pin)
            st = (torch.empty((nq, QW_NSTAT), dtype=torch.int64, device=Q.device, pin_memory=pin)
                  if stats else None)
        mem = _mem_of(Q, ids, dists, st)
        qp = qw_query_params(batch=int(batch), profile=1 if profile else 0, path=PATHS[path],
                             clusters=int(clusters), order=ORDERS[order])
        qw_run_workload(self._h, Q.data_ptr(), nq, int(k), qp, ids.data_ptr(), dists.data_ptr(),
                        st.data_ptr() if st is not None else 0, mem, _stream_of(Q))
        return (ids, dists, st) if stats else (ids, dists)

    def candidates(self, Q, k: int, *, batch: int = 0, path: str = "auto", order: str = "auto"):
        """Kept candidates per query (ascending ids, -1 padded) with their
        collision counts, and the per-query statistics, on Q's device."""
        torch = _torch()
        _f32(Q, "Q")
        nq = Q.shape[0]
        cap = k + self.v
        cid = torch.empty((nq, cap), dtype=torch.int64, device=Q.device)
        ccol = torch.empty((nq, cap), dtype=torch.int32, device=Q.device)
        st = torch.empty((nq, QW_NSTAT), dtype=torch.int64, device=Q.device)
        mem = _mem_of(Q, cid, ccol, st)
        qp = qw_query_params(batch=int(batch), path=PATHS[path], order=ORDERS[order])
        qw_workload_candidates(self._h, Q.data_ptr(), nq, int(k), qp, cid.data_ptr(),
                               ccol.data_ptr(), st.data_ptr(), mem, _stream_of(Q))
        return cid, ccol, st

    def export(self):
        """Host numpy copies: o (m), span (m), entry_bid and entry_id (m x n),
        entries of each projection ordered by (id tile, bid, id)."""
        import numpy as np
        o = np.empty(self.m, np.int32)
        span = np.empty(self.m, np.int32)
        eb = np.empty((self.m, self.n), np.int32)
        ei = np.empty((self.m, self.n), np.int32)
        qw_index_export(self._h, o.ctypes.data, span.ctypes.data, eb.ctypes.data, ei.ctypes.data)
        return o, span, eb, ei

    def free(self):
        if self._h:
            qw_index_free(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def collision_probability(r: float, w: float) -> float:
    """Eq. 1 in closed form (library implementation)."""
    return qw_collision_probability(r, w)


def collision_threshold(m: int, w: float, c: int, n: int, v: int, delta: float = 0.0) -> int:
    return qw_collision_threshold(m, w, c, n, v, delta)


__all__ = ["Index", "hash", "load", "QwError", "collision_probability", "collision_threshold",
           "STAT_FIELDS", "EXPORTED"] + [n for n in EXPORTED]
