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
            "qw_index_get_info", "qw_mlp_create", "qw_mlp_param_count", "qw_mlp_set_params",
            "qw_mlp_get_params", "qw_mlp_loss_grad", "qw_mlp_train", "qw_mlp_predict",
            "qw_mlp_free", "qw_query_features", "qw_index_set_start_model", "qw_autotune",
            "qw_index_export", "qw_index_free", "qw_l2_split_model", "qw_mlp_predict_tc",
            "qw_draw_projections", "qw_index_get_projections", "qw_measure_read_bandwidth",
            "qw_hash_tc", "qw_qalsh_collision_probability", "qw_qalsh_collision_threshold")


class qw_index_params(C.Structure):
    _fields_ = [("m", C.c_int32), ("w", C.c_float), ("c", C.c_int32), ("v", C.c_int32),
                ("l", C.c_int32), ("delta", C.c_float), ("shadow_bf16", C.c_int32),
                ("bitmaps", C.c_int32), ("host_bitmaps", C.c_int32), ("seed", C.c_uint64),
                ("projection", C.c_int32), ("family", C.c_int32)]


class qw_query_params(C.Structure):
    _fields_ = [("batch", C.c_int32), ("profile", C.c_int32), ("path", C.c_int32),
                ("clusters", C.c_int32), ("order", C.c_int32), ("rerank", C.c_int32),
                ("start", C.c_int32), ("graph", C.c_int32), ("bitmap_loads", C.c_int32),
                ("l2_mode", C.c_int32), ("l2_index_permille", C.c_int32),
                ("projection", C.c_int32), ("rerank_rows", C.c_int32),
                ("tiles_per_warp", C.c_int32), ("probes", C.c_int32)]


QW_TUNE_MAX = 32


class qw_tune_report(C.Structure):
    _fields_ = [("tried", C.c_int32), ("params", qw_query_params * QW_TUNE_MAX),
                ("ms", C.c_float * QW_TUNE_MAX), ("best", C.c_int32)]


QW_PATH_AUTO, QW_PATH_CLUSTER, QW_PATH_LEVELS, QW_PATH_BITMAP = 0, 1, 2, 3
PATHS = {"auto": QW_PATH_AUTO, "cluster": QW_PATH_CLUSTER, "levels": QW_PATH_LEVELS,
         "bitmap": QW_PATH_BITMAP}
QW_ORDER_AUTO, QW_ORDER_SIGNATURE, QW_ORDER_GIVEN = 0, 1, 2
QW_RERANK_FP32, QW_RERANK_BF16, QW_RERANK_BF16_TC = 0, 1, 2
RERANKS = {"fp32": QW_RERANK_FP32, "bf16": QW_RERANK_BF16, "bf16_tc": QW_RERANK_BF16_TC}
ORDERS = {"auto": QW_ORDER_AUTO, "signature": QW_ORDER_SIGNATURE, "given": QW_ORDER_GIVEN}
QW_START_PLAIN, QW_START_LEARNED = 0, 1
STARTS = {"plain": QW_START_PLAIN, "learned": QW_START_LEARNED}
QW_PROJ_FP32, QW_PROJ_TENSOR = 0, 1
PROJECTIONS = {"fp32": QW_PROJ_FP32, "tensor": QW_PROJ_TENSOR}
QW_FAMILY_E2LSH, QW_FAMILY_QALSH = 0, 1
FAMILIES = {"e2lsh": QW_FAMILY_E2LSH, "qalsh": QW_FAMILY_QALSH}
QW_LOADS_TMA, QW_LOADS_DIRECT, QW_LOADS_FUSED = 0, 1, 2
LOADS = {"tma": QW_LOADS_TMA, "direct": QW_LOADS_DIRECT, "fused": QW_LOADS_FUSED}
QW_L2_OFF, QW_L2_SPLIT, QW_L2_MODEL = 0, 1, 2
(QW_K_PROJECT, QW_K_SETUP, QW_K_LEVEL, QW_K_DECIDE, QW_K_SELECT, QW_K_RERANK, QW_K_CLUSTER,
 QW_K_ORDER, QW_K_START, QW_K_BUCKET) = range(10)
QW_K_COUNT = 10
KERNEL_CLASSES = ("project", "setup", "level", "decide", "select", "rerank", "cluster", "order",
                  "start", "bucket")


class qw_profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * QW_K_COUNT), ("ms", C.c_double * QW_K_COUNT),
                ("timed_launches", C.c_int64 * QW_K_COUNT), ("queries", C.c_int64),
                ("rerank_candidates", C.c_int64), ("rerank_fp32_rows", C.c_int64),
                ("start_levels_skipped", C.c_int64), ("start_fallbacks", C.c_int64),
                ("level_passes", C.c_int64), ("bitmap_fallbacks", C.c_int64),
                ("bitmap_live_items", C.c_int64), ("bitmap_live_groups", C.c_int64),
                ("bitmap_live_words", C.c_int64), ("l2_setaside_bytes", C.c_int64),
                ("l2_index_permille", C.c_int64), ("bitmap_overflows", C.c_int64)]


class qw_index_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("m", C.c_int32), ("w", C.c_float),
                ("c", C.c_int32), ("v", C.c_int32), ("l", C.c_int32), ("tile", C.c_int32),
                ("n_tiles", C.c_int32), ("span_max", C.c_int32), ("n_fixups", C.c_int64),
                ("device_bytes", C.c_int64), ("bitmap_bytes", C.c_int64),
                ("host_bytes", C.c_int64), ("family", C.c_int32)]


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
    L.qw_qalsh_collision_probability.restype = C.c_double
    L.qw_qalsh_collision_probability.argtypes = [C.c_double, C.c_double]
    L.qw_qalsh_collision_threshold.restype = C.c_int32
    L.qw_qalsh_collision_threshold.argtypes = [C.c_int32, C.c_float, C.c_int32, C.c_int64,
                                               C.c_int32, C.c_float]
    L.qw_hash.restype = C.c_int32
    L.qw_hash.argtypes = [vp, C.c_int64, C.c_int32, vp, vp, C.c_int32, C.c_float, vp,
                          C.POINTER(C.c_int64), vp]
    L.qw_hash_tc.restype = C.c_int32
    L.qw_hash_tc.argtypes = [vp, C.c_int64, C.c_int32, vp, vp, C.c_int32, C.c_float, vp,
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
    L.qw_mlp_create.restype = C.c_int32
    L.qw_mlp_create.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.POINTER(vp)]
    L.qw_mlp_param_count.restype = C.c_int64
    L.qw_mlp_param_count.argtypes = [vp]
    L.qw_mlp_set_params.restype = C.c_int32
    L.qw_mlp_set_params.argtypes = [vp, vp, C.c_int64]
    L.qw_mlp_get_params.restype = C.c_int32
    L.qw_mlp_get_params.argtypes = [vp, vp, C.c_int64]
    L.qw_mlp_loss_grad.restype = C.c_int32
    L.qw_mlp_loss_grad.argtypes = [vp, vp, vp, C.c_int64, C.POINTER(C.c_float), vp, vp]
    L.qw_mlp_train.restype = C.c_int32
    L.qw_mlp_train.argtypes = [vp, vp, vp, C.c_int64, C.c_int32, C.c_int32, C.c_float,
                               C.POINTER(C.c_float), vp]
    L.qw_mlp_predict.restype = C.c_int32
    L.qw_mlp_predict.argtypes = [vp, vp, C.c_int64, vp, vp]
    L.qw_mlp_predict_tc.restype = C.c_int32
    L.qw_mlp_predict_tc.argtypes = [vp, vp, C.c_int64, vp, vp]
    L.qw_mlp_free.restype = None
    L.qw_mlp_free.argtypes = [vp]
    L.qw_autotune.restype = C.c_int32
    L.qw_autotune.argtypes = [vp, vp, C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                              C.POINTER(qw_query_params), C.POINTER(qw_query_params),
                              C.POINTER(qw_tune_report), vp]
    L.qw_query_features.restype = C.c_int32
    L.qw_query_features.argtypes = [vp, vp, C.c_int64, vp, vp]
    L.qw_index_set_start_model.restype = C.c_int32
    L.qw_index_set_start_model.argtypes = [vp, vp, C.c_float]
    L.qw_index_profile.restype = C.c_int32
    L.qw_index_profile.argtypes = [vp, C.POINTER(qw_profile), C.c_int32]
    L.qw_index_get_info.restype = C.c_int32
    L.qw_index_get_info.argtypes = [vp, C.POINTER(qw_index_info)]
    L.qw_index_export.restype = C.c_int32
    L.qw_index_export.argtypes = [vp, vp, vp, vp, vp, vp]
    L.qw_index_free.restype = None
    L.qw_index_free.argtypes = [vp]
    L.qw_draw_projections.restype = None
    L.qw_draw_projections.argtypes = [C.c_uint64, C.c_int32, C.c_int32, C.c_float, vp, vp]
    L.qw_index_get_projections.restype = C.c_int32
    L.qw_index_get_projections.argtypes = [vp, vp, vp, vp]
    L.qw_measure_read_bandwidth.restype = C.c_int32
    L.qw_measure_read_bandwidth.argtypes = [C.c_int64, C.c_int32, C.POINTER(C.c_double), vp]
    L.qw_l2_split_model.restype = C.c_int32
    L.qw_l2_split_model.argtypes = [C.c_double] * 5
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


def qw_qalsh_collision_probability(r: float, w: float) -> float:
    return float(load().qw_qalsh_collision_probability(r, w))


def qw_qalsh_collision_threshold(m: int, w: float, c: int, n: int, v: int,
                                 delta: float = 0.0) -> int:
    return int(load().qw_qalsh_collision_threshold(m, w, c, n, v, delta))


def qw_l2_split_model(setaside: float, index_bytes: float, index_reads: float,
                      data_bytes: float, data_reads: float) -> int:
    """Permille of the persisting-L2 set-aside for the index window (-1: bad
    arguments)."""
    return int(load().qw_l2_split_model(setaside, index_bytes, index_reads, data_bytes,
                                        data_reads))


def _l2_fields(l2) -> dict:
    """qw_query_params fields of query()'s ``l2`` argument: None / "off", "model",
    or an int 0..1000 (permille of the set-aside for the index window)."""
    if l2 is None or l2 == "off":
        return {"l2_mode": QW_L2_OFF, "l2_index_permille": 0}
    if l2 == "model":
        return {"l2_mode": QW_L2_MODEL, "l2_index_permille": 0}
    if isinstance(l2, int) and not isinstance(l2, bool):
        return {"l2_mode": QW_L2_SPLIT, "l2_index_permille": int(l2)}
    raise ValueError("l2 must be None, 'off', 'model' or a permille 0..1000")


def qw_hash(V: int, nv: int, d: int, A: int, b: int, m: int, w: float, H: int, stream: int = 0):
    """Device pointers in, returns the number of FP64 recomputations."""
    fix = C.c_int64(0)
    _check(load().qw_hash(V, nv, d, A, b, m, w, H, C.byref(fix), stream or None))
    return int(fix.value)


def qw_hash_tc(V: int, nv: int, d: int, A: int, b: int, m: int, w: float, H: int,
               stream: int = 0):
    """qw_hash on the tensor cores; returns the number of FP64 recomputations."""
    fix = C.c_int64(0)
    _check(load().qw_hash_tc(V, nv, d, A, b, m, w, H, C.byref(fix), stream or None))
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


def qw_draw_projections(seed: int, m: int, d: int, w: float):
    """The hash family's draws from a seed (host): returns numpy (A m x d, b m)
    float32."""
    import numpy as np
    A = np.empty((m, d), np.float32)
    b = np.empty(m, np.float32)
    load().qw_draw_projections(int(seed), int(m), int(d), float(w), A.ctypes.data, b.ctypes.data)
    return A, b


def qw_index_get_projections(index: int, m: int, d: int):
    """(A m x d, b m, offsets m) of an index as numpy arrays."""
    import numpy as np
    A = np.empty((m, d), np.float32)
    b = np.empty(m, np.float32)
    o = np.empty(m, np.int32)
    _check(load().qw_index_get_projections(index, A.ctypes.data, b.ctypes.data, o.ctypes.data))
    return A, b, o


def qw_measure_read_bandwidth(nbytes: int, reps: int = 20, stream: int = 0) -> float:
    """Best read rate (GB/s) of a device buffer of nbytes (L2 below its size,
    HBM above)."""
    g = C.c_double(0.0)
    _check(load().qw_measure_read_bandwidth(int(nbytes), int(reps), C.byref(g), stream or None))
    return float(g.value)


def qw_index_free(index: int):
    if index:
        load().qw_index_free(index)


# ---------------------------------------------------------------- torch helpers
def _torch():
    import torch
    return torch


def _params_kwargs(p) -> dict:
    """query() keyword arguments of a qw_query_params."""
    inv = lambda d, v: next(k for k, x in d.items() if x == v)  # noqa: E731
    return {"batch": int(p.batch), "path": inv(PATHS, p.path), "order": inv(ORDERS, p.order),
            "rerank": inv(RERANKS, p.rerank), "start": inv(STARTS, p.start),
            "graph": bool(p.graph), "loads": inv(LOADS, p.bitmap_loads),
            "l2": (None if p.l2_mode == QW_L2_OFF else "model" if p.l2_mode == QW_L2_MODEL
                   else int(p.l2_index_permille)),
            "projection": inv(PROJECTIONS, p.projection), "rerank_rows": int(p.rerank_rows),
            "tiles_per_warp": int(p.tiles_per_warp), "probes": int(p.probes)}


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


def hash(V, A, b, w: float, tensor_cores: bool = False):
    """Bucket ids floor((A V^T + b) / w) of CUDA float32 tensors (tensor_cores:
    qw_hash_tc).  Returns (H int32 nv x m on V's device, number of FP64
    recomputations)."""
    torch = _torch()
    _f32(V, "V"), _f32(A, "A"), _f32(b, "b")
    if not (V.is_cuda and A.is_cuda and b.is_cuda):
        raise ValueError("hash() takes CUDA tensors")
    nv, d = V.shape
    m = A.shape[0]
    H = torch.empty((nv, m), dtype=torch.int32, device=V.device)
    fn = qw_hash_tc if tensor_cores else qw_hash
    fix = fn(V.data_ptr(), nv, d, A.data_ptr(), b.data_ptr(), m, float(w), H.data_ptr(),
             _stream_of(V))
    return H, fix


class Index:
    """An LSH index over ``data`` (n x d float32), owning device memory.

    ``A`` (m x d) and ``b`` (m) are the hash family's random draws (Section 3),
    passed in so callers control the seed.  ``l = 0`` derives the collision
    threshold from Eq. 1 (see ``qw_collision_threshold``).  ``family="qalsh"``
    builds QALSH's query-aware buckets instead (Section 2; ``b`` is then not
    used, and queries run on the level path)."""

    def __init__(self, data, A=None, b=None, *, w: float, c: int = 2, v: int = 100, l: int = 0,
                 delta: float = 0.0, shadow_bf16: bool = False, bitmaps: bool = False,
                 host_bitmaps: bool = False, m: int = 0, seed: int = 0,
                 projection: str = "fp32", family: str = "e2lsh"):
        _f32(data, "data")
        n, d = data.shape
        if A is None and b is None:
            # drawn by the library from the seed (qw_draw_projections)
            if m < 1:
                raise ValueError("give A and b, or m (and seed) to draw them")
            mem = _mem_of(data)
            a_ptr = b_ptr = 0
        else:
            _f32(A, "A"), _f32(b, "b")
            mem = _mem_of(data, A, b)
            m, d2 = A.shape
            if d2 != d or b.shape != (m,):
                raise ValueError("shape mismatch between data, A and b")
            a_ptr, b_ptr = A.data_ptr(), b.data_ptr()
        p = qw_index_params(m=m, w=float(w), c=int(c), v=int(v), l=int(l), delta=float(delta),
                            shadow_bf16=1 if shadow_bf16 else 0, bitmaps=1 if bitmaps else 0,
                            host_bitmaps=1 if host_bitmaps else 0, seed=int(seed),
                            projection=PROJECTIONS[projection], family=FAMILIES[family])
        self._h = 0
        self._h = qw_build_index(data.data_ptr(), n, d, a_ptr or None, b_ptr or None, p, mem,
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
                "queries": int(p.queries), "rerank_candidates": int(p.rerank_candidates),
                "rerank_fp32_rows": int(p.rerank_fp32_rows),
                "start_levels_skipped": int(p.start_levels_skipped),
                "start_fallbacks": int(p.start_fallbacks),
                "level_passes": int(p.level_passes),
                "bitmap_fallbacks": int(p.bitmap_fallbacks),
                "bitmap_live_items": int(p.bitmap_live_items),
                "bitmap_live_groups": int(p.bitmap_live_groups),
                "bitmap_live_words": int(p.bitmap_live_words),
                "l2_setaside_bytes": int(p.l2_setaside_bytes),
                "l2_index_permille": int(p.l2_index_permille),
                "bitmap_overflows": int(p.bitmap_overflows)}

    def query(self, Q, k: int, *, batch: int = 0, stats: bool = False, out=None,
              profile: bool = False, path: str = "auto", clusters: int = 0,
              order: str = "auto", rerank: str = "fp32", start: str = "plain",
              graph: bool = False, loads: str = "tma", l2=None, projection: str = "fp32",
              rerank_rows: int = 0, tiles_per_warp: int = 0, probes: int = 0):
        """Top-k of every query row.  Returns (ids int64 nq x k, dists float32
        nq x k[, stats int64 nq x QW_NSTAT]) on Q's device (host tensors in,
        host tensors out).  ``out`` may give preallocated (ids, dists[, stats]).
        ``l2``: persisting-L2 split (None / "off", "model", or the index
        window's permille of the set-aside); speed only."""
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
                             clusters=int(clusters), order=ORDERS[order], rerank=RERANKS[rerank],
                             start=STARTS[start], graph=1 if graph else 0,
                             bitmap_loads=LOADS[loads], projection=PROJECTIONS[projection],
                             rerank_rows=int(rerank_rows), tiles_per_warp=int(tiles_per_warp),
                             probes=int(probes), **_l2_fields(l2))
        qw_run_workload(self._h, Q.data_ptr(), nq, int(k), qp, ids.data_ptr(), dists.data_ptr(),
                        st.data_ptr() if st is not None else 0, mem, _stream_of(Q))
        return (ids, dists, st) if stats else (ids, dists)

    def candidates(self, Q, k: int, *, batch: int = 0, path: str = "auto", order: str = "auto",
                   graph: bool = False, loads: str = "tma", probes: int = 0):
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
        qp = qw_query_params(batch=int(batch), path=PATHS[path], order=ORDERS[order],
                             graph=1 if graph else 0, bitmap_loads=LOADS[loads],
                             probes=int(probes))
        qw_workload_candidates(self._h, Q.data_ptr(), nq, int(k), qp, cid.data_ptr(),
                               ccol.data_ptr(), st.data_ptr(), mem, _stream_of(Q))
        return cid, ccol, st

    def features(self, Q):
        """Start-model features of CUDA float32 queries (nq x (d + m))."""
        torch = _torch()
        _f32(Q, "Q")
        F = torch.empty((Q.shape[0], self.d + self.m), dtype=torch.float32, device=Q.device)
        _check(load().qw_query_features(self._h, Q.data_ptr(), Q.shape[0], F.data_ptr(),
                                        _stream_of(Q) or None))
        return F

    def set_start_model(self, mlp, eps: float = 0.02):
        """Attach a trained Mlp (kept alive by this index) for start='learned'."""
        _check(load().qw_index_set_start_model(self._h, mlp.handle if mlp else None, float(eps)))
        self._start_model = mlp

    def autotune(self, Q, k: int, *, reps: int = 3):
        """Time the workload Q under the candidate settings (qw_autotune) and keep
        the fastest for path='auto' / batch=0.  Returns (best settings as
        query() keyword arguments, [(settings, median ms), ...] of every trial)."""
        _f32(Q, "Q")
        mem = _mem_of(Q)
        best = qw_query_params()
        rep = qw_tune_report()
        _check(load().qw_autotune(self._h, Q.data_ptr(), Q.shape[0], int(k), mem, int(reps), None,
                                  C.byref(best), C.byref(rep), _stream_of(Q) or None))
        trials = [(_params_kwargs(rep.params[i]), float(rep.ms[i])) for i in range(rep.tried)]
        return _params_kwargs(best), trials

    def projections(self):
        """(A m x d, b m, offsets m) numpy copies: the projections the index
        hashes with and its anchors."""
        return qw_index_get_projections(self._h, self.m, self.d)

    def export(self):
        """Host numpy copies: o (m), span (m), entry_bid and entry_id (m x n),
        entries of each projection ordered by (id tile, bid, bank-spread order)."""
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


class Mlp:
    """The learned start model: n_in -> hidden -> hidden -> classes (ReLU),
    softmax cross-entropy, FP16 weights over FP32 masters, Adam; every kernel
    is the library's."""

    def __init__(self, n_in: int, hidden: int, classes: int):
        h = C.c_void_p()
        _check(load().qw_mlp_create(n_in, hidden, classes, C.byref(h)))
        self._h = int(h.value)
        self.n_in, self.hidden, self.classes = n_in, hidden, classes
        self.count = int(load().qw_mlp_param_count(self._h))

    @property
    def handle(self) -> int:
        return self._h

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.count:
            raise ValueError("parameter count mismatch")
        _check(load().qw_mlp_set_params(self._h, p.ctypes.data, p.size))

    def get_params(self):
        import numpy as np
        p = np.empty(self.count, np.float32)
        _check(load().qw_mlp_get_params(self._h, p.ctypes.data, p.size))
        return p

    def loss_grad(self, X, y):
        """Mean loss and flat gradient (numpy) for CUDA X (float32) and y (int32)."""
        import numpy as np
        g = np.empty(self.count, np.float32)
        loss = C.c_float(0.0)
        _check(load().qw_mlp_loss_grad(self._h, X.data_ptr(), y.data_ptr(), X.shape[0],
                                       C.byref(loss), g.ctypes.data, _stream_of(X) or None))
        return float(loss.value), g

    def train(self, X, y, *, epochs: int, batch: int = 1024, lr: float = 1e-3) -> float:
        loss = C.c_float(0.0)
        _check(load().qw_mlp_train(self._h, X.data_ptr(), y.data_ptr(), X.shape[0], epochs, batch,
                                   lr, C.byref(loss), _stream_of(X) or None))
        return float(loss.value)

    def predict(self, X, tensor_cores: bool = False):
        """Class probabilities of CUDA float32 rows X; tensor_cores: the
        tcgen05 forward pass (qw_mlp_predict_tc), else the SIMT one."""
        torch = _torch()
        _f32(X, "X")
        P = torch.empty((X.shape[0], self.classes), dtype=torch.float32, device=X.device)
        fn = load().qw_mlp_predict_tc if tensor_cores else load().qw_mlp_predict
        _check(fn(self._h, X.data_ptr(), X.shape[0], P.data_ptr(), _stream_of(X) or None))
        return P

    def free(self):
        if self._h:
            load().qw_mlp_free(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mlp_init(n_in: int, hidden: int, classes: int, seed: int = 0):
    """He-normal initial weights, zero biases (seeded numpy draws, flat)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((hidden, n_in), (hidden, hidden), (classes, hidden)):
        parts.append((rng.standard_normal((fan_out, fan_in)) * np.sqrt(2.0 / fan_in)).ravel())
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def collision_probability(r: float, w: float) -> float:
    """Eq. 1 in closed form (library implementation)."""
    return qw_collision_probability(r, w)


def collision_threshold(m: int, w: float, c: int, n: int, v: int, delta: float = 0.0) -> int:
    return qw_collision_threshold(m, w, c, n, v, delta)


__all__ = ["Index", "Mlp", "mlp_init", "hash", "load", "QwError", "collision_probability", "collision_threshold",
           "STAT_FIELDS", "EXPORTED"] + [n for n in EXPORTED]
