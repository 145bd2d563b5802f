"""CPU oracle for the LSH query-workload path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, sequential FP64 C implementation (``qwlsh_oracle.c``) of the
index and query procedure of the paper (arXiv 1907.11803, Sections 2, 3, 3.1,
4, Eq. 1), wrapped with ctypes.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package; the CUDA
library shares no code with it and never calls it.

Every function here is argument marshalling around the C code; the arithmetic
is all in ``qwlsh_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "qwlsh_oracle.c")
BUILD_DIR = os.path.join(_HERE, "_build")
NSTAT = 8
CFLAGS = ["-O3", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]

_lock = threading.Lock()


class OracleError(RuntimeError):
    pass


def compile_oracle(source: str = SOURCE, out: Optional[str] = None, extra_flags=()) -> str:
    """Compile the oracle C file into a shared object; returns its path."""
    out = out or os.path.join(BUILD_DIR, "liboracle.so")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", *CFLAGS, *extra_flags, "-o", out, source, "-lm"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise OracleError("oracle compile failed:\n" + res.stderr)
    return out


_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def _opt(ptype):
    """ndpointer that also accepts None."""

    class _Opt(ptype):  # type: ignore[misc, valid-type]
        @classmethod
        def from_param(cls, obj):
            if obj is None:
                return None
            return ptype.from_param(obj)

    return _Opt


@dataclass
class OracleIndex:
    H: np.ndarray       # n x m int32 bucket ids of the data
    o: np.ndarray       # m int32 anchors (min bucket id per projection)
    span: np.ndarray    # m int32 max anchored bucket id per projection
    sbid: Optional[np.ndarray]  # m x n int32 sorted bucket ids
    sid: Optional[np.ndarray]   # m x n int32 ids in the same order


class Oracle:
    """ctypes front-end for one compiled copy of the oracle."""

    def __init__(self, lib_path: Optional[str] = None):
        if lib_path is None:
            with _lock:
                lib_path = os.path.join(BUILD_DIR, "liboracle.so")
                if (not os.path.exists(lib_path)
                        or os.path.getmtime(lib_path) < os.path.getmtime(SOURCE)):
                    compile_oracle(out=lib_path)
        self.path = lib_path
        L = C.CDLL(lib_path)
        L.orc_collision_prob.restype = C.c_double
        L.orc_collision_prob.argtypes = [C.c_double, C.c_double]
        L.orc_alpha.restype = C.c_double
        L.orc_alpha.argtypes = [C.c_double] * 4
        L.orc_qalsh_threshold.restype = C.c_int32
        L.orc_qalsh_threshold.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_int64,
                                          C.c_int32, C.c_double]
        L.orc_threshold.restype = C.c_int32
        L.orc_threshold.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_int64, C.c_int32,
                                    C.c_double]
        L.orc_hash.restype = C.c_int
        L.orc_hash.argtypes = [_f32p, C.c_int64, C.c_int32, _f32p, _f32p, C.c_int32, C.c_float,
                               _i32p]
        L.orc_build_index.restype = C.c_int
        L.orc_build_index.argtypes = [_i32p, C.c_int64, C.c_int32, _i32p, _i32p,
                                      _opt(_i32p), _opt(_i32p)]
        L.orc_collision_counts.restype = None
        L.orc_collision_counts.argtypes = [_i32p, C.c_int64, C.c_int32, _i32p, _i32p,
                                           C.c_int64, _i32p]
        L.orc_range_count.restype = C.c_int64
        L.orc_range_count.argtypes = [_i32p, C.c_int64, C.c_int64, C.c_int64]
        L.orc_sqdist.restype = C.c_double
        L.orc_sqdist.argtypes = [_f32p, _f32p, C.c_int32]
        L.orc_collision_counts_probes.restype = None
        L.orc_collision_counts_probes.argtypes = [_i32p, C.c_int64, C.c_int32, _i32p, _i32p,
                                                  C.c_int64, C.c_int32, _i32p]
        L.orc_query_probes.restype = C.c_int
        L.orc_query_probes.argtypes = [_f32p, C.c_int64, C.c_int32, _i32p, _i32p, _i32p,
                                       C.c_int32, _opt(_i32p), _f32p, _i32p, C.c_int64,
                                       C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                       _i64p, _f64p, _opt(_i64p), _opt(_i32p), _opt(_i64p)]
        L.orc_project.restype = C.c_int
        L.orc_project.argtypes = [_f32p, C.c_int64, C.c_int32, _f32p, C.c_int32, _f64p]
        L.orc_qalsh_counts.restype = None
        L.orc_qalsh_counts.argtypes = [_f64p, C.c_int64, C.c_int32, _f64p, C.c_double, C.c_int64,
                                       _i32p]
        L.orc_qalsh_query.restype = C.c_int
        L.orc_qalsh_query.argtypes = [_f32p, C.c_int64, C.c_int32, _f64p, C.c_int32, _f32p, _f64p,
                                      C.c_int64, C.c_double, C.c_int32, C.c_int32, C.c_int32,
                                      C.c_int32, _i64p, _f64p, _opt(_i64p), _opt(_i32p),
                                      _opt(_i64p)]
        L.orc_qalsh_prob.restype = C.c_double
        L.orc_qalsh_prob.argtypes = [C.c_double, C.c_double]
        L.orc_query.restype = C.c_int
        L.orc_query.argtypes = [_f32p, C.c_int64, C.c_int32, _i32p, _i32p, _i32p, C.c_int32,
                                _opt(_i32p), _f32p, _i32p, C.c_int64, C.c_int32, C.c_int32,
                                C.c_int32, C.c_int32, _i64p, _f64p, _opt(_i64p), _opt(_i32p),
                                _opt(_i64p)]
        L.orc_bruteforce.restype = C.c_int
        L.orc_bruteforce.argtypes = [_f32p, C.c_int64, C.c_int32, _f32p, C.c_int64, C.c_int32,
                                     _i64p, _f64p]
        self.lib = L

    # -- Eq. 1 and the threshold ------------------------------------------
    def collision_prob(self, r: float, w: float) -> float:
        return float(self.lib.orc_collision_prob(r, w))

    def alpha(self, p1: float, p2: float, beta: float, delta: float) -> float:
        return float(self.lib.orc_alpha(p1, p2, beta, delta))

    def threshold(self, m: int, w: float, c: float, n: int, v: int,
                  delta: float = float(np.exp(-1.0))) -> int:
        return int(self.lib.orc_threshold(m, w, c, n, v, delta))

    def qalsh_threshold(self, m: int, w: float, c: float, n: int, v: int,
                        delta: float = float(np.exp(-1.0))) -> int:
        return int(self.lib.orc_qalsh_threshold(m, w, c, n, v, delta))

    # -- hashing and index -------------------------------------------------
    def hash(self, V: np.ndarray, A: np.ndarray, b: np.ndarray, w: float) -> np.ndarray:
        V = np.ascontiguousarray(V, np.float32)
        A = np.ascontiguousarray(A, np.float32)
        b = np.ascontiguousarray(b, np.float32)
        nv, d = V.shape
        m = A.shape[0]
        H = np.empty((nv, m), np.int32)
        st = self.lib.orc_hash(V, nv, d, A, b, m, float(w), H)
        if st != 0:
            raise OracleError(f"orc_hash status {st}")
        return H

    def build_index(self, H: np.ndarray, sorted_arrays: bool = True) -> OracleIndex:
        H = np.ascontiguousarray(H, np.int32)
        n, m = H.shape
        o = np.empty(m, np.int32)
        span = np.empty(m, np.int32)
        sbid = np.empty((m, n), np.int32) if sorted_arrays else None
        sid = np.empty((m, n), np.int32) if sorted_arrays else None
        st = self.lib.orc_build_index(H, n, m, o, span, sbid, sid)
        if st != 0:
            raise OracleError(f"orc_build_index status {st}")
        return OracleIndex(H=H, o=o, span=span, sbid=sbid, sid=sid)

    def collision_counts(self, index: OracleIndex, hq: np.ndarray, R: int,
                         probes: int = 0) -> np.ndarray:
        n, m = index.H.shape
        col = np.empty(n, np.int32)
        hq = np.ascontiguousarray(hq, np.int32)
        if probes:
            self.lib.orc_collision_counts_probes(index.H, n, m, index.o, hq, int(R), int(probes),
                                                 col)
        else:
            self.lib.orc_collision_counts(index.H, n, m, index.o, hq, int(R), col)
        return col

    def range_count(self, index: OracleIndex, i: int, lo: int, hi: int) -> int:
        n = index.H.shape[0]
        row = np.ascontiguousarray(index.sbid[i])
        return int(self.lib.orc_range_count(row, n, int(lo), int(hi)))

    def sqdist(self, x: np.ndarray, q: np.ndarray) -> float:
        x = np.ascontiguousarray(x, np.float32)
        q = np.ascontiguousarray(q, np.float32)
        return float(self.lib.orc_sqdist(x, q, x.shape[0]))

    # -- the query workload ------------------------------------------------
    def query(self, X: np.ndarray, index: OracleIndex, Q: np.ndarray, HQ: np.ndarray, *,
              k: int, v: int, l: int, c: int = 2, want_candidates: bool = True,
              want_stats: bool = True, probes: int = 0):
        X = np.ascontiguousarray(X, np.float32)
        Q = np.ascontiguousarray(Q, np.float32)
        HQ = np.ascontiguousarray(HQ, np.int32)
        n, d = X.shape
        nq = Q.shape[0]
        m = index.H.shape[1]
        cap = k + v
        ids = np.empty((nq, k), np.int64)
        dists = np.empty((nq, k), np.float64)
        cids = np.empty((nq, cap), np.int64) if want_candidates else None
        ccol = np.empty((nq, cap), np.int32) if want_candidates else None
        stats = np.empty((nq, NSTAT), np.int64) if want_stats else None
        if probes:
            st = self.lib.orc_query_probes(X, n, d, index.H, index.o, index.span, m, index.sbid,
                                           Q, HQ, nq, k, v, l, c, int(probes), ids, dists, cids,
                                           ccol, stats)
        else:
            st = self.lib.orc_query(X, n, d, index.H, index.o, index.span, m, index.sbid, Q, HQ,
                                    nq, k, v, l, c, ids, dists, cids, ccol, stats)
        if st != 0:
            raise OracleError(f"orc_query status {st}")
        out = {"ids": ids, "dists": dists}
        if want_candidates:
            out["cand_ids"] = cids
            out["cand_col"] = ccol
        if want_stats:
            out["stats"] = stats
        return out

    # -- QALSH's query-aware buckets (reading R17) ---------------------------
    def project(self, V: np.ndarray, A: np.ndarray) -> np.ndarray:
        """a_i . v in double (nv x m), summed in coordinate order."""
        V = np.ascontiguousarray(V, np.float32)
        A = np.ascontiguousarray(A, np.float32)
        P = np.empty((V.shape[0], A.shape[0]), np.float64)
        st = self.lib.orc_project(V, V.shape[0], V.shape[1], A, A.shape[0], P)
        if st != 0:
            raise OracleError(f"orc_project status {st}")
        return P

    def qalsh_counts(self, P: np.ndarray, pq: np.ndarray, w: float, R: int) -> np.ndarray:
        P = np.ascontiguousarray(P, np.float64)
        col = np.empty(P.shape[0], np.int32)
        self.lib.orc_qalsh_counts(P, P.shape[0], P.shape[1],
                                  np.ascontiguousarray(pq, np.float64), float(w), int(R), col)
        return col

    def qalsh_prob(self, r: float, w: float) -> float:
        return float(self.lib.orc_qalsh_prob(r, w))

    def qalsh_query(self, X: np.ndarray, P: np.ndarray, Q: np.ndarray, PQ: np.ndarray, *,
                    w: float, k: int, v: int, l: int, c: int = 2):
        X = np.ascontiguousarray(X, np.float32)
        Q = np.ascontiguousarray(Q, np.float32)
        P = np.ascontiguousarray(P, np.float64)
        PQ = np.ascontiguousarray(PQ, np.float64)
        n, d = X.shape
        nq, m = PQ.shape
        cap = k + v
        ids = np.empty((nq, k), np.int64)
        dists = np.empty((nq, k), np.float64)
        cids = np.empty((nq, cap), np.int64)
        ccol = np.empty((nq, cap), np.int32)
        stats = np.empty((nq, NSTAT), np.int64)
        st = self.lib.orc_qalsh_query(X, n, d, P, m, Q, PQ, nq, float(w), k, v, l, c, ids, dists,
                                      cids, ccol, stats)
        if st != 0:
            raise OracleError(f"orc_qalsh_query status {st}")
        return {"ids": ids, "dists": dists, "cand_ids": cids, "cand_col": ccol, "stats": stats}

    def bruteforce(self, X: np.ndarray, Q: np.ndarray, k: int):
        X = np.ascontiguousarray(X, np.float32)
        Q = np.ascontiguousarray(Q, np.float32)
        ids = np.empty((Q.shape[0], k), np.int64)
        dists = np.empty((Q.shape[0], k), np.float64)
        st = self.lib.orc_bruteforce(X, X.shape[0], X.shape[1], Q, Q.shape[0], k, ids, dists)
        if st != 0:
            raise OracleError(f"orc_bruteforce status {st}")
        return ids, dists


_default: Optional[Oracle] = None


def get() -> Oracle:
    """The oracle compiled from this directory's source (built on first use)."""
    global _default
    if _default is None:
        _default = Oracle()
    return _default


STAT_FIELDS = ("levels", "final_R", "n_cand_raw", "n_cand", "term", "scanned_last",
               "scanned_full", "n_prev")
