"""The oracle's row-independent calls spread over host threads (test helper).

The oracle is plain C called through ctypes, which releases the interpreter
lock, and keeps no global state: each data row's bucket ids depend on that row
alone and each query's answer on that query alone, so slices of rows or
queries can be handed to threads and the pieces concatenated.  Nothing here
does any of the method's arithmetic.
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np


def threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def _slices(count: int, parts: int):
    return [p for p in np.array_split(np.arange(count), max(1, parts)) if p.size]


def hash_rows(orc, V, A, b, w, nthreads=None):
    parts = _slices(V.shape[0], nthreads or threads())
    with cf.ThreadPoolExecutor(max_workers=len(parts)) as ex:
        Hs = list(ex.map(lambda p: orc.hash(V[p[0]:p[-1] + 1], A, b, w), parts))
    return np.concatenate(Hs)


def query_rows(orc, X, idx, Q, HQ, *, k, v, l, c=2, nthreads=None):
    """orc.query over slices of the queries; the per-query outputs are
    concatenated in query order."""
    parts = _slices(Q.shape[0], nthreads or threads())

    def one(p):
        s, e = p[0], p[-1] + 1
        return orc.query(X, idx, Q[s:e], HQ[s:e], k=k, v=v, l=l, c=c)

    with cf.ThreadPoolExecutor(max_workers=len(parts)) as ex:
        outs = list(ex.map(one, parts))
    return {key: np.concatenate([o[key] for o in outs]) for key in outs[0]}


def project_rows(orc, V, A, nthreads=None):
    """orc.project over slices of the rows."""
    parts = _slices(V.shape[0], nthreads or threads())
    with cf.ThreadPoolExecutor(max_workers=len(parts)) as ex:
        Ps = list(ex.map(lambda p: orc.project(V[p[0]:p[-1] + 1], A), parts))
    return np.concatenate(Ps)


def qalsh_query_rows(orc, X, P, Q, PQ, *, w, k, v, l, c=2, nthreads=None):
    """orc.qalsh_query over slices of the queries, concatenated in query order."""
    parts = _slices(Q.shape[0], nthreads or threads())

    def one(p):
        s, e = p[0], p[-1] + 1
        return orc.qalsh_query(X, P, Q[s:e], PQ[s:e], w=w, k=k, v=v, l=l, c=c)

    with cf.ThreadPoolExecutor(max_workers=len(parts)) as ex:
        outs = list(ex.map(one, parts))
    return {key: np.concatenate([o[key] for o in outs]) for key in outs[0]}
