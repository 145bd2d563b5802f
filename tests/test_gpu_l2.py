"""Persisting-L2 windows (the workload cache split of Section 4 on the GPU's
L2): every split gives the oracle's results, the split in use is reported,
the call leaves the stream's window as it found it, and freeing the index
puts back the context's set-aside."""
import ctypes as C
import functools

import numpy as np
import pytest

import workloads
from test_gpu_parity import TILE, _check_candidates, _check_results

pytestmark = pytest.mark.gpu

CUDA_LIMIT_PERSISTING_L2 = 0x06        # cudaLimitPersistingL2CacheSize
CUDA_STREAM_ATTR_ACCESS_POLICY = 1     # cudaStreamAttributeAccessPolicyWindow


@functools.lru_cache(maxsize=None)
def _cudart():
    for name in ("libcudart.so", "libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return C.CDLL(name)
        except OSError:
            continue
    return None


def _limit():
    rt = _cudart()
    if rt is None:
        return None
    v = C.c_size_t(0)
    assert rt.cudaDeviceGetLimit(C.byref(v), CUDA_LIMIT_PERSISTING_L2) == 0
    return int(v.value)


def _stream_window_bytes(stream_ptr):
    """num_bytes of the stream's access-policy window (0: none)."""
    rt = _cudart()
    if rt is None:
        return None
    buf = (C.c_uint8 * 64)()  # cudaStreamAttrValue (a union, at most 64 bytes)
    assert rt.cudaStreamGetAttribute(C.c_void_p(stream_ptr), CUDA_STREAM_ATTR_ACCESS_POLICY,
                                     C.byref(buf)) == 0
    return int(np.frombuffer(bytes(buf[8:16]), dtype=np.uint64)[0])


@functools.lru_cache(maxsize=None)
def _case():
    import oracle
    orc = oracle.get()
    wl = workloads.make_workload("mix10k_d32", seed=23, n=2 * TILE + 901, nq=48, n_clusters=60)
    s = wl.spec
    l = orc.threshold(s.m, s.w, s.c, s.n, s.v)
    H = orc.hash(wl.X, wl.A, wl.b, s.w)
    HQ = orc.hash(wl.Q, wl.A, wl.b, s.w)
    ref = orc.query(wl.X, orc.build_index(H), wl.Q, HQ, k=s.k, v=s.v, l=l, c=s.c)
    return wl, l, ref


@pytest.mark.parametrize("path,graph,loads", [("levels", False, "tma"), ("levels", True, "tma"),
                                              ("bitmap", False, "direct"),
                                              ("bitmap", True, "direct"),
                                              ("bitmap", True, "tma")])
def test_every_split_gives_the_oracle_results(qwlib, cuda, path, graph, loads):
    import torch
    wl, l, ref = _case()
    s = wl.spec
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)  # noqa: E731
    X, Q, A, b = t(wl.X), t(wl.Q), t(wl.A), t(wl.b)
    index = qwlib.Index(X, A, b, w=s.w, c=s.c, v=s.v, l=l, bitmaps=(path == "bitmap"))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        limit0 = _limit()
        for l2 in (None, "model", 0, 10, 500, 990, 1000, "model"):
            index.profile(reset=True)
            ids, dists, st = index.query(Q, s.k, stats=True, path=path, graph=graph,
                                         loads=loads, l2=l2, batch=20)
            cid, ccol, _ = index.candidates(Q, s.k, path=path, graph=graph, loads=loads,
                                            batch=20)
            stream.synchronize()
            _check_results(ids.cpu().numpy(), dists.cpu().numpy(), ref["ids"], ref["dists"])
            assert np.array_equal(st.cpu().numpy(), ref["stats"])
            _check_candidates(cid.cpu().numpy(), ccol.cpu().numpy(), ref["cand_ids"],
                              ref["cand_col"])
            prof = index.profile()
            if isinstance(l2, int) and prof["l2_setaside_bytes"] > 0:
                assert prof["l2_index_permille"] == l2
            if l2 is not None:
                assert prof["l2_setaside_bytes"] >= 0
                assert 0 <= prof["l2_index_permille"] <= 1000
            # the stream's window does not outlive the call
            if limit0 is not None:
                assert _stream_window_bytes(stream.cuda_stream) == 0
    index.free()
    # the set-aside the index raised is put back when it is freed
    if limit0 is not None:
        assert _limit() == limit0


def test_windows_are_attached_on_this_device(qwlib, cuda):
    """GB300 has a persisting-L2 set-aside: a window mode reports a non-zero
    set-aside and, for QW_L2_MODEL, the cost model's split."""
    import torch
    wl, l, _ = _case()
    s = wl.spec
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)  # noqa: E731
    index = qwlib.Index(t(wl.X), t(wl.A), t(wl.b), w=s.w, c=s.c, v=s.v, l=l, bitmaps=True)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        index.query(t(wl.Q), s.k, path="bitmap", loads="direct", l2=250)
        stream.synchronize()
        p = index.profile()
        assert p["l2_setaside_bytes"] > 0
        assert p["l2_index_permille"] == 250
        index.query(t(wl.Q), s.k, path="bitmap", loads="direct", l2="model")
        stream.synchronize()
        p = index.profile()
        assert p["l2_setaside_bytes"] > 0
        assert 0 <= p["l2_index_permille"] <= 1000
    index.free()


def test_bad_split_arguments_rejected(qwlib, cuda):
    import torch
    wl, l, _ = _case()
    s = wl.spec
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)  # noqa: E731
    index = qwlib.Index(t(wl.X), t(wl.A), t(wl.b), w=s.w, c=s.c, v=s.v, l=l)
    L = qwlib.load()
    ids = torch.empty((4, s.k), dtype=torch.int64, device=cuda)
    dists = torch.empty((4, s.k), dtype=torch.float32, device=cuda)
    Q = t(wl.Q[:4])
    for mode, pm in ((3, 0), (-1, 0), (qwlib.QW_L2_SPLIT, 1001), (qwlib.QW_L2_SPLIT, -5)):
        qp = qwlib.qw_query_params(l2_mode=mode, l2_index_permille=pm)
        assert L.qw_run_workload(index.handle, Q.data_ptr(), 4, s.k, C.byref(qp), ids.data_ptr(),
                                 dists.data_ptr(), None, 0, None) == qwlib.QW_ERR_ARG
    index.free()
