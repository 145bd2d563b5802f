"""qw_run_workload_noalloc: the query path for callers that cannot allocate
device memory at query time (for example a process whose device memory is
already reserved by another framework's allocator, or a latency-critical
thread that must not call cudaMalloc / cudaFree).  It runs on the library's
static device scratch instead of allocating.

Checked here through the C ABI against qw_run_workload, on two calls in a
row: ids identical, distances within the 1e-5 relative tolerance the other
parity tests use, statistics identical.  The index has three tiles and the
workload needs several scratch-sized batches (the last one ragged).
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

DIST_RTOL = 1e-5


def _call_noalloc(qw, index, Q, k):
    import torch
    nq = Q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int64, device=Q.device)
    dists = torch.empty((nq, k), dtype=torch.float32, device=Q.device)
    st = torch.empty((nq, qw.QW_NSTAT), dtype=torch.int64, device=Q.device)
    stream = int(torch.cuda.current_stream(Q.device).cuda_stream)
    qw.qw_run_workload_noalloc(index.handle, Q.data_ptr(), nq, k, ids.data_ptr(), dists.data_ptr(),
                               st.data_ptr(), stream)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dists.cpu().numpy(), st.cpu().numpy()


def _check_same(got, want):
    ids, dists, st = got
    wids, wd, wst = want
    assert np.array_equal(ids, wids)
    fin = np.isfinite(wd)
    assert np.array_equal(fin, np.isfinite(dists))
    rel = np.abs(dists[fin].astype(np.float64) - wd[fin]) / np.maximum(wd[fin].astype(np.float64), 1e-30)
    assert rel.size == 0 or rel.max() <= DIST_RTOL
    assert np.array_equal(st, wst)


def test_noalloc_matches_run_workload_twice(qwlib, cuda):
    import torch
    n = 2 * 32768 + 500
    wl1 = workloads.make_workload("mix10k_d32", seed=21, n=n, nq=1500, d=24, m=12, n_clusters=40)
    wl2 = workloads.make_workload("mix10k_d32", seed=22, n=n, nq=900, d=24, m=12, n_clusters=40)
    X = torch.from_numpy(wl1.X).to(cuda)
    A = torch.from_numpy(wl1.A).to(cuda)
    b = torch.from_numpy(wl1.b).to(cuda)
    index = qwlib.Index(X, A, b, w=4.0, v=30)
    k = 9
    for Qn in (wl1.Q, wl2.Q):
        Q = torch.from_numpy(Qn).to(cuda)
        ids, dists, st = index.query(Q, k, stats=True, path="levels")
        torch.cuda.synchronize()
        want = (ids.cpu().numpy(), dists.cpu().numpy(), st.cpu().numpy())
        got = _call_noalloc(qwlib, index, Q, k)
        _check_same(got, want)
    index.free()


def test_noalloc_arguments_empty_workload_and_no_stats(qwlib, cuda):
    """Bad arguments are refused with QW_ERR_ARG and a message naming the
    entry point; an empty workload is a no-op; without the statistics output
    the results are those of the call with it."""
    import torch
    wl = workloads.make_workload("mix10k_d32", seed=23, n=5000, nq=200, d=16, m=8, n_clusters=10)
    index = qwlib.Index(torch.from_numpy(wl.X).to(cuda), torch.from_numpy(wl.A).to(cuda),
                        torch.from_numpy(wl.b).to(cuda), w=4.0, v=30)
    Q = torch.from_numpy(wl.Q).to(cuda)
    lib = qwlib.load()
    stream = int(torch.cuda.current_stream(cuda).cuda_stream)
    ids = torch.empty((200, 4096), dtype=torch.int64, device=cuda)
    dists = torch.empty((200, 4096), dtype=torch.float32, device=cuda)
    for k, i_ptr, q_ptr in ((4090, ids.data_ptr(), Q.data_ptr()),   # k + v > 4096
                            (5001, ids.data_ptr(), Q.data_ptr()),   # k > n
                            (0, ids.data_ptr(), Q.data_ptr()),      # k < 1
                            (5, None, Q.data_ptr()),                # null ids
                            (5, ids.data_ptr(), None)):             # null queries
        st = lib.qw_run_workload_noalloc(index.handle, q_ptr, 200, k, i_ptr, dists.data_ptr(),
                                         None, stream)
        assert st == qwlib.QW_ERR_ARG
        assert b"qw_run_workload_noalloc" in lib.qw_last_error()
    assert lib.qw_run_workload_noalloc(index.handle, None, 0, 5, None, None, None, stream) == qwlib.QW_OK
    k = 7
    with_stats = _call_noalloc(qwlib, index, Q, k)
    ids2 = torch.empty((200, k), dtype=torch.int64, device=cuda)
    d2 = torch.empty((200, k), dtype=torch.float32, device=cuda)
    qwlib.qw_run_workload_noalloc(index.handle, Q.data_ptr(), 200, k, ids2.data_ptr(),
                                  d2.data_ptr(), 0, stream)
    torch.cuda.synchronize()
    assert np.array_equal(ids2.cpu().numpy(), with_stats[0])
    assert np.array_equal(d2.cpu().numpy(), with_stats[1])
    index.free()
