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
