"""QALSH's query-aware buckets (Section 2) on the GPU against the oracle,
through the C ABI: per query the statistics, the kept candidates with their
collision counts and the result ids bit-exact, distances within 1e-5
relative.  Cases: the hand-worked points (objects exactly on interval ends),
ragged tiles and batches, an integer grid where thousands of projections fall
exactly on an interval end and share values, duplicates, queries far from the
data, c = 3, v >= n, host memory, graph mode, the no-allocation entry point,
and a 1M x 128 index with 64 projections sampled query by query."""
import json
import os

import numpy as np
import pytest

import oracle_par
import workloads
from test_gpu_parity import _check_candidates, _check_results, _t

pytestmark = pytest.mark.gpu

TILE = 32768


def _w32(w):
    # the library keeps w in float32; the oracle gets the same value
    return float(np.float32(w))


def _oracle(orc, X, Q, A, *, w, k, v, l, c=2, threaded=False):
    if threaded:
        P = oracle_par.project_rows(orc, X, A)
        PQ = oracle_par.project_rows(orc, Q, A)
        return oracle_par.qalsh_query_rows(orc, X, P, Q, PQ, w=_w32(w), k=k, v=v, l=l, c=c)
    P = orc.project(X, A)
    PQ = orc.project(Q, A)
    return orc.qalsh_query(X, P, Q, PQ, w=_w32(w), k=k, v=v, l=l, c=c)


def _gpu(qw, dev, X, Q, A, *, w, k, v, l, c=2, batch=0, graph=False, host=False):
    import torch
    b = np.zeros(A.shape[0], np.float32)
    if host:
        Xd, Ad, bd, Qd = (torch.from_numpy(np.ascontiguousarray(a)) for a in (X, A, b, Q))
    else:
        Xd, Ad, bd, Qd = _t(X, dev), _t(A, dev), _t(b, dev), _t(Q, dev)
    index = qw.Index(Xd, Ad, bd, w=w, c=c, v=v, l=l, family="qalsh")
    ids, dists, st = index.query(Qd, k, batch=batch, stats=True, graph=graph)
    cid, ccol, st2 = index.candidates(Qd, k, batch=batch, graph=graph)
    torch.cuda.synchronize()
    out = dict(ids=ids.cpu().numpy(), dists=dists.cpu().numpy(), stats=st.cpu().numpy(),
               cid=cid.cpu().numpy(), ccol=ccol.cpu().numpy(), stats2=st2.cpu().numpy())
    return out, index


def _parity(orc, qw, dev, X, Q, A, *, w, k, v, l, c=2, batch=0, graph=False, host=False):
    ref = _oracle(orc, X, Q, A, w=w, k=k, v=v, l=l, c=c)
    g, index = _gpu(qw, dev, X, Q, A, w=w, k=k, v=v, l=l, c=c, batch=batch, graph=graph,
                    host=host)
    assert np.array_equal(g["stats"], ref["stats"]), "per-query statistics differ"
    assert np.array_equal(g["stats2"], ref["stats"])
    _check_candidates(g["cid"], g["ccol"], ref["cand_ids"], ref["cand_col"])
    _check_results(g["ids"], g["dists"], ref["ids"], ref["dists"])
    index.free()
    return ref


def _shifted(wl, dist):
    """Queries pushed by `dist` along every projection (far below and above
    the data)."""
    shift = np.linalg.pinv(wl.A.astype(np.float64)) @ np.full(wl.A.shape[0], dist)
    Q = wl.Q.copy()
    Q[:3] = (Q[:3] - shift).astype(np.float32)
    Q[3:5] = (Q[3:5] + shift).astype(np.float32)
    return Q


@pytest.mark.parametrize("graph", [False, True])
def test_qalsh_hand_worked(qwlib, cuda, graph):
    """The ten hand-worked points (tests/golden/hand_worked_query.json,
    section "qalsh"): statistics, kept candidates, ids and distances."""
    import torch
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "hand_worked_query.json")
    g = json.load(open(path))
    p, qa = g["params"], g["qalsh"]
    X = np.array(g["X"], np.float32)
    A = np.array(g["A"], np.float32)
    Q = np.array(qa["Q"], np.float32)
    out, index = _gpu(qwlib, cuda, X, Q, A, w=qa["w"], k=p["k"], v=p["v"], l=p["l"], c=p["c"],
                      graph=graph)
    for qi, q in enumerate(qa["queries"]):
        assert out["stats"][qi].tolist() == q["stats"], qi
        assert out["ids"][qi].tolist() == q["ids"], qi
        want = np.sqrt(np.array(q["sqdists"], np.float64))
        assert np.allclose(out["dists"][qi], want, rtol=1e-6, atol=0), qi
        kept = sorted(q["kept"])
        got = out["cid"][qi][out["cid"][qi] >= 0].tolist()
        assert got == kept, qi
        cols = dict(zip(q["kept"], q["kept_col"]))
        assert out["ccol"][qi][: len(kept)].tolist() == [cols[i] for i in kept], qi
    index.free()
    del torch


@pytest.mark.parametrize("graph,batch", [(False, 0), (True, 0), (False, 37), (True, 250)])
def test_qalsh_matches_oracle(orc, qwlib, cuda, graph, batch):
    """Three id tiles (the last ragged), queries near the data and far from it,
    several batches."""
    wl = workloads.make_workload("mix10k_d32", seed=51, n=2 * TILE + 500, nq=400, d=24, m=12,
                                 n_clusters=40)
    Q = _shifted(wl, 60.0)
    _parity(orc, qwlib, cuda, wl.X, Q, wl.A, w=2.719, k=7, v=40, l=7, graph=graph, batch=batch)


def test_qalsh_integer_grid_boundaries(orc, qwlib, cuda):
    """Integer data and projections with w = 2: every interval end p_i(q) +- R
    is an integer, so objects land exactly on interval ends and projections
    repeat across the three tiles; the ends are inside."""
    rng = np.random.default_rng(52)
    n, d, m = 2 * TILE + 777, 6, 10
    X = rng.integers(-6, 7, size=(n, d)).astype(np.float32)
    A = rng.integers(-2, 3, size=(m, d)).astype(np.float32)
    Q = np.concatenate([X[rng.choice(n, 150, replace=False)],
                        rng.integers(-9, 10, size=(50, d))]).astype(np.float32)
    ref = _parity(orc, qwlib, cuda, X, Q, A, w=2.0, k=5, v=60, l=8)
    # the case does reach interval ends: some query has an object exactly at p(q) +- R
    P, PQ = X @ A.T, Q @ A.T
    R = ref["stats"][:, 1]
    on_end = np.abs(np.abs(P[None, :200, :] - PQ[:, None, :]) - R[:, None, None]) == 0
    assert on_end.any()


def test_qalsh_duplicates_tie_by_id(orc, qwlib, cuda):
    """Each point stored four times (equal projections in different tiles):
    candidates and results tie-break by id."""
    wl = workloads.make_workload("mix10k_d32", seed=53, n=20000, nq=120, d=16, m=8,
                                 n_clusters=20)
    X = np.concatenate([wl.X] * 4)
    _parity(orc, qwlib, cuda, X, wl.Q, wl.A, w=2.719, k=9, v=50, l=5)


def test_qalsh_c3_and_single_projection(orc, qwlib, cuda):
    wl = workloads.make_workload("mix10k_d32", seed=54, n=TILE + 99, nq=150, d=12, m=9,
                                 n_clusters=15)
    _parity(orc, qwlib, cuda, wl.X, _shifted(wl, 25.0), wl.A, w=1.5, k=4, v=30, l=5, c=3)
    _parity(orc, qwlib, cuda, wl.X, wl.Q, wl.A[:1].copy(), w=2.719, k=4, v=30, l=1)


def test_qalsh_v_ge_n_is_exact_knn(orc, qwlib, cuda):
    """k + v > n: every query ends by the radius rule, keeps every object and
    returns the exact nearest neighbours."""
    wl = workloads.make_workload("mix10k_d32", seed=55, n=900, nq=60, d=10, m=6, n_clusters=8)
    ref = _parity(orc, qwlib, cuda, wl.X, _shifted(wl, 40.0), wl.A, w=2.719, k=6, v=1000, l=3)
    assert (ref["stats"][:, 4] == 3).all()
    bf_ids, _ = orc.bruteforce(wl.X, _shifted(wl, 40.0), 6)
    assert np.array_equal(ref["ids"], bf_ids)


def test_qalsh_host_memory(orc, qwlib, cuda):
    wl = workloads.make_workload("mix10k_d32", seed=56, n=5000, nq=90, d=16, m=8, n_clusters=10)
    _parity(orc, qwlib, cuda, wl.X, wl.Q, wl.A, w=2.719, k=5, v=40, l=5, host=True)


def test_qalsh_noalloc(orc, qwlib, cuda):
    """The no-allocation entry point answers a QALSH index like the oracle."""
    import torch
    wl = workloads.make_workload("mix10k_d32", seed=57, n=TILE + 1234, nq=700, d=20, m=10,
                                 n_clusters=30)
    ref = _oracle(orc, wl.X, wl.Q, wl.A, w=2.719, k=8, v=40, l=6)
    index = qwlib.Index(_t(wl.X, cuda), _t(wl.A, cuda), _t(np.zeros(10, np.float32), cuda),
                        w=2.719, v=40, l=6, family="qalsh")
    Q = _t(wl.Q, cuda)
    ids = torch.empty((700, 8), dtype=torch.int64, device=cuda)
    dists = torch.empty((700, 8), dtype=torch.float32, device=cuda)
    st = torch.empty((700, qwlib.QW_NSTAT), dtype=torch.int64, device=cuda)
    stream = int(torch.cuda.current_stream(cuda).cuda_stream)
    qwlib.qw_run_workload_noalloc(index.handle, Q.data_ptr(), 700, 8, ids.data_ptr(),
                                  dists.data_ptr(), st.data_ptr(), stream)
    torch.cuda.synchronize()
    assert np.array_equal(st.cpu().numpy(), ref["stats"])
    _check_results(ids.cpu().numpy(), dists.cpu().numpy(), ref["ids"], ref["dists"])
    index.free()


def test_qalsh_refuses_other_paths_and_options(qwlib, cuda):
    import torch
    wl = workloads.make_workload("mix10k_d32", seed=58, n=3000, nq=10, d=8, m=6, n_clusters=5)
    X, A, b = _t(wl.X, cuda), _t(wl.A, cuda), _t(wl.b, cuda)
    with pytest.raises(qwlib.QwError):
        qwlib.Index(X, A, b, w=2.719, v=20, family="qalsh", bitmaps=True)
    with pytest.raises(qwlib.QwError):
        qwlib.Index(X, A, b, w=2.719, v=20, family="qalsh", projection="tensor")
    index = qwlib.Index(X, A, b, w=2.719, v=20, family="qalsh")
    assert index.info.family == qwlib.QW_FAMILY_QALSH
    assert index.l == qwlib.qw_qalsh_collision_threshold(6, 2.719, 2, 3000, 20)
    Q = _t(wl.Q, cuda)
    for kw in ({"path": "bitmap"}, {"path": "cluster"}, {"start": "learned"}, {"probes": 1},
               {"projection": "tensor"}):
        with pytest.raises(qwlib.QwError):
            index.query(Q, 3, **kw)
    with pytest.raises(qwlib.QwError):
        index.export()
    index.free()
    del torch


def test_qalsh_full_size_sampled(orc, qwlib, cuda):
    """1,000,000 x 128 with 64 projections (w = 2.719, the experiments'
    default; k = 100, v = 700): 32 sampled queries of a 2,000-query workload
    against the oracle, the whole workload against graph mode."""
    import torch
    wl = workloads.make_workload("mix1m_d128", seed=59, nq=2000)
    X, A = wl.X, wl.A
    n, m = X.shape[0], A.shape[0]
    k, v = 100, 700
    l = qwlib.qw_qalsh_collision_threshold(m, 2.719, 2, n, v)
    index = qwlib.Index(_t(X, cuda), _t(A, cuda), _t(np.zeros(m, np.float32), cuda), w=2.719,
                        v=v, l=l, family="qalsh")
    Qd = _t(wl.Q, cuda)
    ids, dists, st = index.query(Qd, k, stats=True)
    ids2, dists2, st2 = index.query(Qd, k, stats=True, graph=True)
    torch.cuda.synchronize()
    ids, dists, st = ids.cpu().numpy(), dists.cpu().numpy(), st.cpu().numpy()
    assert np.array_equal(ids, ids2.cpu().numpy())
    assert np.array_equal(st, st2.cpu().numpy())
    sample = np.random.default_rng(0).choice(wl.Q.shape[0], 32, replace=False)
    ref = _oracle(orc, X, wl.Q[sample], A, w=2.719, k=k, v=v, l=l, threaded=True)
    assert np.array_equal(st[sample], ref["stats"])
    _check_results(ids[sample], dists[sample], ref["ids"], ref["dists"])
    index.free()
