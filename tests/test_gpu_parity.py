"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Bar: bucket ids, anchors, spans, sorted arrays, levels, candidate sets with
their collision counts, statistics and result ids bit-exact; distances within
1e-5 relative (the tolerance the path is specified to).
"""
import numpy as np
import pytest

import oracle_par
import workloads

pytestmark = pytest.mark.gpu

DIST_RTOL = 1e-5
TILE = 32768
# "graph": the level path with its level loop run as a CUDA graph; "bitmap":
# counts from the index's level bitmaps staged by TMA ("bitmap_graph": the same
# in graph mode; "bitmap_direct": summary filter then counts of the live groups
# by plain loads; "bitmap_direct_graph": the same in graph mode)
PATHS = pytest.mark.parametrize("path", ["levels", "cluster", "graph", "bitmap", "bitmap_graph",
                                         "bitmap_direct", "bitmap_direct_graph", "bitmap_fused",
                                         "bitmap_fused_graph"])


def _t(x, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def _oracle_run(orc, X, Q, A, b, w, k, v, l, c=2):
    H = orc.hash(X, A, b, w)
    HQ = orc.hash(Q, A, b, w)
    idx = orc.build_index(H)
    ref = orc.query(X, idx, Q, HQ, k=k, v=v, l=l, c=c)
    return H, HQ, idx, ref


def _check_results(ids, dists, ref_ids, ref_dists):
    assert ids.shape == ref_ids.shape
    bad = np.nonzero((ids != ref_ids).any(axis=1))[0]
    assert bad.size == 0, f"ids differ on queries {bad[:10]}: gpu {ids[bad[0]]} oracle {ref_ids[bad[0]]}"
    fin = np.isfinite(ref_dists)
    assert np.array_equal(fin, np.isfinite(dists))
    rel = np.abs(dists[fin].astype(np.float64) - ref_dists[fin]) / np.maximum(ref_dists[fin], 1e-300)
    assert rel.size == 0 or rel.max() <= DIST_RTOL, f"max rel dist err {rel.max():.3g}"


def _check_candidates(cid, ccol, ref_cid, ref_ccol):
    nq = ref_cid.shape[0]
    for q in range(nq):
        keep = ref_cid[q] >= 0
        order = np.argsort(ref_cid[q][keep], kind="stable")
        want_ids = ref_cid[q][keep][order]
        want_col = ref_ccol[q][keep][order]
        got = cid[q][cid[q] >= 0]
        assert np.array_equal(got, want_ids), f"candidate set differs on query {q}"
        assert np.array_equal(ccol[q][: got.size], want_col), f"counts differ on query {q}"


def _gpu_workload(qw, dev, X, Q, A, b, *, w, k, v, l, c=2, batch=0, host=False, path="auto",
                  order="auto", rerank="fp32"):
    import torch
    if host:
        Xd, Ad, bd = (torch.from_numpy(np.ascontiguousarray(a)) for a in (X, A, b))
        Qd = torch.from_numpy(np.ascontiguousarray(Q))
    else:
        Xd, Qd, Ad, bd = _t(X, dev), _t(Q, dev), _t(A, dev), _t(b, dev)
    index = qw.Index(Xd, Ad, bd, w=w, c=c, v=v, l=l, shadow_bf16=rerank in ("bf16", "bf16_tc"),
                     bitmaps=path.startswith("bitmap"))
    graph = path in ("graph", "bitmap_graph", "bitmap_direct_graph", "bitmap_fused_graph")
    loads = ("direct" if path.startswith("bitmap_direct") else
             "fused" if path.startswith("bitmap_fused") else "tma")
    path = {"graph": "levels", "bitmap_graph": "bitmap", "bitmap_direct": "bitmap",
            "bitmap_direct_graph": "bitmap", "bitmap_fused": "bitmap",
            "bitmap_fused_graph": "bitmap"}.get(path, path)
    ids, dists, st = index.query(Qd, k, batch=batch, stats=True, path=path, order=order,
                                 rerank=rerank, graph=graph, loads=loads)
    cid, ccol, st2 = index.candidates(Qd, k, batch=batch, path=path, order=order, graph=graph,
                                      loads=loads)
    torch.cuda.synchronize()
    out = dict(ids=ids.cpu().numpy(), dists=dists.cpu().numpy(), stats=st.cpu().numpy(),
               cid=cid.cpu().numpy(), ccol=ccol.cpu().numpy(), stats2=st2.cpu().numpy(),
               index=index)
    return out


def _full_parity(orc, qw, dev, X, Q, A, b, *, w, k, v, l=None, c=2, batch=0, host=False,
                 path="auto", order="auto", rerank="fp32"):
    n = X.shape[0]
    if l is None:
        l = orc.threshold(A.shape[0], w, c, n, v)
    H, HQ, oidx, ref = _oracle_run(orc, X, Q, A, b, w, k, v, l, c)
    g = _gpu_workload(qw, dev, X, Q, A, b, w=w, k=k, v=v, l=l, c=c, batch=batch, host=host,
                      path=path, order=order, rerank=rerank)
    _check_results(g["ids"], g["dists"], ref["ids"], ref["dists"])
    assert np.array_equal(g["stats"], ref["stats"]), "per-query statistics differ"
    assert np.array_equal(g["stats2"], ref["stats"])
    _check_candidates(g["cid"], g["ccol"], ref["cand_ids"], ref["cand_col"])
    g["index"].free()
    return ref, g


# ---------------------------------------------------------------- hand-worked case
@PATHS
def test_hand_worked_golden(qwlib, cuda, path):
    """The workload worked out by hand (tests/golden/hand_worked_query.json):
    every path returns its statistics, kept candidates with their counts,
    ids and distances (the oracle is pinned to the same values)."""
    import json
    import math
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "hand_worked_query.json")) as fh:
        g = json.load(fh)
    p = g["params"]
    X, Q = (np.array(g[key], np.float32) for key in ("X", "Q"))
    A, b = np.array(g["A"], np.float32), np.array(g["b"], np.float32)
    H, _ = qwlib.hash(_t(X, cuda), _t(A, cuda), _t(b, cuda), p["w"])
    assert np.array_equal(H.cpu().numpy(), np.array(g["H"]))
    out = _gpu_workload(qwlib, cuda, X, Q, A, b, w=p["w"], k=p["k"], v=p["v"], l=p["l"],
                        c=p["c"], path=path)
    cap = p["k"] + p["v"]
    for qi, q in enumerate(g["queries"]):
        assert out["stats"][qi].tolist() == q["stats"], f"query {qi} statistics"
        assert out["stats2"][qi].tolist() == q["stats"]
        assert out["ids"][qi].tolist() == q["ids"], f"query {qi} ids"
        want_d = [math.sqrt(x) if x is not None else math.inf for x in q["sqdists"]]
        fin = np.isfinite(want_d)
        assert np.array_equal(np.isfinite(out["dists"][qi]), fin)
        assert np.allclose(out["dists"][qi][fin], np.array(want_d)[fin], rtol=DIST_RTOL, atol=0)
        order = np.argsort(q["kept"], kind="stable")
        kept = np.array(q["kept"], np.int64)[order]
        col = np.array(q["kept_col"], np.int32)[order]
        assert out["cid"][qi].tolist() == kept.tolist() + [-1] * (cap - kept.size)
        assert out["ccol"][qi][: kept.size].tolist() == col.tolist()
    out["index"].free()


# ---------------------------------------------------------------- multi-probe
@pytest.mark.parametrize("graph", [False, True])
def test_multi_probe_hand_worked(qwlib, cuda, graph):
    """The hand-worked multi-probe cases (one probe on each side) on the level
    path: statistics, kept candidates and results."""
    import json
    import math
    import os
    import torch
    with open(os.path.join(os.path.dirname(__file__), "golden", "hand_worked_query.json")) as fh:
        g = json.load(fh)
    p, mp = g["params"], g["multi_probe"]
    X = np.array(g["X"], np.float32)
    A, b = np.array(g["A"], np.float32), np.array(g["b"], np.float32)
    Q = _t(np.array(mp["Q"], np.float32), cuda)
    index = qwlib.Index(_t(X, cuda), _t(A, cuda), _t(b, cuda), w=p["w"], c=p["c"], v=p["v"],
                        l=p["l"])
    ids, dists, st = index.query(Q, p["k"], stats=True, path="levels", graph=graph,
                                 probes=mp["probes"])
    cid, ccol, st2 = index.candidates(Q, p["k"], path="levels", graph=graph, probes=mp["probes"])
    torch.cuda.synchronize()
    cap = p["k"] + p["v"]
    for qi, q in enumerate(mp["queries"]):
        assert st[qi].tolist() == q["stats"] and st2[qi].tolist() == q["stats"]
        assert ids[qi].tolist() == q["ids"]
        assert np.allclose(dists[qi].cpu().numpy(), [math.sqrt(x) for x in q["sqdists"]],
                           rtol=DIST_RTOL, atol=0)
        assert cid[qi].tolist() == sorted(q["kept"]) + [-1] * (cap - len(q["kept"]))
    with pytest.raises(qwlib.QwError):
        index.query(Q, p["k"], path="bitmap", probes=1)
    index.free()


@pytest.mark.parametrize("probes", [1, 2])
def test_multi_probe_matches_oracle(orc, qwlib, cuda, probes):
    """Multi-probe on the level path (host loop, graph mode, learned first
    levels) against the oracle, with queries far below and above the data on
    every projection (the radius rule waits for R > -g_i) over several tiles."""
    import torch
    wl = workloads.make_workload("mix10k_d32", seed=40 + probes, n=2 * TILE + 999, nq=60, d=24,
                                 m=16, n_clusters=25)
    Q = wl.Q.copy()
    shift = np.linalg.pinv(wl.A.astype(np.float64)) @ np.full(16, 300.0)
    Q[:4] = (Q[:4] - shift).astype(np.float32)
    Q[4:7] = (Q[4:7] + shift).astype(np.float32)
    k, v = 10, 120
    l = orc.threshold(16, 4.0, 2, wl.X.shape[0], v)
    H = orc.hash(wl.X, wl.A, wl.b, 4.0)
    HQ = orc.hash(Q, wl.A, wl.b, 4.0)
    oidx = orc.build_index(H)
    ref = orc.query(wl.X, oidx, Q, HQ, k=k, v=v, l=l, probes=probes)
    index = qwlib.Index(_t(wl.X, cuda), _t(wl.A, cuda), _t(wl.b, cuda), w=4.0, v=v, l=l)
    Qd = _t(Q, cuda)
    for graph in (False, True):
        ids, dists, st = index.query(Qd, k, stats=True, graph=graph, probes=probes)
        cid, ccol, _ = index.candidates(Qd, k, graph=graph, probes=probes)
        torch.cuda.synchronize()
        _check_results(ids.cpu().numpy(), dists.cpu().numpy(), ref["ids"], ref["dists"])
        assert np.array_equal(st.cpu().numpy(), ref["stats"])
        _check_candidates(cid.cpu().numpy(), ccol.cpu().numpy(), ref["cand_ids"], ref["cand_col"])
    # learned first levels (recomputed where a first level was the last)
    _, _, stt = index.query(Qd, k, stats=True, probes=probes)
    labels = (stt[:, 0] - 1).clamp(0, 15).to(torch.int32).contiguous()
    F = index.features(Qd)
    mlp = qwlib.Mlp(F.shape[1], 256, 16)
    mlp.set_params(qwlib.mlp_init(F.shape[1], 256, 16, seed=3))
    mlp.train(F, labels, epochs=5, batch=64, lr=1e-3)
    index.set_start_model(mlp, eps=0.5)
    ids2, dists2, st2 = index.query(Qd, k, stats=True, start="learned", probes=probes)
    torch.cuda.synchronize()
    _check_results(ids2.cpu().numpy(), dists2.cpu().numpy(), ref["ids"], ref["dists"])
    assert np.array_equal(st2.cpu().numpy(), ref["stats"])
    index.free()
    mlp.free()


# ---------------------------------------------------------------- boundary: seeded draws
def test_seeded_projections_and_getter(orc, qwlib, cuda):
    """An index built without A and b draws them from its seed
    (qw_draw_projections); qw_index_get_projections returns exactly those and
    the anchors, and the oracle given them reproduces the index's answers."""
    wl = workloads.make_workload("mix10k_d32", seed=44, n=6000, nq=40, d=24, m=12)
    index = qwlib.Index(_t(wl.X, cuda), w=4.0, v=60, m=12, seed=99, bitmaps=True)
    A, b, o = index.projections()
    wantA, wantb = qwlib.qw_draw_projections(99, 12, 24, 4.0)
    assert np.array_equal(A, wantA) and np.array_equal(b, wantb)
    l = index.l
    H, HQ, oidx, ref = _oracle_run(orc, wl.X, wl.Q, A, b, 4.0, 10, 60, l)
    assert np.array_equal(o, oidx.o)
    for path in ("levels", "bitmap"):
        ids, dists, st = index.query(_t(wl.Q, cuda), 10, stats=True, path=path)
        _check_results(ids.cpu().numpy(), dists.cpu().numpy(), ref["ids"], ref["dists"])
        assert np.array_equal(st.cpu().numpy(), ref["stats"])
    index.free()
    # given projections are returned unchanged
    ix2 = qwlib.Index(_t(wl.X, cuda), _t(wl.A, cuda), _t(wl.b, cuda), w=4.0, v=60)
    A2, b2, _ = ix2.projections()
    assert np.array_equal(A2, wl.A) and np.array_equal(b2, wl.b)
    ix2.free()


# ---------------------------------------------------------------- a1 + a2: hashing
@pytest.mark.parametrize("tc", [False, True], ids=["fp32", "tensor"])
@pytest.mark.parametrize("n,d,m,scale", [(10_000, 32, 16, 1.0), (1_007, 33, 5, 3.0),
                                         (20_000, 128, 64, 1.0), (4_099, 512, 7, 0.5),
                                         (3_000, 64, 128, 2.0), (129, 200, 100, 1.0)])
def test_hash_bit_exact(orc, qwlib, cuda, n, d, m, scale, tc):
    """FP32 CUDA-core and tensor-core projections (several 128-row tiles and a
    ragged one, d not a multiple of the staged chunk, m not a multiple of 16)
    against the FP64 definition."""
    wl = workloads.make_workload("mix10k_d32", seed=n, n=n, nq=1, d=d, m=m)
    X = (wl.X * scale).astype(np.float32)
    want = orc.hash(X, wl.A, wl.b, 4.0)
    H, fix = qwlib.hash(_t(X, cuda), _t(wl.A, cuda), _t(wl.b, cuda), 4.0, tensor_cores=tc)
    got = H.cpu().numpy()
    assert np.array_equal(got, want), f"{int((got != want).sum())} bucket ids differ"
    assert 0 <= fix <= want.size * (0.2 if tc else 0.05)


def test_hash_tensor_cores_on_1e8_entries(qwlib, cuda):
    """The tensor-core projection's window holds on 2,000,000 rows x 64
    projections (1.28e8 entries, d = 128, the benchmark's data scale): its
    bucket ids equal those of the FP32 pass (itself exact against the FP64
    definition), and the share recomputed in FP64 stays small."""
    import torch
    g = torch.Generator(device=cuda).manual_seed(11)
    n, d, m = 2_000_000, 128, 64
    X = torch.randn((n, d), generator=g, device=cuda, dtype=torch.float32) * 1.0
    X += torch.rand((n // 1000 + 1, d), generator=g, device=cuda).repeat_interleave(1000, 0)[:n] * 20 - 10
    A = torch.randn((m, d), generator=g, device=cuda, dtype=torch.float32)
    b = torch.rand((m,), generator=g, device=cuda, dtype=torch.float32) * 4.0
    H1, fix1 = qwlib.hash(X.contiguous(), A, b, 4.0)
    H2, fix2 = qwlib.hash(X.contiguous(), A, b, 4.0, tensor_cores=True)
    assert torch.equal(H1, H2)
    assert fix2 < 0.1 * n * m, f"{fix2} recomputations"


def test_hash_boundary_points_take_fp64(orc, qwlib, cuda):
    """Points placed within ~1e-6 w of a bucket edge of projection 0 must be
    re-evaluated in FP64 and still match the FP64 definition."""
    rng = np.random.default_rng(7)
    d, m, w = 128, 8, 4.0
    A = rng.standard_normal((m, d), dtype=np.float32)
    b = (rng.random(m) * w).astype(np.float32)
    X0 = rng.standard_normal((4096, d)).astype(np.float64) * 5.0
    a0 = A[0].astype(np.float64)
    t0 = X0 @ a0 + float(b[0])
    target = np.round(t0 / w) * w + rng.uniform(-1e-6, 1e-6, size=t0.shape) * w
    X = (X0 + np.outer(target - t0, a0) / (a0 @ a0)).astype(np.float32)
    want = orc.hash(X, A, b, w)
    for tc in (False, True):
        H, fix = qwlib.hash(_t(X, cuda), _t(A, cuda), _t(b, cuda), w, tensor_cores=tc)
        assert np.array_equal(H.cpu().numpy(), want)
        assert fix >= 2000, f"only {fix} entries were recomputed in FP64"


@pytest.mark.parametrize("path", ["levels", "bitmap_direct_graph"])
def test_workload_with_tensor_core_projection(orc, qwlib, cuda, path):
    """Index built and queries projected on the tensor cores: the oracle's
    statistics, candidates and results."""
    import torch
    wl = workloads.make_workload("mix10k_d32", seed=17, n=9000, nq=60, d=48, m=24)
    l = orc.threshold(24, 4.0, 2, 9000, 80)
    H, HQ, oidx, ref = _oracle_run(orc, wl.X, wl.Q, wl.A, wl.b, 4.0, 10, 80, l)
    index = qwlib.Index(_t(wl.X, cuda), _t(wl.A, cuda), _t(wl.b, cuda), w=4.0, v=80, l=l,
                        bitmaps=True, projection="tensor")
    o, span, _, _ = index.export()
    assert np.array_equal(o, oidx.o) and np.array_equal(span, oidx.span)
    graph = path.endswith("graph")
    ids, dists, st = index.query(_t(wl.Q, cuda), 10, stats=True, projection="tensor",
                                 path="bitmap" if path != "levels" else "levels", graph=graph,
                                 loads="direct")
    torch.cuda.synchronize()
    _check_results(ids.cpu().numpy(), dists.cpu().numpy(), ref["ids"], ref["dists"])
    assert np.array_equal(st.cpu().numpy(), ref["stats"])
    index.free()


@pytest.mark.parametrize("loads", ["direct", "fused"])
def test_tile_shapes_same_results(orc, qwlib, cuda, loads):
    """Every tile shape the autotuner may pick (tiles per warp of the filter /
    fused kernels, candidate rows per warp of the distance kernels, FP32 and
    BF16 pre-filter) gives the oracle's results; the index spans several tiles
    and a ragged one."""
    import torch
    wl = workloads.make_workload("mix10k_d32", seed=19, n=5 * TILE + 777, nq=70, d=40, m=20,
                                 n_clusters=30)
    l = orc.threshold(20, 4.0, 2, wl.X.shape[0], 150)
    _, _, _, ref = _oracle_run(orc, wl.X, wl.Q, wl.A, wl.b, 4.0, 12, 150, l)
    index = qwlib.Index(_t(wl.X, cuda), _t(wl.A, cuda), _t(wl.b, cuda), w=4.0, v=150, l=l,
                        bitmaps=True, shadow_bf16=True)
    Q = _t(wl.Q, cuda)
    for tpw in (4, 8, 16):
        for rows in (2, 4, 8):
            for rerank in ("fp32", "bf16", "bf16_tc"):
                for graph in (False, True):
                    ids, dists, st = index.query(Q, 12, stats=True, path="bitmap", loads=loads,
                                                 graph=graph, tiles_per_warp=tpw,
                                                 rerank_rows=rows, rerank=rerank)
                    torch.cuda.synchronize()
                    _check_results(ids.cpu().numpy(), dists.cpu().numpy(), ref["ids"],
                                   ref["dists"])
                    assert np.array_equal(st.cpu().numpy(), ref["stats"])
    with pytest.raises(qwlib.QwError):
        index.query(Q, 12, path="bitmap", loads=loads, tiles_per_warp=5)
    with pytest.raises(qwlib.QwError):
        index.query(Q, 12, rerank_rows=3)
    index.free()


# ---------------------------------------------------------------- a3: index build
@pytest.mark.parametrize("n,d,m", [(10_000, 32, 16), (2 * TILE + 1234, 16, 8), (TILE, 8, 3),
                                   (1, 4, 2), (TILE + 1, 12, 5)])
def test_build_matches_oracle(orc, qwlib, cuda, n, d, m):
    wl = workloads.make_workload("mix10k_d32", seed=3, n=n, nq=1, d=d, m=m,
                                 n_clusters=min(50, n))
    H = orc.hash(wl.X, wl.A, wl.b, 4.0)
    oidx = orc.build_index(H)
    index = qwlib.Index(_t(wl.X, cuda), _t(wl.A, cuda), _t(wl.b, cuda), w=4.0, v=100)
    o, span, eb, ei = index.export()
    index.free()
    assert np.array_equal(o, oidx.o)
    assert np.array_equal(span, oidx.span)
    for i in range(m):
        tile = ei[i] // TILE
        assert np.all(np.diff(tile) >= 0), "entries not grouped by tile"
        for t in np.unique(tile):
            sel = tile == t
            bb = eb[i][sel]
            assert np.all(np.diff(bb) >= 0), "entries of a tile not grouped by bucket id"
        order = np.lexsort((ei[i], eb[i]))
        assert np.array_equal(eb[i][order], oidx.sbid[i])
        assert np.array_equal(ei[i][order], oidx.sid[i])


# ---------------------------------------------------------------- a4..a9: workloads
@PATHS
def test_workload_small_config(orc, qwlib, cuda, path):
    wl = workloads.make_workload("mix10k_d32", seed=0)
    s = wl.spec
    _full_parity(orc, qwlib, cuda, wl.X, wl.Q, wl.A, wl.b, w=s.w, k=s.k, v=s.v, path=path)


@PATHS
@pytest.mark.parametrize("order", ["given", "signature"])
def test_workload_ragged_tiles_and_batches(orc, qwlib, cuda, path, order):
    """Three index tiles (the last one ragged), small k + v so the truncation
    and its tie rule run, several query batches with a ragged last batch, in
    the caller's order and in signature order."""
    wl = workloads.make_workload("mix10k_d32", seed=11, n=2 * TILE + 777, nq=61, d=24, m=12,
                                 n_clusters=40)
    _full_parity(orc, qwlib, cuda, wl.X, wl.Q, wl.A, wl.b, w=4.0, k=7, v=20, batch=13, path=path,
                 order=order)


@PATHS
def test_workload_host_memory(orc, qwlib, cuda, path):
    wl = workloads.make_workload("mix10k_d32", seed=5, n=5000, nq=40)
    s = wl.spec
    _full_parity(orc, qwlib, cuda, wl.X, wl.Q, wl.A, wl.b, w=s.w, k=s.k, v=s.v, host=True,
                 batch=16, path=path)


@PATHS
def test_workload_v_ge_n_is_exact_knn(orc, qwlib, cuda, path):
    """v >= n: the k + v bound never stops a query, the last level holds every
    point, and the answer is the exact k-NN (queries are data rows)."""
    wl = workloads.make_workload("mix10k_d32", seed=2, n=600, nq=25, n_clusters=6)
    Q = wl.X[:25].copy()
    ref, g = _full_parity(orc, qwlib, cuda, wl.X, Q, wl.A, wl.b, w=4.0, k=10, v=600, l=10, path=path)
    bf_ids, bf_d = orc.bruteforce(wl.X, Q, 10)
    assert np.array_equal(g["ids"], bf_ids)
    assert np.all(g["stats"][:, 4] == 3)


@PATHS
def test_workload_single_projection(orc, qwlib, cuda, path):
    """m = 1, l = 1: plain E2LSH bucket lookup with growing radius."""
    wl = workloads.make_workload("mix10k_d32", seed=4, n=3000, nq=30, m=1)
    _full_parity(orc, qwlib, cuda, wl.X, wl.Q, wl.A, wl.b, w=4.0, k=5, v=10, l=1, path=path)


@PATHS
def test_workload_far_queries_and_padding(orc, qwlib, cuda, path):
    """Queries far outside the data: many levels, bucket ids below the anchor,
    fewer than k candidates (padded with -1 / inf)."""
    wl = workloads.make_workload("mix10k_d32", seed=9, n=2000, nq=12)
    Q = wl.Q.copy()
    Q[:6] += 400.0
    Q[6:] -= 400.0
    _full_parity(orc, qwlib, cuda, wl.X, Q, wl.A, wl.b, w=4.0, k=10, v=100, path=path)


@PATHS
def test_workload_duplicates_tie_by_id(orc, qwlib, cuda, path):
    """Exact duplicate rows: equal distances are ordered by id."""
    wl = workloads.make_workload("mix10k_d32", seed=6, n=1500, nq=20)
    X = np.repeat(wl.X[:300], 5, axis=0)
    _full_parity(orc, qwlib, cuda, X, wl.Q, wl.A, wl.b, w=4.0, k=12, v=30, path=path)


@PATHS
def test_workload_tiny_index(orc, qwlib, cuda, path):
    X = np.array([[0.5, -1.0, 2.0]], np.float32)
    A = np.array([[1.0, 0.0, 0.0], [0.3, 0.2, -0.7]], np.float32)
    b = np.array([0.25, 1.5], np.float32)
    Q = np.array([[0.4, -1.1, 2.0], [30.0, 30.0, 30.0]], np.float32)
    _full_parity(orc, qwlib, cuda, X, Q, A, b, w=2.0, k=1, v=3, l=1, path=path)


@PATHS
def test_workload_k_equals_n(orc, qwlib, cuda, path):
    wl = workloads.make_workload("mix10k_d32", seed=8, n=64, nq=5, n_clusters=3)
    _full_parity(orc, qwlib, cuda, wl.X, wl.Q, wl.A, wl.b, w=4.0, k=64, v=0, l=4, path=path)


@pytest.mark.parametrize("path", ["bitmap_direct", "bitmap_direct_graph", "bitmap"])
@pytest.mark.parametrize("m", [40, 100, 127])
def test_bitmap_many_projections(orc, qwlib, cuda, path, m):
    """More than 32 and more than 64 projections: a tile's bucket summaries
    span two or four lanes' rows in the filter, and a live group's projection
    mask one or two words."""
    wl = workloads.make_workload("mix10k_d32", seed=40 + m, n=TILE + 5000, nq=24, d=32, m=m,
                                 n_clusters=30)
    _full_parity(orc, qwlib, cuda, wl.X, wl.Q, wl.A, wl.b, w=4.0, k=10, v=60, path=path)


@pytest.mark.parametrize("rerank", ["fp32", "bf16", "bf16_tc"])
@pytest.mark.parametrize("path", ["levels", "bitmap_direct_graph"])
@pytest.mark.parametrize("shell", [12, 60])
def test_rerank_near_ties_at_k(orc, qwlib, cuda, path, shell, rerank):
    """A shell of `shell` points whose distances to the query agree to about
    1e-7 holds the k-th nearest: FP32 cannot order them, the rerank must take
    the FP64 order (ties by id).  With 12 points the run past position k is
    short; with 60 it is longer than the selection extends, and the whole
    candidate array is sorted instead.  v >= n keeps every point."""
    rng = np.random.default_rng(100 + shell)
    d, n, k = 32, 600, 10
    q = rng.standard_normal(d)
    u = rng.standard_normal((n, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = np.concatenate([rng.uniform(0.3, 0.9, 5),                      # nearer than the shell
                        1.0 + 2e-8 * np.arange(shell),                  # the shell
                        rng.uniform(2.0, 5.0, n - 5 - shell)])           # farther
    perm = rng.permutation(n)
    X = (q + u * r[perm, None]).astype(np.float32)
    Q = q[None, :].astype(np.float32)
    wl = workloads.make_workload("mix10k_d32", seed=7, n=64, nq=1, d=d, m=8)
    _full_parity(orc, qwlib, cuda, X, Q, wl.A, wl.b, w=4.0, k=k, v=n, l=2, path=path,
                 rerank=rerank)


def test_empty_workload(qwlib, cuda):
    import torch
    wl = workloads.make_workload("mix10k_d32", seed=1, n=500, nq=1)
    index = qwlib.Index(_t(wl.X, cuda), _t(wl.A, cuda), _t(wl.b, cuda), w=4.0)
    ids, dists = index.query(torch.empty((0, wl.X.shape[1]), dtype=torch.float32, device=cuda), 5)
    assert ids.shape == (0, 5)
    index.free()


@pytest.mark.parametrize("rerank", ["bf16", "bf16_tc"])
@pytest.mark.parametrize("path", ["levels", "bitmap_direct_graph"])
@pytest.mark.parametrize("d", [32, 30, 100])
def test_bf16_prefilter_rerank_is_exact(orc, qwlib, cuda, d, path, rerank):
    """The BF16 pre-filter (on CUDA cores, or with its dot products on the
    tensor cores) keeps every candidate that could be among the k nearest:
    same ids as the oracle, distances within 1e-5 (d = 30 and 100 take the
    scalar, unaligned loads and a dimension padded to the MMA's 16; an index
    with bitmaps keeps its residual copy in the locality order, one without in
    data order)."""
    wl = workloads.make_workload("mix10k_d32", seed=31, n=6000, nq=80, d=d)
    _full_parity(orc, qwlib, cuda, wl.X, wl.Q, wl.A, wl.b, w=4.0, k=10, v=300, rerank=rerank,
                 path=path)


@pytest.mark.parametrize("rerank", ["bf16", "bf16_tc"])
def test_bf16_prefilter_many_candidates(orc, qwlib, cuda, rerank):
    """Both pre-filter forms at k + v = 4,096 candidates per query in d = 256
    (the CUDA-core form's 16-byte loads and two-pass k-th bound; 32 MMA tiles
    per query, the largest shared-memory layout, for the tensor-core form),
    with a ragged last tile, and at d = 512: the oracle's ids."""
    wl = workloads.make_workload("mix10k_d32", seed=34, n=30000, nq=40, d=256, m=16,
                                 n_clusters=8)
    _full_parity(orc, qwlib, cuda, wl.X, wl.Q, wl.A, wl.b, w=4.0, k=10, v=4086, l=2,
                 rerank=rerank, path="levels")
    _full_parity(orc, qwlib, cuda, wl.X, wl.Q, wl.A, wl.b, w=4.0, k=7, v=1000, l=2,
                 rerank=rerank, path="levels")
    wl = workloads.make_workload("mix10k_d32", seed=35, n=8000, nq=24, d=512, m=16,
                                 n_clusters=8)
    _full_parity(orc, qwlib, cuda, wl.X, wl.Q, wl.A, wl.b, w=4.0, k=10, v=1500, l=2,
                 rerank=rerank, path="levels")


@pytest.mark.parametrize("rerank", ["bf16", "bf16_tc"])
def test_bf16_prefilter_ragged_groups_and_duplicates(orc, qwlib, cuda, rerank):
    """Residual groups of 128 rows with a ragged last group, exact duplicate
    rows (zero residual spread within a tie) and queries that are data rows
    (distance 0): the bound must hold at both ends."""
    wl = workloads.make_workload("mix10k_d32", seed=33, n=5 * 128 + 37, nq=30, n_clusters=4)
    X = wl.X.copy()
    X[100:140] = X[99]
    Q = np.concatenate([X[[3, 99, 120, 600]], wl.Q[:26]]).astype(np.float32)
    for path in ("levels", "bitmap_direct"):
        _full_parity(orc, qwlib, cuda, X, Q, wl.A, wl.b, w=4.0, k=12, v=200, rerank=rerank,
                     path=path)


def test_bf16_prefilter_reads_fewer_fp32_rows(qwlib, cuda):
    import torch
    wl = workloads.make_workload("mix10k_d32", seed=32, n=20000, nq=200, d=64, m=16)
    X, A, b = (torch.from_numpy(a).to(cuda) for a in (wl.X, wl.A, wl.b))
    index = qwlib.Index(X, A, b, w=4.0, v=400, shadow_bf16=True)
    Q = torch.from_numpy(wl.Q).to(cuda)
    ref_ids, ref_d = index.query(Q, 10, rerank="fp32")
    index.profile(reset=True)
    for rerank in ("bf16", "bf16_tc"):
        ids, dists = index.query(Q, 10, rerank=rerank, profile=True)
        p = index.profile(reset=True)
        assert torch.equal(ids, ref_ids), rerank
        assert torch.equal(dists, ref_d), rerank
        assert p["rerank_fp32_rows"] < p["rerank_candidates"], rerank
    index.free()
    with pytest.raises(qwlib.QwError):
        plain = qwlib.Index(X, A, b, w=4.0, v=400)
        try:
            plain.query(Q, 10, rerank="bf16")
        finally:
            plain.free()


def test_cluster_path_refuses_oversized_index(qwlib, cuda):
    """More than 96 tiles do not fit the cluster path: forcing it is an argument
    error, and the automatic choice runs the level path instead."""
    import torch
    n = 96 * TILE + 5
    rng = np.random.default_rng(0)
    X = torch.from_numpy(rng.standard_normal((n, 4), dtype=np.float32)).to(cuda)
    A = torch.from_numpy(rng.standard_normal((2, 4), dtype=np.float32)).to(cuda)
    b = torch.from_numpy(np.array([0.5, 1.0], np.float32)).to(cuda)
    index = qwlib.Index(X, A, b, w=4.0, v=10, l=1)
    Q = X[:3].clone()
    with pytest.raises(qwlib.QwError) as e:
        index.query(Q, 2, path="cluster")
    assert e.value.status == qwlib.QW_ERR_ARG
    ids, _ = index.query(Q, 2)
    assert ids.shape == (3, 2)
    index.free()


def test_argument_errors(qwlib, cuda):
    wl = workloads.make_workload("mix10k_d32", seed=1, n=500, nq=4)
    index = qwlib.Index(_t(wl.X, cuda), _t(wl.A, cuda), _t(wl.b, cuda), w=4.0)
    Q = _t(wl.Q, cuda)
    with pytest.raises(qwlib.QwError) as e:
        index.query(Q, 0)
    assert e.value.status == qwlib.QW_ERR_ARG
    with pytest.raises(qwlib.QwError):
        index.query(Q, 501)
    with pytest.raises(qwlib.QwError):
        index.query(Q, 4000)  # k + v > 4096
    index.free()
    with pytest.raises(qwlib.QwError) as e:
        qwlib.Index(_t(wl.X, cuda), _t(wl.A, cuda), _t(wl.b, cuda), w=0.0)
    assert e.value.status == qwlib.QW_ERR_ARG
    with pytest.raises(qwlib.QwError) as e:
        qwlib.Index(_t(wl.X * 1e12, cuda), _t(wl.A, cuda), _t(wl.b, cuda), w=1e-6)
    assert e.value.status == qwlib.QW_ERR_RANGE


# ---------------------------------------------------------------- full size, sampled
@pytest.mark.slow
def test_full_size_sampled(orc, qwlib, cuda):
    """The benchmarked workload (1M x 128, 64 projections, 10,000 queries,
    k = 100, v = 700, l = 43) run whole on the GPU in the benchmark's launch
    configuration (bitmap path, signature order, learned first levels, graph
    mode) and in the plain one; the oracle recomputes a seeded sample of 128
    queries one by one."""
    import torch
    wl = workloads.make_workload("mix1m_d128", seed=0, n_train=8_000)
    s = wl.spec
    v, l = 700, 43
    index = qwlib.Index(_t(wl.X, cuda), _t(wl.A, cuda), _t(wl.b, cuda), w=s.w, c=s.c, v=v, l=l,
                        bitmaps=True)
    Qd = _t(wl.Q, cuda)
    # start model trained on earlier queries of the workload, as the benchmark does
    Qt = _t(wl.Q_train, cuda)
    _, _, stt = index.query(Qt, s.k, stats=True, path="bitmap")
    labels = (stt[:, 0] - 1).clamp(0, 15).to(torch.int32).contiguous()
    F = index.features(Qt)
    mlp = qwlib.Mlp(F.shape[1], 256, 16)
    mlp.set_params(qwlib.mlp_init(F.shape[1], 256, 16, seed=5))
    mlp.train(F, labels, epochs=10, batch=512, lr=1e-3)
    index.set_start_model(mlp, eps=0.02)
    ids, dists, st = index.query(Qd, s.k, stats=True, path="bitmap", order="signature",
                                 start="learned", graph=True, loads="direct")
    prof = index.profile(reset=True)
    ids2, dists2, st2 = index.query(Qd, s.k, stats=True, path="levels", order="given")
    torch.cuda.synchronize()
    ids, dists, st = ids.cpu().numpy(), dists.cpu().numpy(), st.cpu().numpy()
    # the two configurations agree on every query
    assert np.array_equal(ids, ids2.cpu().numpy())
    assert np.array_equal(st, st2.cpu().numpy())
    assert np.array_equal(dists, dists2.cpu().numpy())
    assert prof["start_levels_skipped"] > 0
    H = oracle_par.hash_rows(orc, wl.X, wl.A, wl.b, s.w)
    oidx = orc.build_index(H, sorted_arrays=True)
    assert index.info.l == l
    # 128 seeded queries recomputed by the oracle, spread over the host threads
    sample = np.random.default_rng(123).choice(s.nq, size=128, replace=False)
    sample.sort()
    HQ = orc.hash(wl.Q[sample], wl.A, wl.b, s.w)
    ref = oracle_par.query_rows(orc, wl.X, oidx, wl.Q[sample], HQ, k=s.k, v=v, l=l, c=s.c)
    _check_results(ids[sample], dists[sample], ref["ids"], ref["dists"])
    assert np.array_equal(st[sample], ref["stats"])
    # properties that hold for every query
    assert np.all((st[:, 4] == 2) | (st[:, 4] == 3))
    assert np.all(st[:, 3] <= s.k + v)
    assert np.all(np.diff(dists, axis=1)[np.isfinite(dists[:, 1:])] >= 0)
    index.free()
    mlp.free()


def test_full_size_10m_sampled(orc, qwlib, cuda):
    """The benchmark's largest workload, 10,000,000 x 128 (10,000 clusters,
    64 projections, w = 4, v = 1,000, l derived from Eq. 1) with its 100,000
    queries: the benchmark's configuration (bitmap path, signature order,
    learned first levels, graph mode) against the plain-start bitmap path on
    every query, and 32 seeded queries recomputed by the oracle."""
    import torch
    wl = workloads.make_workload("mix10m_d128", seed=0, n_train=20_000)
    s = wl.spec
    v = 1000
    index = qwlib.Index(_t(wl.X, cuda), _t(wl.A, cuda), _t(wl.b, cuda), w=s.w, c=s.c, v=v, l=0,
                        bitmaps=True)
    l = index.l
    assert l == orc.threshold(s.m, s.w, s.c, s.n, v)
    Qd = _t(wl.Q, cuda)
    Qt = _t(wl.Q_train, cuda)
    _, _, stt = index.query(Qt, s.k, stats=True, path="bitmap")
    labels = (stt[:, 0] - 1).clamp(0, 15).to(torch.int32).contiguous()
    F = index.features(Qt)
    mlp = qwlib.Mlp(F.shape[1], 256, 16)
    mlp.set_params(qwlib.mlp_init(F.shape[1], 256, 16, seed=5))
    mlp.train(F, labels, epochs=10, batch=512, lr=1e-3)
    index.set_start_model(mlp, eps=0.02)
    index.profile(reset=True)
    ids, dists, st = index.query(Qd, s.k, stats=True, path="bitmap", order="signature",
                                 start="learned", graph=True, loads="direct")
    prof = index.profile(reset=True)
    ids2, dists2, st2 = index.query(Qd, s.k, stats=True, path="bitmap", order="given",
                                    start="plain", loads="direct")
    torch.cuda.synchronize()
    ids, dists, st = ids.cpu().numpy(), dists.cpu().numpy(), st.cpu().numpy()
    assert np.array_equal(ids, ids2.cpu().numpy())
    assert np.array_equal(st, st2.cpu().numpy())
    assert np.array_equal(dists, dists2.cpu().numpy())
    assert prof["start_levels_skipped"] > 0
    H = oracle_par.hash_rows(orc, wl.X, wl.A, wl.b, s.w)
    oidx = orc.build_index(H, sorted_arrays=False)
    sample = np.sort(np.random.default_rng(321).choice(s.nq, size=32, replace=False))
    HQ = orc.hash(wl.Q[sample], wl.A, wl.b, s.w)
    ref = oracle_par.query_rows(orc, wl.X, oidx, wl.Q[sample], HQ, k=s.k, v=v, l=l, c=s.c)
    _check_results(ids[sample], dists[sample], ref["ids"], ref["dists"])
    # the oracle's index without sorted arrays does not count the entries
    # scanned (statistics 5 and 6); every other statistic is compared
    cols = [0, 1, 2, 3, 4, 7]
    assert np.array_equal(st[sample][:, cols], ref["stats"][:, cols])
    assert np.all((st[:, 4] == 2) | (st[:, 4] == 3))
    index.free()
    mlp.free()


@pytest.mark.parametrize("graph", [False, True])
def test_bitmap_path_large_tie_classes(orc, qwlib, cuda, graph):
    """Ten distinct points, 20,000 copies each: whole tiles of candidates and
    tie classes of 20,000 ids with the same count, more than the bitmap path's
    tie list holds.  The selection then picks the smallest ids of the tie
    class from the candidate list itself; every output equals the oracle's
    and no query needs the level path."""
    rng = np.random.default_rng(31)
    base = rng.uniform(-10, 10, size=(10, 16)).astype(np.float32)
    X = np.repeat(base, 20_000, axis=0)
    Q = (base[[0, 3, 7, 9]] + rng.normal(0, 0.05, size=(4, 16))).astype(np.float32)
    wl = workloads.make_workload("mix10k_d32", seed=3, n=1000, nq=1, d=16, m=16)
    for loads in ("tma", "direct"):
        _full_parity(orc, qwlib, cuda, X, Q, wl.A, wl.b, w=4.0, k=10, v=90, l=12,
                     path=("bitmap_graph" if graph else "bitmap") if loads == "tma" else
                     ("bitmap_direct_graph" if graph else "bitmap_direct"))
    index = qwlib.Index(_t(X, cuda), _t(wl.A, cuda), _t(wl.b, cuda), w=4.0, v=90, l=12,
                        bitmaps=True)
    index.profile(reset=True)
    index.query(_t(Q, cuda), 10, path="bitmap", graph=graph, loads="direct")
    assert index.profile()["bitmap_fallbacks"] == 0
    index.free()


@pytest.mark.parametrize("graph", [False, True])
def test_bitmap_path_overflow_of_duplicates(orc, qwlib, cuda, graph):
    """270,000 copies of one point (plus a few others): the query's first
    level holds 270,000 candidates with one count, more than the bitmap path's
    per-query list (262,144).  The list is rebuilt with the smallest original
    ids of that tie class (by id bins), no query needs the level path, and
    every output equals the oracle's."""
    rng = np.random.default_rng(37)
    base = rng.uniform(-10, 10, size=(4, 16)).astype(np.float32)
    X = np.concatenate([np.repeat(base[:1], 270_000, axis=0), np.repeat(base[1:], 300, axis=0)])
    Q = (base[[0, 1, 2]] + rng.normal(0, 0.05, size=(3, 16))).astype(np.float32)
    wl = workloads.make_workload("mix10k_d32", seed=3, n=1000, nq=1, d=16, m=16)
    for path in (("bitmap_direct_graph", "bitmap_graph") if graph else ("bitmap_direct", "bitmap")):
        _full_parity(orc, qwlib, cuda, X, Q, wl.A, wl.b, w=4.0, k=10, v=90, l=12, path=path)
    index = qwlib.Index(_t(X, cuda), _t(wl.A, cuda), _t(wl.b, cuda), w=4.0, v=90, l=12,
                        bitmaps=True)
    index.profile(reset=True)
    index.query(_t(Q, cuda), 10, path="bitmap", graph=graph, loads="direct", profile=True)
    prof = index.profile()
    assert prof["bitmap_overflows"] >= 1
    assert prof["bitmap_fallbacks"] == 0
    index.free()


def _cluster_overflow_case():
    """400,000 points, most in one tight Gaussian cluster (sigma 0.3, d = 16),
    and 96 queries at distances 4 to 9 from its centre: one doubling of the
    radius sweeps most of the cluster into the last level of about a quarter
    of the queries (262,000 to 380,000 candidates, with up to 83 of the
    previous level's), above the bitmap path's list of 262,144."""
    rng = np.random.default_rng(43)
    d, m, n = 16, 16, 400_000
    base = rng.uniform(-10, 10, size=(3, d)).astype(np.float32)
    X = np.concatenate([base[0] + rng.normal(0, 0.3, size=(n - 20_000, d)),
                        base[1] + rng.normal(0, 0.3, size=(20_000, d))]).astype(np.float32)
    A = rng.standard_normal((m, d), dtype=np.float32)
    b = (rng.random(m) * 4).astype(np.float32)
    rq = np.random.default_rng(5)

    def queries(count):
        dirs = rq.normal(size=(count, d))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        return (base[0] + dirs * rq.uniform(4, 9, size=count)[:, None]).astype(np.float32)

    Q = queries(96)
    return X, Q, A, b, queries(3000)


@pytest.mark.slow
def test_bitmap_path_overflow_from_clusters(orc, qwlib, cuda):
    """Last levels larger than the candidate list, from a real cluster: every
    bitmap variant rebuilds those lists and returns the oracle's candidate
    sets, counts, statistics and results, with no query on the level path;
    learned first levels (recounted previous level) and over-eager ones
    (answered again from level 0) give the same results."""
    import torch
    X, Q, A, b, Qt = _cluster_overflow_case()
    kw = dict(w=4.0, k=10, v=90, l=10)
    ref, _ = _full_parity(orc, qwlib, cuda, X, Q, A, b, path="bitmap", **kw)
    for path in ("bitmap_direct", "bitmap_direct_graph", "bitmap_fused", "bitmap_fused_graph"):
        _check_same(qwlib, cuda, X, Q, A, b, ref, path=path, **kw)
    assert int((ref["stats"][:, 2] > 262_144).sum()) >= 10
    index = qwlib.Index(_t(X, cuda), _t(A, cuda), _t(b, cuda), w=4.0, v=90, l=10, bitmaps=True)
    Qd, Qtd = _t(Q, cuda), _t(Qt, cuda)
    index.profile(reset=True)
    ids0, d0, st0 = index.query(Qd, 10, stats=True, path="bitmap", loads="direct", profile=True)
    prof = index.profile(reset=True)
    assert prof["bitmap_overflows"] >= 10 and prof["bitmap_fallbacks"] == 0
    assert np.array_equal(ids0.cpu().numpy(), ref["ids"])
    # learned first levels
    _, _, stt = index.query(Qtd, 10, stats=True, path="bitmap", loads="direct")
    labels = (stt[:, 0] - 1).clamp(0, 15).to(torch.int32).contiguous()
    F = index.features(Qtd)
    mlp = qwlib.Mlp(F.shape[1], 256, 16)
    mlp.set_params(qwlib.mlp_init(F.shape[1], 256, 16, seed=7))
    mlp.train(F, labels, epochs=10, batch=256, lr=1e-3)
    # eps = 0.999 predicts some first levels past the last level the loop
    # runs for the batch; they start at their own last useful level instead
    for eps in (0.02, 0.999):
        index.set_start_model(mlp, eps=eps)
        for path, graph, loads in (("bitmap", False, "direct"), ("bitmap", True, "direct"),
                                   ("bitmap", True, "tma"), ("bitmap", False, "fused"),
                                   ("bitmap", True, "fused"), ("levels", False, "tma"),
                                   ("levels", True, "tma")):
            ids, dd, st = index.query(Qd, 10, stats=True, path=path, start="learned",
                                      graph=graph, loads=loads, profile=True)
            p = index.profile(reset=True)
            assert torch.equal(ids, ids0) and torch.equal(dd, d0) and torch.equal(st, st0), \
                (eps, path, graph, loads)
            assert p["bitmap_fallbacks"] == 0
            if eps < 0.5 and path == "bitmap":
                assert p["start_levels_skipped"] > 0
    index.free()
    mlp.free()


def _check_same(qwlib, cuda, X, Q, A, b, ref, *, w, k, v, l, path):
    """Another path's outputs against an oracle run already checked."""
    g = _gpu_workload(qwlib, cuda, X, Q, A, b, w=w, k=k, v=v, l=l, path=path)
    _check_results(g["ids"], g["dists"], ref["ids"], ref["dists"])
    assert np.array_equal(g["stats"], ref["stats"]), "per-query statistics differ"
    assert np.array_equal(g["stats2"], ref["stats"])
    _check_candidates(g["cid"], g["ccol"], ref["cand_ids"], ref["cand_col"])
    g["index"].free()
    return g
