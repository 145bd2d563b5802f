"""The autotuner: it tries the settings it documents, picks one of them, and
whatever it picks answers the workload exactly as the plain level path does.
Graph mode of the level loop against the host-driven loop."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _index(qwlib, cuda, wl, **kw):
    import torch
    X, A, b = (torch.from_numpy(a).to(cuda) for a in (wl.X, wl.A, wl.b))
    return qwlib.Index(X, A, b, w=4.0, **kw)


def test_autotune_choice_keeps_results(qwlib, cuda):
    import torch
    wl = workloads.make_workload("mix10k_d32", seed=21, n=70_000, nq=300, n_clusters=60)
    index = _index(qwlib, cuda, wl, v=60, shadow_bf16=True, bitmaps=True)
    Q = torch.from_numpy(wl.Q).to(cuda)
    ids0, d0, st0 = index.query(Q, 10, stats=True, path="levels", order="given")
    best, trials = index.autotune(Q, 10, reps=2)
    tried = [t for t, _ in trials]
    assert len(trials) >= 7
    assert all(ms > 0 for _, ms in trials)
    # coordinates the tuner documents: path, batch sizes, graph, order, rerank
    assert any(t["path"] == "cluster" for t in tried)
    assert any(t["path"] == "bitmap" for t in tried)
    assert any(t["graph"] for t in tried)
    assert any(t["order"] == "given" for t in tried)
    assert any(t["rerank"] == "bf16" for t in tried)
    assert len({t["batch"] for t in tried}) >= 3
    assert best in tried
    # the chosen setting is at least as fast as the first one tried
    ms_of = {repr(t): ms for t, ms in trials}
    assert ms_of[repr(best)] <= trials[0][1]
    for kw in (best, {}):  # the tuned setting, and path="auto" after tuning
        ids, d, st = index.query(Q, 10, stats=True, **kw)
        assert torch.equal(ids, ids0) and torch.equal(d, d0) and torch.equal(st, st0)
    index.free()


def test_autotune_host_memory_and_errors(qwlib, cuda):
    import torch
    wl = workloads.make_workload("mix10k_d32", seed=22, n=5000, nq=50)
    index = _index(qwlib, cuda, wl, v=40)
    Qh = torch.from_numpy(wl.Q)
    best, trials = index.autotune(Qh, 5, reps=1)
    assert not any(t["rerank"] == "bf16" for t, _ in trials)  # no BF16 copy: not tried
    ids0, d0 = index.query(torch.from_numpy(wl.Q).to(cuda), 5, path="levels")
    ids, d = index.query(Qh, 5, **best)
    assert torch.equal(ids, ids0.cpu()) and torch.equal(d, d0.cpu())
    with pytest.raises(qwlib.QwError):
        index.autotune(Qh, 5, reps=0)
    index.free()


@pytest.mark.parametrize("batch", [0, 7])
@pytest.mark.parametrize("path", ["levels", "bitmap"])
def test_graph_mode_equals_host_loop(qwlib, cuda, batch, path):
    """Same kernels, driven by a conditional WHILE node instead of the host:
    identical ids, distances and statistics; graphs cached across calls."""
    import torch
    wl = workloads.make_workload("mix10k_d32", seed=23, n=40_000, nq=45, n_clusters=30)
    index = _index(qwlib, cuda, wl, v=50, bitmaps=True)
    Q = torch.from_numpy(wl.Q).to(cuda)
    ref = index.query(Q, 10, stats=True, path="levels", batch=batch)
    index.profile(reset=True)
    for _ in range(3):
        got = index.query(Q, 10, stats=True, path=path, batch=batch, graph=True)
        for a, b2 in zip(ref, got):
            assert torch.equal(a, b2)
    prof = index.profile(reset=True)
    levels_run = ref[2][:, 0].max().item()
    assert prof["launches"]["level"] >= 3 * levels_run
    with pytest.raises(qwlib.QwError):
        index.query(Q, 10, path="cluster", graph=True)
    index.free()


def test_bitmap_path_needs_bitmaps_and_reports_their_size(qwlib, cuda):
    """QW_PATH_BITMAP on an index without bitmaps is an argument error; with
    them, qw_index_info.bitmap_bytes equals the documented layout: per
    projection and tile, one 4 KiB bitmap per level-L bucket, levels up to the
    first c^L above the span."""
    import torch
    wl = workloads.make_workload("mix10k_d32", seed=24, n=40_000, nq=10, n_clusters=30)
    plain = _index(qwlib, cuda, wl, v=50)
    Q = torch.from_numpy(wl.Q).to(cuda)
    with pytest.raises(qwlib.QwError):
        plain.query(Q, 5, path="bitmap")
    assert plain.info.bitmap_bytes == 0
    for c in (2, 3):
        index = _index(qwlib, cuda, wl, v=50, bitmaps=True, c=c)
        o, span, _, _ = index.export()
        nT = index.info.n_tiles
        want = 0
        for sp in span.tolist():
            R = 1
            while True:
                want += sp // R + 1
                if R > sp:
                    break
                R *= c
        assert index.info.bitmap_bytes == want * nT * 4096
        a = index.query(Q, 5, stats=True, path="levels")
        b2 = index.query(Q, 5, stats=True, path="bitmap")
        for x, y in zip(a, b2):
            assert torch.equal(x, y)
        index.free()
    plain.free()


@pytest.mark.parametrize("path", ["levels", "bitmap"])
def test_graph_cache_tells_batch_capacities_apart(qwlib, cuda, path):
    """Batches of 20 then of 10: both calls have a 10-query batch, carved from
    workspace laid out for different capacities; each must get its own graph."""
    import torch
    wl = workloads.make_workload("mix10k_d32", seed=25, n=20_000, nq=30, n_clusters=20)
    index = _index(qwlib, cuda, wl, v=40, bitmaps=True)
    Q = torch.from_numpy(wl.Q).to(cuda)
    ref = index.query(Q, 8, stats=True, path="levels")
    for batch in (20, 10, 20, 30):
        got = index.query(Q, 8, stats=True, path=path, batch=batch, graph=True,
                          profile=batch == 10)
        for a, b2 in zip(ref, got):
            assert torch.equal(a, b2)
    index.free()
