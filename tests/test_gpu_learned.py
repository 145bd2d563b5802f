"""The learned start model: CUDA forward/backward against the FP64 reference,
training on the GPU, and the learned path against the plain one (same results,
fewer level passes)."""
import numpy as np
import pytest

import workloads
from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


def test_mlp_gradient_matches_fp64_reference(qwlib, cuda):
    import torch
    n_in, hidden, classes, n = 37, 48, 6, 203
    rng = np.random.default_rng(0)
    p = rng.standard_normal(M.param_count(n_in, hidden, classes)) * 0.3
    p = p.astype(np.float16).astype(np.float32)  # FP16-representable: the copies equal the masters
    X = rng.standard_normal((n, n_in)).astype(np.float32)
    y = rng.integers(0, classes, size=n).astype(np.int32)
    mlp = qwlib.Mlp(n_in, hidden, classes)
    mlp.set_params(p)
    loss, g = mlp.loss_grad(torch.from_numpy(X).to(cuda), torch.from_numpy(y).to(cuda))
    want_loss, want_g = M.loss_and_grad(p.astype(np.float64), X, y, n_in, hidden, classes)
    assert abs(loss - want_loss) <= 1e-5 * max(1.0, abs(want_loss))
    scale = np.abs(want_g).max()
    assert np.abs(g - want_g).max() <= 2e-5 * scale
    mlp.free()


def test_mlp_training_reduces_loss(qwlib, cuda):
    import torch
    rng = np.random.default_rng(1)
    n, n_in, classes = 4096, 16, 4
    centers = rng.standard_normal((classes, n_in)) * 3
    y = rng.integers(0, classes, size=n).astype(np.int32)
    X = (centers[y] + rng.standard_normal((n, n_in))).astype(np.float32)
    mlp = qwlib.Mlp(n_in, 64, classes)
    mlp.set_params(qwlib.mlp_init(n_in, 64, classes, seed=1))
    Xd, yd = torch.from_numpy(X).to(cuda), torch.from_numpy(y).to(cuda)
    loss0, _ = mlp.loss_grad(Xd, yd)
    loss = mlp.train(Xd, yd, epochs=20, batch=256, lr=2e-3)
    assert loss < 0.2 * loss0
    acc = (mlp.predict(Xd).argmax(1).cpu().numpy() == y).mean()
    assert acc > 0.9
    mlp.free()


@pytest.mark.parametrize("n_in,classes,n", [(192, 16, 1000), (576, 32, 300), (64, 16, 128)])
def test_mlp_tensor_core_forward(qwlib, cuda, n_in, classes, n):
    """The tcgen05 forward pass (FP16 activations, FP32 accumulation in tensor
    memory) against the FP64 definition and the SIMT pass, on ragged row
    counts (several 128-row tiles and a partial one) and the input widths of
    the 1M x 128, 4M x 512 and a minimal network."""
    import torch
    hidden = 256
    rng = np.random.default_rng(n_in + classes)
    p = rng.standard_normal(M.param_count(n_in, hidden, classes)) * (1.0 / np.sqrt(n_in))
    p = p.astype(np.float16).astype(np.float32)  # FP16-representable: the copies equal the masters
    X = rng.uniform(-1.5, 1.5, size=(n, n_in)).astype(np.float32)
    mlp = qwlib.Mlp(n_in, hidden, classes)
    mlp.set_params(p)
    Xd = torch.from_numpy(X).to(cuda)
    p_tc = mlp.predict(Xd, tensor_cores=True).cpu().numpy().astype(np.float64)
    p_simt = mlp.predict(Xd).cpu().numpy().astype(np.float64)
    want = M.predict_proba(p.astype(np.float64), X.astype(np.float64), n_in, hidden, classes)
    assert np.all(np.isfinite(p_tc))
    assert np.abs(p_simt - want).max() <= 1e-4
    assert np.abs(p_tc - want).max() <= 5e-3
    assert np.abs(p_tc.sum(axis=1) - 1.0).max() <= 1e-5
    # same decision for clear-cut rows
    clear = want.max(axis=1) > 0.6
    assert np.array_equal(p_tc[clear].argmax(1), want[clear].argmax(1))
    mlp.free()


def test_mlp_tensor_core_rejects_other_shapes(qwlib, cuda):
    import torch
    mlp = qwlib.Mlp(80, 256, 16)
    mlp.set_params(qwlib.mlp_init(80, 256, 16, seed=2))
    X = torch.zeros((10, 80), dtype=torch.float32, device=cuda)
    with pytest.raises(qwlib.QwError):
        mlp.predict(X, tensor_cores=True)
    mlp.free()


def _train_start_model(qwlib, cuda, index, Q_train, k, epochs=30):
    import torch
    Qt = torch.from_numpy(Q_train).to(cuda)
    _, _, st = index.query(Qt, k, stats=True, path="levels")
    labels = (st[:, 0] - 1).clamp(0, 15).to(torch.int32).contiguous()
    F = index.features(Qt)
    mlp = qwlib.Mlp(F.shape[1], 256, 16)
    mlp.set_params(qwlib.mlp_init(F.shape[1], 256, 16, seed=5))
    mlp.train(F, labels, epochs=epochs, batch=512, lr=1e-3)
    return mlp, labels


@pytest.mark.parametrize("w", [4.0, 0.4])
def test_learned_start_same_results_fewer_levels(qwlib, cuda, w):
    """w = 4 keeps every anchored bucket id below 256, w = 0.4 needs 16 bits:
    the bitmap path's recount reads rows of either width."""
    import torch
    spec = dict(n=60_000, d=48, m=32, n_clusters=120, query_clusters=30)
    wl = workloads.make_workload("mix1m_d128", seed=7, nq=600, n_train=3000, **spec)
    X, A, b = (torch.from_numpy(a).to(cuda) for a in (wl.X, wl.A, wl.b))
    index = qwlib.Index(X, A, b, w=w, v=300, bitmaps=True)
    mlp, labels = _train_start_model(qwlib, cuda, index, wl.Q_train, 20)
    index.set_start_model(mlp, eps=0.02)
    Q = torch.from_numpy(wl.Q).to(cuda)
    ids0, d0, st0 = index.query(Q, 20, stats=True, path="levels")
    index.profile(reset=True)
    ids1, d1, st1 = index.query(Q, 20, stats=True, start="learned")
    prof = index.profile(reset=True)
    assert torch.equal(ids0, ids1)
    assert torch.equal(d0, d1)
    assert torch.equal(st0, st1)
    assert prof["start_levels_skipped"] > 0
    # graph mode: the same loop driven on the device, the same counters
    ids3, d3, st3 = index.query(Q, 20, stats=True, start="learned", graph=True)
    prof3 = index.profile(reset=True)
    assert torch.equal(ids0, ids3) and torch.equal(d0, d3) and torch.equal(st0, st3)
    assert prof3["start_levels_skipped"] == prof["start_levels_skipped"]
    assert prof3["start_fallbacks"] == prof["start_fallbacks"]
    # bitmap path, host loop and graph mode: it starts at the predicted last
    # level itself (the previous level's candidates are recounted), so it
    # skips at least as many levels
    for graph, loads in ((False, "tma"), (True, "tma"), (False, "direct"), (True, "direct"),
                         (False, "fused"), (True, "fused")):
        ids5, d5, st5 = index.query(Q, 20, stats=True, start="learned", path="bitmap", graph=graph,
                                    loads=loads)
        prof5 = index.profile(reset=True)
        assert torch.equal(ids0, ids5) and torch.equal(d0, d5) and torch.equal(st0, st5)
        assert prof5["start_levels_skipped"] >= prof["start_levels_skipped"]
    # an over-eager model (eps close to 1) starts too late for many queries:
    # they are recomputed from level 0 and the results still match
    index.set_start_model(mlp, eps=0.999)
    ids2, d2, st2 = index.query(Q, 20, stats=True, start="learned")
    prof2 = index.profile(reset=True)
    assert torch.equal(ids0, ids2) and torch.equal(st0, st2)
    assert prof2["start_fallbacks"] > 0
    ids4, d4, st4 = index.query(Q, 20, stats=True, start="learned", graph=True)
    prof4 = index.profile(reset=True)
    assert torch.equal(ids0, ids4) and torch.equal(st0, st4)
    assert prof4["start_fallbacks"] == prof2["start_fallbacks"]
    # on the bitmap path an over-eager start leaves some queries whose
    # previous level already met the stop rule: they are answered again by the
    # bitmap path from level 0 (none of them needs the level path)
    for graph, loads in ((False, "direct"), (True, "direct"), (True, "tma"), (True, "fused")):
        ids6, d6, st6 = index.query(Q, 20, stats=True, start="learned", path="bitmap",
                                    graph=graph, loads=loads)
        prof6 = index.profile(reset=True)
        assert torch.equal(ids0, ids6) and torch.equal(d0, d6) and torch.equal(st0, st6)
        assert prof6["start_fallbacks"] > 0
        assert prof6["bitmap_fallbacks"] == 0
    index.free()
    mlp.free()
