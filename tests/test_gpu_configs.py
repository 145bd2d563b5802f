"""CUDA path vs the oracle on the shapes of the larger workloads (Zipf-skewed
1M x 256, 4M x 512 with k = 50, 10M x 128 with mixed query noise), scaled
down in n so the oracle finishes in seconds while the index still spans
several tiles and a ragged last tile.  Every path must give the oracle's ids,
distances (1e-5 relative), statistics and candidate sets."""
import functools

import numpy as np
import pytest

import workloads
from test_gpu_parity import TILE, _check_candidates, _check_results, _gpu_workload

pytestmark = pytest.mark.gpu

CONFIGS = {
    # name: (spec, overrides) -- n spans 2-3 tiles with a ragged tail
    "zipf1m_d256": dict(n=2 * TILE + 1_531, nq=40, n_clusters=120),
    "mix4m_d512": dict(n=TILE + 9_001, nq=24, n_clusters=60),
    "mix10m_d128": dict(n=2 * TILE + 4_321, nq=45, n_clusters=150),
}


@functools.lru_cache(maxsize=None)
def _case(name):
    import oracle
    orc = oracle.get()
    wl = workloads.make_workload(name, seed=17, **CONFIGS[name])
    s = wl.spec
    l = orc.threshold(s.m, s.w, s.c, s.n, s.v)
    H = orc.hash(wl.X, wl.A, wl.b, s.w)
    HQ = orc.hash(wl.Q, wl.A, wl.b, s.w)
    idx = orc.build_index(H)
    ref = orc.query(wl.X, idx, wl.Q, HQ, k=s.k, v=s.v, l=l, c=s.c)
    return wl, l, ref


@pytest.mark.parametrize("name", list(CONFIGS))
@pytest.mark.parametrize("path", ["levels", "bitmap_direct", "bitmap_graph", "bitmap_fused_graph"])
def test_config_parity(qwlib, cuda, name, path):
    wl, l, ref = _case(name)
    s = wl.spec
    g = _gpu_workload(qwlib, cuda, wl.X, wl.Q, wl.A, wl.b, w=s.w, k=s.k, v=s.v, l=l, c=s.c,
                      path=path, order="signature", batch=17)
    _check_results(g["ids"], g["dists"], ref["ids"], ref["dists"])
    assert np.array_equal(g["stats"], ref["stats"])
    assert np.array_equal(g["stats2"], ref["stats"])
    _check_candidates(g["cid"], g["ccol"], ref["cand_ids"], ref["cand_col"])
    g["index"].free()


@pytest.mark.parametrize("path", ["levels", "bitmap_direct_graph"])
def test_bf16_rerank_config_parity(qwlib, cuda, path):
    """The BF16 pre-filter on the 512-dimensional shape with k = 50 (the
    configuration the pre-filter is specified for): oracle ids and distances."""
    wl, l, ref = _case("mix4m_d512")
    s = wl.spec
    g = _gpu_workload(qwlib, cuda, wl.X, wl.Q, wl.A, wl.b, w=s.w, k=s.k, v=s.v, l=l, c=s.c,
                      path=path, order="signature", batch=17, rerank="bf16")
    _check_results(g["ids"], g["dists"], ref["ids"], ref["dists"])
    assert np.array_equal(g["stats"], ref["stats"])
    g["index"].free()
