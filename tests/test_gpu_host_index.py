"""Level bitmaps kept in pinned host memory (host_bitmaps): the kernels read
them directly from host memory (on GB300 the Grace memory over NVLink-C2C),
the paper's setting of an index on external storage.  Every bitmap-path
variant must still give the oracle's ids, distances, statistics and
candidate sets, and the index must report where its bitmaps live."""
import functools

import numpy as np
import pytest

import workloads
from test_gpu_parity import TILE, _check_candidates, _check_results

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def _case():
    import oracle
    orc = oracle.get()
    wl = workloads.make_workload("mix10k_d32", seed=41, n=2 * TILE + 3_007, nq=50, n_clusters=70)
    s = wl.spec
    l = orc.threshold(s.m, s.w, s.c, s.n, s.v)
    H = orc.hash(wl.X, wl.A, wl.b, s.w)
    HQ = orc.hash(wl.Q, wl.A, wl.b, s.w)
    ref = orc.query(wl.X, orc.build_index(H), wl.Q, HQ, k=s.k, v=s.v, l=l, c=s.c)
    return wl, l, ref


def test_host_bitmaps_match_oracle(qwlib, cuda):
    import torch
    wl, l, ref = _case()
    s = wl.spec
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)  # noqa: E731
    Q = t(wl.Q)
    index = qwlib.Index(t(wl.X), t(wl.A), t(wl.b), w=s.w, c=s.c, v=s.v, l=l, bitmaps=True,
                        host_bitmaps=True)
    info = index.info
    assert info.host_bytes > 0 and info.host_bytes == info.bitmap_bytes
    dev = qwlib.Index(t(wl.X), t(wl.A), t(wl.b), w=s.w, c=s.c, v=s.v, l=l, bitmaps=True)
    assert dev.info.host_bytes == 0
    assert index.info.device_bytes + info.bitmap_bytes == dev.info.device_bytes
    dev.free()
    for graph in (False, True):
        for loads in ("direct", "tma", "fused"):  # TMA reads host bitmaps directly too
            ids, dists, st = index.query(Q, s.k, stats=True, path="bitmap", graph=graph,
                                         loads=loads, order="signature", batch=17)
            cid, ccol, st2 = index.candidates(Q, s.k, path="bitmap", graph=graph, loads=loads)
            torch.cuda.synchronize()
            _check_results(ids.cpu().numpy(), dists.cpu().numpy(), ref["ids"], ref["dists"])
            assert np.array_equal(st.cpu().numpy(), ref["stats"])
            assert np.array_equal(st2.cpu().numpy(), ref["stats"])
            _check_candidates(cid.cpu().numpy(), ccol.cpu().numpy(), ref["cand_ids"],
                              ref["cand_col"])
    index.free()


def test_host_bitmaps_need_bitmaps(qwlib, cuda):
    import torch
    wl, l, _ = _case()
    s = wl.spec
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)  # noqa: E731
    with pytest.raises(qwlib.QwError):
        qwlib.Index(t(wl.X), t(wl.A), t(wl.b), w=s.w, c=s.c, v=s.v, l=l, host_bitmaps=True)
