"""The seeded input generators: deterministic, right shapes, the structure
the workloads call for."""
import numpy as np

import workloads


def test_deterministic_and_shapes():
    a = workloads.make_workload("mix10k_d32", seed=0)
    b = workloads.make_workload("mix10k_d32", seed=0)
    c = workloads.make_workload("mix10k_d32", seed=1)
    for x, y in ((a.X, b.X), (a.Q, b.Q), (a.A, b.A), (a.b, b.b)):
        assert x.dtype == np.float32 and x.flags.c_contiguous
        assert np.array_equal(x, y)
    assert not np.array_equal(a.X, c.X)
    s = a.spec
    assert a.X.shape == (s.n, s.d) and a.Q.shape == (s.nq, s.d)
    assert a.A.shape == (s.m, s.d) and a.b.shape == (s.m,)


def test_offsets_in_range():
    wl = workloads.make_workload("mix10k_d32", seed=3, m=500)
    assert np.all(wl.b >= 0) and np.all(wl.b < wl.spec.w)


def test_queries_near_their_source_rows():
    wl = workloads.make_workload("mix10k_d32", seed=2)
    dev = np.linalg.norm(wl.Q - wl.X[wl.q_src], axis=1)
    # noise sigma 0.1 in 32 dimensions: about 0.1 * sqrt(32)
    assert 0.3 < np.median(dev) < 0.9


def test_query_locality():
    wl = workloads.make_workload("mix1m_d128", seed=0, n=50_000, nq=2000)
    labs = np.unique(wl.labels[wl.q_src])
    assert labs.size <= wl.spec.query_clusters


def test_zipf_skew():
    wl = workloads.make_workload("zipf1m_d256", seed=0, n=40_000, nq=4000, d=8)
    counts = np.bincount(wl.labels, minlength=wl.spec.n_clusters)
    assert counts[0] > 20 * np.median(counts[counts > 0])
    qcounts = np.bincount(wl.labels[wl.q_src], minlength=wl.spec.n_clusters)
    assert qcounts[0] == qcounts.max()


def test_mixed_noise_thirds():
    wl = workloads.make_workload("mix10m_d128", seed=0, n=20_000, nq=300, n_clusters=50)
    dev = np.linalg.norm(wl.Q - wl.X[wl.q_src], axis=1) / np.sqrt(wl.spec.d)
    assert abs(np.median(dev[0::3]) - 0.05) < 0.02
    assert abs(np.median(dev[1::3]) - 0.5) < 0.1
    assert abs(np.median(dev[2::3]) - 2.0) < 0.3


def test_training_queries_same_pool_and_independent_of_count():
    a = workloads.make_workload("mix1m_d128", seed=4, n=30_000, nq=500)
    b = workloads.make_workload("mix1m_d128", seed=4, n=30_000, nq=500, n_train=2000)
    assert a.Q_train is None
    assert np.array_equal(a.Q, b.Q) and np.array_equal(a.X, b.X)
    assert b.Q_train.shape == (2000, b.spec.d) and b.Q_train.dtype == np.float32
    # the training queries sit in the same clusters as the workload's queries
    def near_label(Q):
        d2 = (b.X ** 2).sum(1)[None, :] - 2.0 * Q @ b.X.T
        return b.labels[d2.argmin(1)]
    pool = set(b.extra["query_pool"].tolist())
    assert set(b.labels[b.q_src].tolist()) <= pool
    assert set(near_label(b.Q_train[:300]).tolist()) <= pool
