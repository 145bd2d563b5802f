"""Seeded synthetic inputs for the LSH query-workload path.

This module is the one piece shared by the CUDA path's callers (tests, bench) and
by the oracle's callers: it draws random numbers and nothing else. It holds none
of the method's arithmetic (no hashing, no bucketing, no distances).

What it draws, and why (the paper's datasets are not available, so these stand
in for them, see the design notes):

* data: a Gaussian mixture, centres uniform in [-10, 10]^d, isotropic sigma = 1
  around each centre; cluster sizes uniform-random or Zipf-skewed;
* queries: taken from dense regions of the data (the paper draws its workload
  queries from dense regions, Section 6.2): a random data row of a chosen
  cluster plus isotropic Gaussian noise;
* the LSH family's own random draws (Section 3): projection vectors
  a_i ~ N(0, I_d) and offsets b_i ~ U[0, w). The method draws these; here they
  are drawn once and passed as inputs to both implementations.

All arrays are float32, row-major, C-contiguous. Every draw comes from
``numpy.random.default_rng(seed)`` streams derived from one seed, so the same
seed gives the same bytes on x86 and Arm.
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict
from typing import Optional

import numpy as np

__all__ = [
    "WorkloadSpec",
    "SPECS",
    "Workload",
    "make_data",
    "make_queries",
    "make_projections",
    "make_workload",
]


@dataclass(frozen=True)
class WorkloadSpec:
    """Shape of one synthetic workload.

    ``query_noise`` is the standard deviation of the isotropic noise added to a
    data row to make a query; a tuple gives a mix in equal shares.
    ``query_clusters`` limits queries to that many clusters (workload locality);
    0 means any cluster.  ``zipf`` > 0 makes both cluster sizes and cluster
    popularity Zipf-distributed with that exponent.
    """

    name: str
    n: int
    d: int
    n_clusters: int
    nq: int
    k: int
    m: int
    w: float = 4.0
    c: int = 2
    v: int = 100
    query_clusters: int = 0
    query_noise: tuple = (0.1,)
    zipf: float = 0.0
    sigma: float = 1.0
    center_range: float = 10.0

    def as_dict(self):
        return asdict(self)


# The five workloads of the method's hot path, smallest first.  The first is
# small enough for the oracle to finish in seconds; the second is the one the
# benchmark times.
SPECS = {
    "mix10k_d32": WorkloadSpec("mix10k_d32", n=10_000, d=32, n_clusters=50,
                               nq=100, k=10, m=16),
    "mix1m_d128": WorkloadSpec("mix1m_d128", n=1_000_000, d=128, n_clusters=1000,
                               nq=10_000, k=100, m=64, query_clusters=100),
    "zipf1m_d256": WorkloadSpec("zipf1m_d256", n=1_000_000, d=256, n_clusters=2000,
                                nq=50_000, k=10, m=64, zipf=1.1),
    "mix4m_d512": WorkloadSpec("mix4m_d512", n=4_000_000, d=512, n_clusters=4000,
                               nq=20_000, k=50, m=64),
    "mix10m_d128": WorkloadSpec("mix10m_d128", n=10_000_000, d=128, n_clusters=10_000,
                                nq=100_000, k=10, m=64, query_noise=(0.05, 0.5, 2.0)),
}


@dataclass
class Workload:
    spec: WorkloadSpec
    X: np.ndarray          # n x d float32
    labels: np.ndarray     # n int32, cluster of each row
    Q: np.ndarray          # nq x d float32
    q_src: np.ndarray      # nq int64, data row each query was drawn from
    A: np.ndarray          # m x d float32, projection vectors
    b: np.ndarray          # m float32, offsets in [0, w)
    seed: int = 0
    extra: dict = field(default_factory=dict)
    Q_train: Optional[np.ndarray] = None  # n_train x d: earlier queries of the same workload


def _streams(seed: int):
    ss = np.random.SeedSequence(seed)
    return [np.random.default_rng(s) for s in ss.spawn(4)]


def _zipf_weights(count: int, s: float) -> np.ndarray:
    ranks = np.arange(1, count + 1, dtype=np.float64)
    wts = ranks ** (-s)
    return wts / wts.sum()


def make_data(n: int, d: int, n_clusters: int, rng: np.random.Generator, *,
              zipf: float = 0.0, sigma: float = 1.0, center_range: float = 10.0,
              chunk: int = 1 << 18):
    """Gaussian mixture: returns (X float32 n x d, labels int32 n, centres)."""
    centers = rng.uniform(-center_range, center_range,
                          size=(n_clusters, d)).astype(np.float32)
    if zipf > 0.0:
        p = _zipf_weights(n_clusters, zipf)
        labels = rng.choice(n_clusters, size=n, p=p).astype(np.int32)
    else:
        labels = rng.integers(0, n_clusters, size=n, dtype=np.int32)
    X = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        noise = rng.standard_normal((e - s, d), dtype=np.float32)
        noise *= np.float32(sigma)
        X[s:e] = centers[labels[s:e]] + noise
    return X, labels, centers


def make_queries(X: np.ndarray, labels: np.ndarray, nq: int, rng: np.random.Generator, *,
                 n_clusters: int, query_clusters: int = 0, zipf: float = 0.0,
                 noise=(0.1,), pool=None, return_pool: bool = False):
    """Queries from dense regions: a data row of a chosen cluster + noise.

    Returns (Q float32 nq x d, src int64 nq), plus the cluster pool the queries
    were limited to (None when unlimited) if ``return_pool``.  Passing ``pool``
    reuses an earlier draw's pool: more queries of the same workload.
    """
    n, d = X.shape
    present = np.unique(labels)
    if query_clusters and query_clusters < present.size:
        if pool is None:
            pool = rng.choice(present, size=query_clusters, replace=False)
        qlab = pool[rng.integers(0, pool.size, size=nq)]
    elif zipf > 0.0:
        p = _zipf_weights(n_clusters, zipf)
        qlab = rng.choice(n_clusters, size=nq, p=p)
        # a Zipf label may name an empty cluster on tiny inputs: remap to present
        miss = ~np.isin(qlab, present)
        qlab[miss] = present[rng.integers(0, present.size, size=int(miss.sum()))]
    else:
        qlab = present[rng.integers(0, present.size, size=nq)]
    order = np.argsort(labels, kind="stable")
    sorted_lab = labels[order]
    starts = np.searchsorted(sorted_lab, qlab, side="left")
    ends = np.searchsorted(sorted_lab, qlab, side="right")
    pick = starts + (rng.random(nq) * (ends - starts)).astype(np.int64)
    pick = np.minimum(pick, ends - 1)
    src = order[pick].astype(np.int64)
    sig = np.asarray(noise, dtype=np.float32)
    qsig = sig[np.arange(nq) % sig.size] if sig.size > 1 else np.full(nq, sig[0], np.float32)
    Q = X[src] + rng.standard_normal((nq, d), dtype=np.float32) * qsig[:, None]
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    if return_pool:
        return Q, src, pool
    return Q, src


def make_projections(m: int, d: int, w: float, rng: np.random.Generator):
    """The LSH family's random draws (Section 3): a ~ N(0, I_d), b ~ U[0, w)."""
    A = rng.standard_normal((m, d), dtype=np.float32)
    b = (rng.random(m, dtype=np.float64) * w).astype(np.float32)
    b = np.minimum(b, np.nextafter(np.float32(w), np.float32(0)))  # keep b < w in fp32
    return np.ascontiguousarray(A), np.ascontiguousarray(b)


def make_workload(spec, seed: int = 0, *, n: Optional[int] = None, nq: Optional[int] = None,
                  n_train: int = 0, **overrides) -> Workload:
    """Build a whole workload from a spec name or a ``WorkloadSpec``.

    ``n``/``nq`` and any other field can be overridden to get a smaller case
    with the same structure.  ``n_train`` > 0 also draws that many training
    queries (``Q_train``): the same data, cluster pool and noise mix as ``Q``,
    from a separate random stream, so ``Q`` does not depend on ``n_train``.
    """
    if isinstance(spec, str):
        spec = SPECS[spec]
    fields = spec.as_dict()
    if n is not None:
        fields["n"] = n
    if nq is not None:
        fields["nq"] = nq
    fields.update(overrides)
    spec = WorkloadSpec(**fields)
    r_data, r_query, r_proj, r_extra = _streams(seed)
    X, labels, _ = make_data(spec.n, spec.d, spec.n_clusters, r_data, zipf=spec.zipf,
                             sigma=spec.sigma, center_range=spec.center_range)
    Q, src, pool = make_queries(X, labels, spec.nq, r_query, n_clusters=spec.n_clusters,
                                query_clusters=spec.query_clusters, zipf=spec.zipf,
                                noise=spec.query_noise, return_pool=True)
    A, b = make_projections(spec.m, spec.d, spec.w, r_proj)
    Q_train = None
    if n_train > 0:
        Q_train, _ = make_queries(X, labels, n_train, r_extra, n_clusters=spec.n_clusters,
                                  query_clusters=spec.query_clusters, zipf=spec.zipf,
                                  noise=spec.query_noise, pool=pool)
    return Workload(spec=spec, X=X, labels=labels, Q=Q, q_src=src, A=A, b=b, seed=seed,
                    extra={"query_pool": pool}, Q_train=Q_train)
