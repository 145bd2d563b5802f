"""Pins for the CPU oracle: checks against what the paper and mathematics fix,
none of which re-types the oracle's own code.

Each pin takes an ``oracle.Oracle`` and returns a list of failure messages
(empty = pinned).  ``test_oracle_pins`` runs them on the real oracle;
``test_oracle_mutants`` plants plausible mistakes in copies of the oracle
source and checks that some pin fails for each.
"""
from __future__ import annotations

import math
from collections import defaultdict

import numpy as np

import workloads


def _small(seed=0, n=2000, nq=30, d=16, m=12, n_clusters=20, **kw):
    return workloads.make_workload("mix10k_d32", seed=seed, n=n, nq=nq, d=d, m=m,
                                   n_clusters=n_clusters, **kw)


# ---------------------------------------------------------------- Eq. 1
def pin_collision_prob_quadrature(orc):
    """Eq. 1's integral evaluated by adaptive quadrature equals the closed form."""
    from scipy.integrate import quad
    fails = []
    for w in (0.5, 2.719, 4.0, 10.0):
        for r in (0.1, 0.5, 1.0, 2.0, 3.0, 8.0, 40.0):
            f = lambda t: (1.0 / r) * (2.0 / math.sqrt(2.0 * math.pi)) * math.exp(-t * t / (2 * r * r)) * (1.0 - t / w)
            want, err = quad(f, 0.0, w, epsabs=1e-14, epsrel=1e-13)
            got = orc.collision_prob(r, w)
            if not abs(got - want) <= 1e-10:
                fails.append(f"P(r={r}, w={w}) = {got}, quadrature {want}")
    return fails


def pin_collision_prob_limits(orc):
    """P -> 1 as r -> 0, P decreases in r, and r P(r) / w -> 1/sqrt(2 pi)."""
    fails = []
    w = 4.0
    if not orc.collision_prob(1e-4, w) > 1.0 - 1e-3:
        fails.append("P(r) does not tend to 1 for small r")
    rs = np.linspace(0.05, 50.0, 400)
    ps = np.array([orc.collision_prob(float(r), w) for r in rs])
    if not np.all(np.diff(ps) < 0):
        fails.append("P(r) not strictly decreasing")
    big = 1e5
    if not abs(big * orc.collision_prob(big, w) / w - 1.0 / math.sqrt(2.0 * math.pi)) < 1e-4:
        fails.append("large-r asymptote of P(r) wrong")
    return fails


# ---------------------------------------------------------------- threshold
def pin_threshold_balance(orc):
    """alpha solves ln(1/delta)/(p1-a)^2 = ln(2/beta)/(a-p2)^2 (found here by a
    root finder), lies in (p2, p1), and l = ceil(alpha m)."""
    from scipy.optimize import brentq
    fails = []
    delta = math.exp(-1.0)
    for w, c, n, v, m in ((4.0, 2, 10_000, 100, 16), (4.0, 2, 1_000_000, 100, 64),
                          (2.719, 2, 54_387, 100, 64), (4.0, 3, 4_000_000, 100, 64)):
        p1, p2 = orc.collision_prob(1.0, w), orc.collision_prob(float(c), w)
        beta = v / n
        f = lambda a: math.log(1 / delta) / (p1 - a) ** 2 - math.log(2 / beta) / (a - p2) ** 2
        root = brentq(f, p2 + 1e-9, p1 - 1e-9, xtol=1e-15)
        got = orc.alpha(p1, p2, beta, delta)
        if not abs(got - root) < 1e-10:
            fails.append(f"alpha {got} != balance root {root} for {(w, c, n, v)}")
        if not (p2 < got < p1):
            fails.append("alpha outside (p2, p1)")
        l = orc.threshold(m, w, c, n, v, delta)
        if l != min(m, max(1, math.ceil(root * m))):
            fails.append(f"l = {l} for alpha {root}, m {m}")
    return fails


# ---------------------------------------------------------------- hashing
def pin_hash_exact_sum(orc):
    """Bucket ids equal floor((fsum_j a_ij x_j + b_i) / w) with the exactly
    rounded sum (products of float32 are exact in double); both sides agree
    wherever the value is not within 1e-9 of an integer, and such cases are
    rare."""
    fails = []
    rng = np.random.default_rng(1)
    for d, m, w, scale in ((16, 12, 4.0, 3.0), (7, 5, 0.7, 10.0), (64, 9, 2.719, 1.0)):
        X = (rng.standard_normal((300, d)) * scale).astype(np.float32)
        A = rng.standard_normal((m, d)).astype(np.float32)
        b = (rng.random(m) * w).astype(np.float32)
        H = orc.hash(X, A, b, w)
        close = 0
        for r in range(X.shape[0]):
            for i in range(m):
                t = math.fsum(float(A[i, j]) * float(X[r, j]) for j in range(d))
                u = (t + float(b[i])) / float(w)
                if abs(u - round(u)) < 1e-9:
                    close += 1
                    continue
                if H[r, i] != math.floor(u):
                    fails.append(f"h[{r},{i}] = {H[r, i]}, exact floor {math.floor(u)}")
                    break
        if close > 3:
            fails.append(f"{close} values within 1e-9 of a bucket edge")
        if not (H < 0).any():
            fails.append("sample has no negative bucket ids (floor vs trunc untested)")
    return fails[:5]


# ---------------------------------------------------------------- index
def pin_index_sorted_arrays(orc):
    """o = column minimum, span = max - min, sorted arrays = lexsort by
    (bid, id) of the anchored ids."""
    fails = []
    wl = _small(seed=3)
    H = orc.hash(wl.X, wl.A, wl.b, 4.0)
    ix = orc.build_index(H)
    if not np.array_equal(ix.o, H.min(axis=0)):
        fails.append("anchors are not the column minima")
    if not np.array_equal(ix.span, H.max(axis=0) - H.min(axis=0)):
        fails.append("spans wrong")
    B = H - H.min(axis=0)
    for i in range(H.shape[1]):
        order = np.lexsort((np.arange(H.shape[0]), B[:, i]))
        if not (np.array_equal(ix.sbid[i], B[order, i]) and np.array_equal(ix.sid[i], order)):
            fails.append(f"sorted arrays of projection {i} differ from lexsort")
    return fails


def _level_counts_numpy(B, g, R):
    """#col at radius R by the bucket form floor(bid / R) == floor(g / R)."""
    return (np.floor_divide(B, R) == np.floor_divide(g, R)[None, :]).sum(axis=1)


def pin_collision_counts(orc):
    """Counts equal the bucket-form count, the sorted-array range counts equal
    the number of bids in the level bucket, and levels nest (counts never
    decrease from R to cR, so C_R is contained in C_cR)."""
    fails = []
    wl = _small(seed=4, nq=12)
    H = orc.hash(wl.X, wl.A, wl.b, 4.0)
    HQ = orc.hash(wl.Q, wl.A, wl.b, 4.0)
    ix = orc.build_index(H)
    B = (H - ix.o).astype(np.int64)
    for q in range(HQ.shape[0]):
        g = HQ[q].astype(np.int64) - ix.o
        prev = None
        for R in (1, 2, 4, 8, 16, 64, 1024):
            col = orc.collision_counts(ix, HQ[q], R)
            want = _level_counts_numpy(B, g, R)
            if not np.array_equal(col, want):
                fails.append(f"counts differ at q={q} R={R}")
                return fails
            if prev is not None and np.any(col < prev):
                fails.append(f"counts decrease from R/2 to R={R}")
            prev = col
            for i in range(0, H.shape[1], 5):
                beta = g[i] // R
                cnt = orc.range_count(ix, i, beta * R, beta * R + R - 1)
                if cnt != int(np.count_nonzero(B[:, i] // R == beta)):
                    fails.append(f"range count wrong at q={q} i={i} R={R}")
    # the nesting of buckets itself: floor(floor(x/R)/c) == floor(x/(cR))
    x = np.arange(-5000, 5000)
    for R, c in ((1, 2), (3, 2), (4, 3), (8, 2)):
        if not np.array_equal(np.floor_divide(np.floor_divide(x, R), c), np.floor_divide(x, R * c)):
            fails.append("bucket nesting identity fails")
    return fails


def pin_single_projection_is_e2lsh(orc):
    """m = 1, l = 1: the first level's candidates are exactly the points in the
    query's E2LSH bucket (a hash table keyed by bucket id)."""
    fails = []
    wl = _small(seed=5, m=1, nq=40)
    H = orc.hash(wl.X, wl.A, wl.b, 4.0)
    HQ = orc.hash(wl.Q, wl.A, wl.b, 4.0)
    table = defaultdict(set)
    for j, h in enumerate(H[:, 0]):
        table[int(h)].add(j)
    ix = orc.build_index(H)
    for q in range(HQ.shape[0]):
        col = orc.collision_counts(ix, HQ[q], 1)
        got = set(np.nonzero(col >= 1)[0].tolist())
        if got != table.get(int(HQ[q, 0]), set()):
            fails.append(f"query {q}: level-1 candidates differ from the E2LSH bucket")
    return fails


def _exact_knn_numpy(X, Q, k):
    Xd, Qd = X.astype(np.float64), Q.astype(np.float64)
    out_ids = np.empty((Q.shape[0], k), np.int64)
    out_d = np.empty((Q.shape[0], k))
    for q in range(Q.shape[0]):
        dist = np.sqrt(((Xd - Qd[q]) ** 2).sum(axis=1))
        order = np.lexsort((np.arange(X.shape[0]), dist))[:k]
        out_ids[q], out_d[q] = order, dist[order]
    return out_ids, out_d


def pin_bruteforce(orc):
    """The oracle's exact k-NN equals a numpy exact k-NN (ties by id)."""
    wl = _small(seed=6, n=1500, nq=20)
    ids, dist = orc.bruteforce(wl.X, wl.Q, 9)
    want_ids, want_d = _exact_knn_numpy(wl.X, wl.Q, 9)
    fails = []
    if not np.array_equal(ids, want_ids):
        fails.append("brute-force ids differ from numpy exact k-NN")
    if not np.allclose(dist, want_d, rtol=1e-12, atol=0):
        fails.append("brute-force distances differ")
    return fails


def pin_v_ge_n_exact(orc):
    """v >= n and queries equal to data rows: no level reaches k + v, the last
    level holds every point, and the result is the exact k-NN."""
    fails = []
    wl = _small(seed=7, n=400, nq=1, n_clusters=5)
    Q = wl.X[:15].copy()
    H = orc.hash(wl.X, wl.A, wl.b, 4.0)
    HQ = orc.hash(Q, wl.A, wl.b, 4.0)
    ix = orc.build_index(H)
    res = orc.query(wl.X, ix, Q, HQ, k=8, v=400, l=9)
    want_ids, want_d = _exact_knn_numpy(wl.X, Q, 8)
    if not np.array_equal(res["ids"], want_ids):
        fails.append("v >= n does not give the exact k-NN")
    if not np.all(res["stats"][:, 4] == 3) or not np.all(res["stats"][:, 2] == 400):
        fails.append("v >= n does not end with every point a candidate")
    return fails


def pin_workload_semantics(orc):
    """For every query of a small workload, rebuild the answer from the
    definition with numpy: the first level (R = 1, c, c^2, ...) whose candidate
    count reaches k + v, or the first R above every bucket id; the kept set =
    previous level's candidates + best (count desc, id asc) up to k + v; the
    result = k nearest kept by exact distance (ties by id)."""
    fails = []
    for seed, k, v, n, c in ((8, 5, 12, 1500, 2), (9, 10, 100, 3000, 2), (10, 3, 7, 900, 3)):
        wl = _small(seed=seed, n=n, nq=25, m=10)
        X, Q = wl.X, wl.Q
        Q[:3] += 60.0  # some queries outside the data
        H = orc.hash(X, wl.A, wl.b, 4.0)
        HQ = orc.hash(Q, wl.A, wl.b, 4.0)
        ix = orc.build_index(H)
        l = 7
        res = orc.query(X, ix, Q, HQ, k=k, v=v, l=l, c=c)
        B = (H - ix.o).astype(np.int64)
        cap = k + v
        for q in range(Q.shape[0]):
            g = HQ[q].astype(np.int64) - ix.o
            top = max(int(ix.span.max()), int(g.max()))
            R, prev_set, levels = 1, np.zeros(n, bool), 0
            while True:
                levels += 1
                col = _level_counts_numpy(B, g, R)
                cand = col >= l
                if cand.sum() >= cap:
                    term = 2
                    break
                if R > top:
                    term = 3
                    break
                prev_set = cand
                R *= c
            st = res["stats"][q]
            if (st[0], st[1], st[2], st[4], st[7]) != (levels, R, int(cand.sum()), term,
                                                       int(prev_set.sum())):
                fails.append(f"seed {seed} q {q}: stats {st[[0, 1, 2, 4, 7]]} want "
                             f"{(levels, R, int(cand.sum()), term, int(prev_set.sum()))}")
                continue
            idx = np.nonzero(cand)[0]
            order = np.lexsort((idx, -col[idx], ~prev_set[idx]))
            kept = idx[order][:cap]
            if set(kept.tolist()) != set(res["cand_ids"][q][res["cand_ids"][q] >= 0].tolist()):
                fails.append(f"seed {seed} q {q}: kept candidate set differs")
                continue
            dist = np.sqrt(((X[kept].astype(np.float64) - Q[q].astype(np.float64)) ** 2).sum(1))
            o2 = np.lexsort((kept, dist))[:k]
            want = np.full(k, -1, np.int64)
            want[: o2.size] = kept[o2]
            if not np.array_equal(res["ids"][q], want):
                fails.append(f"seed {seed} q {q}: top-k differs")
            if o2.size < k and not np.all(np.isinf(res["dists"][q][o2.size:])):
                fails.append("padding distances are not inf")
    return fails[:6]


def pin_t3_fixpoint(orc):
    """A query stopped because R passed every bucket id has C_R = all points if
    at least l of its anchored ids g_i are >= 0, else no point."""
    fails = []
    wl = _small(seed=12, n=800, nq=20)
    Q = wl.Q.copy()
    Q[:10] += 200.0
    Q[10:] -= 200.0
    H = orc.hash(wl.X, wl.A, wl.b, 4.0)
    HQ = orc.hash(Q, wl.A, wl.b, 4.0)
    ix = orc.build_index(H)
    l = 6
    res = orc.query(wl.X, ix, Q, HQ, k=5, v=2000, l=l)
    for q in range(Q.shape[0]):
        st = res["stats"][q]
        if st[4] != 3:
            fails.append(f"query {q} did not stop by the radius rule")
            continue
        g = HQ[q].astype(np.int64) - ix.o
        want = 800 if int((g >= 0).sum()) >= l else 0
        if st[2] != want:
            fails.append(f"query {q}: |C_R| = {st[2]}, expected {want}")
    return fails


def pin_ratio_invariant(orc):
    """Returned distances are ascending and the i-th is >= the true i-th
    nearest distance (the c-k-ANN ratio of Section 3 is >= 1)."""
    fails = []
    wl = _small(seed=13, n=2500, nq=30)
    H = orc.hash(wl.X, wl.A, wl.b, 4.0)
    HQ = orc.hash(wl.Q, wl.A, wl.b, 4.0)
    ix = orc.build_index(H)
    res = orc.query(wl.X, ix, wl.Q, HQ, k=10, v=20, l=8)
    _, true_d = _exact_knn_numpy(wl.X, wl.Q, 10)
    d = res["dists"]
    fin = np.isfinite(d)
    if np.any(d[fin] < true_d[fin] * (1 - 1e-12)):
        fails.append("a returned distance is below the true i-th distance")
    if np.any(np.diff(np.where(fin, d, np.inf), axis=1) < 0):
        fails.append("returned distances not ascending")
    return fails


def pin_duplicates_tie_by_id(orc):
    """Exact duplicate rows have equal distances; the smaller id comes first."""
    fails = []
    wl = _small(seed=14, n=600, nq=10)
    X = np.repeat(wl.X[:150], 4, axis=0)
    H = orc.hash(X, wl.A, wl.b, 4.0)
    HQ = orc.hash(wl.Q, wl.A, wl.b, 4.0)
    ix = orc.build_index(H)
    res = orc.query(X, ix, wl.Q, HQ, k=8, v=600, l=4)
    want_ids, _ = _exact_knn_numpy(X, wl.Q, 8)
    if not np.array_equal(res["ids"], want_ids):
        fails.append("ties between duplicates not broken by smaller id")
    return fails


def pin_hand_worked_golden(orc):
    """A workload of 10 points, 3 projections and 3 queries worked out by hand
    (tests/golden/hand_worked_query.json): bucket ids, anchors and spans,
    every level's collision counts, the stop level (the k + v bound of
    Section 3.1, or the radius past every bucket), the kept candidates in
    truncation order, the statistics and the top-k."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "hand_worked_query.json")
    with open(path) as fh:
        g = json.load(fh)
    p = g["params"]
    X = np.array(g["X"], np.float32)
    Q = np.array(g["Q"], np.float32)
    A = np.array(g["A"], np.float32)
    b = np.array(g["b"], np.float32)
    fails = []
    H = orc.hash(X, A, b, p["w"])
    HQ = orc.hash(Q, A, b, p["w"])
    if not np.array_equal(H, np.array(g["H"])) or not np.array_equal(HQ, np.array(g["HQ"])):
        return ["bucket ids differ from the hand-worked ones"]
    ix = orc.build_index(H)
    if ix.o.tolist() != g["o"] or ix.span.tolist() != g["span"]:
        fails.append(f"anchors {ix.o.tolist()} / spans {ix.span.tolist()} differ")
    for qi, q in enumerate(g["queries"]):
        for lv in q["levels"]:
            col = orc.collision_counts(ix, HQ[qi], lv["R"])
            if col.tolist() != lv["col"]:
                fails.append(f"query {qi}, R = {lv['R']}: counts {col.tolist()} want {lv['col']}")
    res = orc.query(X, ix, Q, HQ, k=p["k"], v=p["v"], l=p["l"], c=p["c"])
    cap = p["k"] + p["v"]
    for qi, q in enumerate(g["queries"]):
        st = res["stats"][qi].tolist()
        if st != q["stats"]:
            fails.append(f"query {qi}: stats {st} want {q['stats']}")
        kept = res["cand_ids"][qi].tolist()
        want_kept = q["kept"] + [-1] * (cap - len(q["kept"]))
        if kept != want_kept:
            fails.append(f"query {qi}: kept {kept} want {want_kept} (truncation order)")
        kcol = res["cand_col"][qi][: len(q["kept"])].tolist()
        if kcol != q["kept_col"]:
            fails.append(f"query {qi}: kept counts {kcol} want {q['kept_col']}")
        if res["ids"][qi].tolist() != q["ids"]:
            fails.append(f"query {qi}: ids {res['ids'][qi].tolist()} want {q['ids']}")
        want_d = [math.sqrt(x) if x is not None else math.inf for x in q["sqdists"]]
        if not np.array_equal(res["dists"][qi], np.array(want_d)):
            fails.append(f"query {qi}: dists {res['dists'][qi].tolist()} want {want_d}")
    for qi, q in enumerate(g["queries"]):
        for t, i in enumerate(q["kept"]):
            if orc.sqdist(X[i], Q[qi]) != q["kept_sqdist"][t]:
                fails.append(f"query {qi}: squared distance to {i} differs")
    # the same points with one probe on each side
    mp = g["multi_probe"]
    P = mp["probes"]
    Qp = np.array(mp["Q"], np.float32)
    HQp = orc.hash(Qp, A, b, p["w"])
    if not np.array_equal(HQp, np.array(mp["HQ"])):
        return fails + ["multi-probe query bucket ids differ"]
    for qi, q in enumerate(mp["queries"]):
        for lv in q["levels"]:
            col = orc.collision_counts(ix, HQp[qi], lv["R"], probes=P)
            if col.tolist() != lv["col"]:
                fails.append(f"probe query {qi}, R = {lv['R']}: counts {col.tolist()}")
    res = orc.query(X, ix, Qp, HQp, k=p["k"], v=p["v"], l=p["l"], c=p["c"], probes=P)
    for qi, q in enumerate(mp["queries"]):
        if res["stats"][qi].tolist() != q["stats"]:
            fails.append(f"probe query {qi}: stats {res['stats'][qi].tolist()} want {q['stats']}")
        kept = res["cand_ids"][qi].tolist()
        if kept != q["kept"] + [-1] * (cap - len(q["kept"])):
            fails.append(f"probe query {qi}: kept {kept} want {q['kept']}")
        if res["ids"][qi].tolist() != q["ids"]:
            fails.append(f"probe query {qi}: ids {res['ids'][qi].tolist()} want {q['ids']}")
        want_d = [math.sqrt(x) for x in q["sqdists"]]
        if not np.array_equal(res["dists"][qi], np.array(want_d)):
            fails.append(f"probe query {qi}: dists differ")
    return fails


def pin_multi_probe_semantics(orc):
    """Multi-probe restated independently: an object collides on projection i
    when its level-R bucket index floor(bid / R) is within P of the query's
    (a distance between bucket indices, not the oracle's bid range); the level
    loop stops at the first level with |C_R| >= k + v or past every bucket
    index the query can still reach (for P > 0 also R > -g_i); the kept set
    and the result follow as without probes.  Queries far below and above the
    data are included, and C_R grows with P."""
    fails = []
    for seed, P, c in ((21, 1, 2), (22, 2, 2), (23, 1, 3)):
        wl = _small(seed=seed, n=1200, nq=20, m=10)
        X, Q = wl.X, wl.Q
        # queries below the data on every projection (A dq = -300: bucket ids
        # far under the anchors), and above it
        shift = np.linalg.pinv(wl.A.astype(np.float64)) @ np.full(wl.A.shape[0], 300.0)
        Q[:3] = (Q[:3] - shift).astype(np.float32)
        Q[3:5] = (Q[3:5] + shift).astype(np.float32)
        H = orc.hash(X, wl.A, wl.b, 4.0)
        HQ = orc.hash(Q, wl.A, wl.b, 4.0)
        ix = orc.build_index(H)
        k, v, l = 5, 25, 7
        res = orc.query(X, ix, Q, HQ, k=k, v=v, l=l, c=c, probes=P)
        res0 = orc.query(X, ix, Q, HQ, k=k, v=v, l=l, c=c)
        B = (H - ix.o).astype(np.int64)
        cap = k + v
        for q in range(Q.shape[0]):
            g = HQ[q].astype(np.int64) - ix.o
            top = max(int(ix.span.max()), int(g.max()), int((-g).max()))
            R, prev_set, levels = 1, np.zeros(X.shape[0], bool), 0
            while True:
                levels += 1
                col = (np.abs(np.floor_divide(B, R) - np.floor_divide(g, R)[None, :]) <= P).sum(1)
                cand = col >= l
                if cand.sum() >= cap:
                    term = 2
                    break
                if R > top:
                    term = 3
                    break
                prev_set = cand
                R *= c
            st = res["stats"][q]
            if (st[0], st[1], st[2], st[4], st[7]) != (levels, R, int(cand.sum()), term,
                                                       int(prev_set.sum())):
                fails.append(f"seed {seed} q {q}: stats {st[[0, 1, 2, 4, 7]]} want "
                             f"{(levels, R, int(cand.sum()), term, int(prev_set.sum()))}")
                continue
            idx = np.nonzero(cand)[0]
            order = np.lexsort((idx, -col[idx], ~prev_set[idx]))
            kept = idx[order][:cap]
            if kept.tolist() != res["cand_ids"][q][res["cand_ids"][q] >= 0].tolist():
                fails.append(f"seed {seed} q {q}: kept candidates differ")
            col0 = orc.collision_counts(ix, HQ[q], R)
            colP = orc.collision_counts(ix, HQ[q], R, probes=P)
            if np.any(colP < col0):
                fails.append(f"seed {seed} q {q}: a count falls when probes are added")
        if np.all(res["stats"][:, 0] == res0["stats"][:, 0]):
            fails.append(f"seed {seed}: probes never change the stop level")
    return fails[:6]


# ---------------------------------------------------------------- QALSH (Section 2)
def pin_qalsh_hand_worked(orc):
    """The ten hand-worked points with QALSH's query-centred buckets
    (tests/golden/hand_worked_query.json, section "qalsh"): every level's
    counts, with points exactly on an interval end counted as inside; the stop
    level, the kept candidates in truncation order, the statistics and the
    top-k, all worked out by hand."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "hand_worked_query.json")
    with open(path) as fh:
        g = json.load(fh)
    p = g["params"]
    qa = g["qalsh"]
    X = np.array(g["X"], np.float32)
    A = np.array(g["A"], np.float32)
    Q = np.array(qa["Q"], np.float32)
    P = orc.project(X, A)
    PQ = orc.project(Q, A)
    if not np.array_equal(P, X[:, :3].astype(np.float64)):
        return ["projections of the hand-worked points differ from their first three coordinates"]
    fails = []
    for qi, q in enumerate(qa["queries"]):
        for lv in q["levels"]:
            col = orc.qalsh_counts(P, PQ[qi], qa["w"], lv["R"])
            if col.tolist() != lv["col"]:
                fails.append(f"qalsh query {qi}, R = {lv['R']}: counts {col.tolist()} want {lv['col']}")
    res = orc.qalsh_query(X, P, Q, PQ, w=qa["w"], k=p["k"], v=p["v"], l=p["l"], c=p["c"])
    cap = p["k"] + p["v"]
    for qi, q in enumerate(qa["queries"]):
        st = res["stats"][qi].tolist()
        if st != q["stats"]:
            fails.append(f"qalsh query {qi}: stats {st} want {q['stats']}")
        kept = res["cand_ids"][qi].tolist()
        if kept != q["kept"] + [-1] * (cap - len(q["kept"])):
            fails.append(f"qalsh query {qi}: kept {kept} want {q['kept']} (truncation order)")
        if res["cand_col"][qi][: len(q["kept"])].tolist() != q["kept_col"]:
            fails.append(f"qalsh query {qi}: kept counts differ")
        if res["ids"][qi].tolist() != q["ids"]:
            fails.append(f"qalsh query {qi}: ids {res['ids'][qi].tolist()} want {q['ids']}")
        want_d = [math.sqrt(x) for x in q["sqdists"]]
        if not np.array_equal(res["dists"][qi], np.array(want_d)):
            fails.append(f"qalsh query {qi}: dists {res['dists'][qi].tolist()} want {want_d}")
    return fails


def pin_qalsh_prob_quadrature(orc):
    """QALSH's collision probability: for a projection a with i.i.d. N(0, 1)
    entries, a . (o - q) is N(0, r^2), and the probability that it lands in a
    bucket of width w centred on q is the normal density integrated over
    [-w/2, w/2] -- evaluated here by adaptive quadrature -- and, sampled, the
    fraction of Gaussian projections within w/2."""
    from scipy.integrate import quad
    fails = []
    for w in (0.5, 2.719, 4.0):
        for r in (0.05, 0.5, 1.0, 2.0, 7.5, 40.0):
            dens = lambda t: math.exp(-t * t / (2 * r * r)) / (r * math.sqrt(2 * math.pi))
            want, _ = quad(dens, -w / 2, w / 2, epsabs=1e-14, epsrel=1e-13)
            got = orc.qalsh_prob(r, w)
            if not abs(got - want) <= 1e-10:
                fails.append(f"qalsh P(r={r}, w={w}) = {got}, quadrature {want}")
    rng = np.random.default_rng(5)
    o = np.zeros(16)
    q = np.zeros(16)
    q[0] = 1.5                                            # r = 1.5
    proj = rng.standard_normal((200000, 16)) @ (o - q)
    frac = float(np.mean(np.abs(proj) <= 2.719 / 2))
    want = orc.qalsh_prob(1.5, 2.719)
    if not abs(frac - want) <= 5 * math.sqrt(want * (1 - want) / 200000):
        fails.append(f"sampled collision rate {frac} vs {want}")
    return fails


def pin_qalsh_threshold_balance(orc):
    """QALSH's l: the balance point of the two Hoeffding bounds (root finder)
    between p2 = erf(w / (2 sqrt2 c)) and p1 = erf(w / (2 sqrt2)), taken from
    scipy's erf, and l = ceil(alpha m)."""
    from scipy.optimize import brentq
    from scipy.special import erf
    fails = []
    delta = math.exp(-1.0)
    for w, c, n, v, m in ((2.719, 2, 10_000, 100, 16), (2.719, 2, 1_000_000, 700, 64),
                          (1.0, 3, 4_000_000, 100, 64)):
        p1 = float(erf(w / (2 * math.sqrt(2.0))))
        p2 = float(erf(w / (2 * math.sqrt(2.0) * c)))
        beta = v / n
        f = lambda a: math.log(1 / delta) / (p1 - a) ** 2 - math.log(2 / beta) / (a - p2) ** 2
        root = brentq(f, p2 + 1e-9, p1 - 1e-9, xtol=1e-15)
        l = orc.qalsh_threshold(m, w, c, n, v, delta)
        if l != min(m, max(1, math.ceil(root * m))):
            fails.append(f"qalsh l = {l} for alpha {root}, m {m}")
    return fails


def pin_qalsh_project_exact(orc):
    """a_i . v on small integers is exact in any summation order: the
    projections equal the integer matrix product."""
    rng = np.random.default_rng(8)
    V = rng.integers(-50, 50, size=(300, 33)).astype(np.float32)
    A = rng.integers(-9, 9, size=(11, 33)).astype(np.float32)
    want = (V.astype(np.int64) @ A.astype(np.int64).T).astype(np.float64)
    got = orc.project(V, A)
    return [] if np.array_equal(got, want) else ["projections differ from the integer product"]


def pin_qalsh_v_ge_n_exact(orc):
    """With k + v > n no level can reach the k + v bound, so the query runs
    until every interval holds all the data (the radius rule), keeps every
    object and returns the exact k nearest neighbours; the stop radius is the
    first R = c^j with w R / 2 >= max_i max_o |p_i(o) - p_i(q)|."""
    fails = []
    wl = _small(seed=31, n=300, nq=12, d=8, m=6, n_clusters=5)
    P = orc.project(wl.X, wl.A)
    PQ = orc.project(wl.Q, wl.A)
    res = orc.qalsh_query(wl.X, P, wl.Q, PQ, w=2.719, k=7, v=400, l=3, c=2)
    want_ids, want_d = _exact_knn_numpy(wl.X, wl.Q, 7)
    if not np.array_equal(res["ids"], want_ids):
        fails.append("v >= n: ids are not the exact neighbours")
    if not np.allclose(res["dists"], want_d, rtol=1e-12, atol=0):
        fails.append("v >= n: distances differ from the exact ones")
    for qi in range(wl.Q.shape[0]):
        spread = np.abs(P - PQ[qi][None, :]).max()
        R = 1
        while 2.719 * R / 2 < spread:
            R *= 2
        st = res["stats"][qi]
        if st[4] != 3 or st[3] != 300 or st[1] != R:
            fails.append(f"v >= n, query {qi}: term {st[4]}, kept {st[3]}, R {st[1]} want 3, 300, {R}")
    return fails


def pin_qalsh_semantics(orc):
    """The query-centred level loop restated with numpy broadcasting on small
    workloads (c = 2 and 3): per level, counts of projections within w R / 2,
    the k + v stop, the radius rule, the kept set in truncation order and the
    statistics."""
    fails = []
    for seed, c in ((41, 2), (42, 3)):
        wl = _small(seed=seed, n=1500, nq=16, m=10)
        P = orc.project(wl.X, wl.A)
        PQ = orc.project(wl.Q, wl.A)
        w, k, v, l = 2.719, 5, 30, 6
        res = orc.qalsh_query(wl.X, P, wl.Q, PQ, w=w, k=k, v=v, l=l, c=c)
        cap = k + v
        for q in range(wl.Q.shape[0]):
            dev = np.abs(P - PQ[q][None, :])
            spread = dev.max()
            R, prev_set, levels, full = 1, np.zeros(P.shape[0], bool), 0, 0
            while True:
                levels += 1
                inside = dev <= w * R / 2
                col = inside.sum(1)
                full += int(inside.sum())
                cand = col >= l
                if cand.sum() >= cap:
                    term = 2
                    break
                if w * R / 2 >= spread:
                    term = 3
                    break
                prev_set = cand
                R *= c
            want = (levels, R, int(cand.sum()), min(int(cand.sum()), cap), term,
                    int(inside.sum()), full, int(prev_set.sum()))
            if tuple(res["stats"][q].tolist()) != want:
                fails.append(f"seed {seed} q {q}: stats {res['stats'][q].tolist()} want {want}")
                continue
            idx = np.nonzero(cand)[0]
            kept = idx[np.lexsort((idx, -col[idx], ~prev_set[idx]))][:cap]
            if kept.tolist() != res["cand_ids"][q][res["cand_ids"][q] >= 0].tolist():
                fails.append(f"seed {seed} q {q}: kept candidates differ")
    return fails[:6]


ALL_PINS = [pin_collision_prob_quadrature, pin_collision_prob_limits, pin_threshold_balance,
            pin_hash_exact_sum, pin_index_sorted_arrays, pin_collision_counts,
            pin_single_projection_is_e2lsh, pin_bruteforce, pin_v_ge_n_exact,
            pin_workload_semantics, pin_t3_fixpoint, pin_ratio_invariant,
            pin_duplicates_tie_by_id, pin_hand_worked_golden, pin_multi_probe_semantics,
            pin_qalsh_hand_worked, pin_qalsh_prob_quadrature, pin_qalsh_threshold_balance,
            pin_qalsh_project_exact,
            pin_qalsh_v_ge_n_exact, pin_qalsh_semantics]
