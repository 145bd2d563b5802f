"""The BF16 pre-filter's distance bounds, restated on the CPU in float32.

The pre-filter (rerank_bf16_kernel) drops a candidate only when the lower
bound of its distance exceeds the k-th smallest upper bound, so the result is
exact as long as every bound holds.  The GPU parity tests show identical ids
on the benchmark's data; here the kernel's float32 arithmetic (the build's
residual copy and per-row constants, the per-lane FMA chains and butterfly
sums in the kernel's element order, and the bound formula with its margins)
is replayed step by step in numpy on cases chosen to strain the bound:
queries on top of a candidate, at the group mean and far away, large
coordinates with tiny residuals, and every load form of the kernel (d a
multiple of 256, of 4, and neither).  The square roots are moved 2 ulp in the
unfavourable direction (rsqrtf's error).  Every exact squared distance must
lie within [lo^2, hi^2]."""
import numpy as np
import pytest

F32 = np.float32
U = 2.0 ** -24


def bf16(x):
    """float32 -> BF16 (round to nearest even), returned as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def fma(a, b, c):
    """float32 fused multiply-add (one rounding of the exact a * b + c; the
    float64 product of two float32 values is exact)."""
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(F32) \
        if isinstance(a, np.ndarray) or isinstance(c, np.ndarray) else \
        F32(np.float64(a) * np.float64(b) + np.float64(c))


def lane_order(d, chunk):
    """Element indices each of the 32 lanes visits, in order: lane l takes the
    chunks l, l + 32, ... of `chunk` consecutive elements."""
    nch = d // chunk
    order = []
    for lane in range(32):
        idx = []
        for c in range(lane, nch, 32):
            idx.extend(range(c * chunk, c * chunk + chunk))
        order.append(idx)
    return order


def warp_dot(terms_a, terms_b, order, sub=None):
    """Per-lane FMA chains then the xor butterfly (16, 8, 4, 2, 1), all in
    float32.  terms_*: (N, d) float32; with `sub`, the chain sums
    (a - sub)^2 instead of a * b.  Returns (N,) float32."""
    n = terms_a.shape[0]
    acc = np.zeros((32, n), dtype=F32)
    for lane in range(32):
        s = np.zeros(n, dtype=F32)
        for e in order[lane]:
            if sub is None:
                s = fma(terms_a[:, e], terms_b[:, e], s)
            else:
                t = (terms_a[:, e] - sub[:, e]).astype(F32)
                s = fma(t, t, s)
        acc[lane] = s
    for off in (16, 8, 4, 2, 1):
        acc = (acc + acc[np.arange(32) ^ off]).astype(F32)
    return acc[0]


def f32_up(x64):
    """float64 -> float32 rounded toward +infinity."""
    f = x64.astype(F32)
    low = f.astype(np.float64) < x64
    f[low] = np.nextafter(f[low], F32(np.inf))
    return f


def build_copy(X):
    """The residual BF16 copy of rows X (n x d float32, one group of at most
    128 rows per call): C_g, r~, R >= |r|, C_g . r~ and |r~|^2."""
    Cg = bf16((X.astype(np.float64).mean(axis=0)).astype(F32))
    r = (X - Cg[None, :]).astype(F32)
    rt = bf16(r)
    R = f32_up(np.sqrt((r.astype(np.float64) ** 2).sum(axis=1)) * (1 + 1e-12))
    cr = (rt.astype(np.float64) @ Cg.astype(np.float64)).astype(F32)
    rr = (rt.astype(np.float64) ** 2).sum(axis=1).astype(F32)
    return Cg, rt, R, cr, rr


def bounds(q, Cg, rt, R, cr, rr, d):
    """The kernel's lower and upper bounds of |q - x|^2 for one group's rows."""
    n = rt.shape[0]
    form = 8 if d % 256 == 0 else (4 if d % 4 == 0 else 1)
    Q = np.broadcast_to(q, (n, d)).astype(F32)
    P = warp_dot(Q, rt, lane_order(d, form))
    gform = 8 if d % 8 == 0 else 1
    S = warp_dot(q[None, :], None, lane_order(d, gform), sub=Cg[None, :])[0]
    qq = warp_dot(q[None, :], q[None, :], lane_order(d, 1))[0]
    rho = ((d + 31) // 32 + 12) * 5.9604644775390625e-08 * 1.02
    rho_s = gam = F32(rho * 1.01)
    qn = F32(np.sqrt(qq, dtype=F32) * F32(1.01))
    two = F32(2.0)
    a = ((F32(S) - two * P).astype(F32) + two * cr).astype(F32)
    a = (a + rr).astype(F32)
    Rt = (R * F32(1.004)).astype(F32)
    Cn = F32(qn + F32(np.sqrt(F32(S), dtype=F32)) * F32(1.01))
    absum = (F32(S) + two * np.abs(P) + two * np.abs(cr) + rr).astype(F32)
    E2 = (F32(1.01) * (rho_s * F32(S) + two * gam * qn * Rt + F32(2.0 ** -23) * Cn * Rt
                       + F32(2.0 ** -24) * rr + F32(3.03 * 2.0 ** -24) * absum)).astype(F32)
    tlo = (np.maximum(a - E2, F32(0)) * F32(1 - 2.0 ** -20)).astype(F32)
    thi = ((a + E2) * F32(1 + 2.0 ** -20)).astype(F32)
    # rsqrtf is within 2 ulp: move both roots the unfavourable way
    wlo = (np.sqrt(tlo, dtype=F32) * F32(1 + 2.0 ** -22)).astype(F32)
    whi = (np.sqrt(thi, dtype=F32) * F32(1 - 2.0 ** -22)).astype(F32)
    e = (F32(F32(1.001) * F32(2.0 ** -8 + 2.0 ** -15)) * R).astype(F32)
    lo = np.maximum(wlo * F32(1 - 2.0 ** -18) - e * F32(1 + 2.0 ** -18), F32(0)).astype(F32)
    hi = ((whi + e) * F32(1 + 2.0 ** -18)).astype(F32)
    return (lo * lo * F32(1 - 2.0 ** -18)).astype(F32), (hi * hi * F32(1 + 2.0 ** -18)).astype(F32)


CASES = [
    # d, centre scale, residual scale, query kind
    (128, 30.0, 1.0, "member"),
    (128, 30.0, 1.0, "mean"),
    (128, 30.0, 1.0, "far"),
    (256, 5.0, 0.05, "member"),
    (256, 1e4, 1e-2, "member"),
    (256, 1e4, 1e-2, "far"),
    (512, 30.0, 3.0, "member"),
    (512, 30.0, 3.0, "exact"),
    (100, 30.0, 1.0, "member"),
    (37, 100.0, 0.5, "member"),
    (37, 100.0, 0.5, "exact"),
    (512, 1e-3, 1e-3, "far"),
]


@pytest.mark.parametrize("d,cscale,rscale,kind", CASES)
def test_bounds_hold(d, cscale, rscale, kind):
    rng = np.random.default_rng(d * 1000 + int(rscale * 100) + len(kind))
    centre = (rng.standard_normal(d) * cscale).astype(F32)
    X = (centre[None, :] + rng.standard_normal((128, d)) * rscale).astype(F32)
    Cg, rt, R, cr, rr = build_copy(X)
    for trial in range(6):
        j = int(rng.integers(0, 128))
        if kind == "member":
            q = (X[j] + rng.standard_normal(d) * rscale * 1e-3).astype(F32)
        elif kind == "exact":
            q = X[j].copy()
        elif kind == "mean":
            q = (Cg + rng.standard_normal(d) * rscale * 1e-2).astype(F32)
        else:
            q = (rng.standard_normal(d) * cscale * 3).astype(F32)
        lo2, hi2 = bounds(q, Cg, rt, R, cr, rr, d)
        true = ((X.astype(np.float64) - q.astype(np.float64)) ** 2).sum(axis=1)
        assert np.all(lo2.astype(np.float64) <= true), (kind, d, np.max(lo2 - true))
        assert np.all(true <= hi2.astype(np.float64)), (kind, d, np.max(true - hi2))


def test_bounds_tight_at_the_bf16_worst_case():
    """The residual's BF16 rounding at its worst: every component of r sits on
    a rounding midpoint (1 + 2^-8 times a power of two, rounded down to even),
    so |r - r~| is 2^-8 |r| / (1 + 2^-8), and the queries are placed along and
    against that error, where | |q - x| - |q - C_g - r~| | equals it.  The
    bounds must hold there and sit within 1e-3 of the exact distance (a
    bound that took the rounding error as 2^-9 |r| would fail here)."""
    d = 256
    rng = np.random.default_rng(11)
    C = bf16((rng.standard_normal(d) * 4).astype(F32))
    sgn = np.where(rng.random(d) < 0.5, -1.0, 1.0).astype(F32)
    r = (sgn * F32(2.0 ** -4) * F32(1 + 2.0 ** -8)).astype(F32)
    # rows C + r and C - r: the group mean is C exactly
    X = np.stack([C + r, C - r] * 64).astype(F32)
    Cg, rt, R, cr, rr = build_copy(X)
    assert np.array_equal(Cg, C) and np.array_equal(rt[0], sgn * F32(2.0 ** -4))
    delta = (r - rt[0]).astype(np.float64)
    dhat = delta / np.linalg.norm(delta)
    t = 0.5
    for direction in (1.0, -1.0):
        q = (C.astype(np.float64) + rt[0] + direction * t * dhat).astype(F32)
        lo2, hi2 = bounds(q, Cg, rt, R, cr, rr, d)
        true = ((X[0].astype(np.float64) - q.astype(np.float64)) ** 2).sum()
        assert lo2[0] <= true <= hi2[0]
        # the side the rounding error works against is within 1e-3
        gap = (true - lo2[0]) if direction > 0 else (hi2[0] - true)
        assert gap <= 1e-3 * true, (direction, gap / true)


def test_bounds_separate_near_and_far():
    """On a compact group with a query near one member, the near member's
    upper bound lies below the far members' lower bounds (the filter can
    drop them)."""
    d = 256
    rng = np.random.default_rng(7)
    centre = (rng.standard_normal(d) * 30).astype(F32)
    X = (centre[None, :] + rng.standard_normal((128, d)) * 0.5).astype(F32)
    Cg, rt, R, cr, rr = build_copy(X)
    q = (X[3] + rng.standard_normal(d) * 1e-3).astype(F32)
    lo2, hi2 = bounds(q, Cg, rt, R, cr, rr, d)
    others = np.delete(np.arange(128), 3)
    assert hi2[3] < np.min(lo2[others])


def test_bf16_rounding_matches_torch():
    """The numpy BF16 rounding used above is torch's round-to-nearest-even."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(4096) * np.exp(rng.uniform(-20, 20, 4096))).astype(F32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(bf16(x), ref)
