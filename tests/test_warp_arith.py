"""Two claims about the distance kernels' warp arithmetic, checked by emulating
the 32 lanes in numpy (float32, as the kernels compute):

* the multi-row butterfly of the BF16 pre-filter (rows_sum: at each of the
  first log2 R xor steps a lane keeps half of its row values and adds its
  partner's half) leaves in lane l exactly the float32 sum the per-row
  butterfly (warp_sum: xor 16, 8, 4, 2, 1 on one value) gives for row
  l >> (5 - log2 R), bit for bit;
* the two-pass radix bound of the k-th smallest key (block_kth_upper: 11-bit
  bins of bits 31..21, then 20..10, the result with bits 9..0 set) has at least
  k keys at or below it and, for non-negative floats, exceeds the k-th
  smallest by less than 2^-13 of it."""
import numpy as np
import pytest

F32 = np.float32


def warp_sum(v):
    """v: (32,) float32 per lane -> (32,) after xor 16, 8, 4, 2, 1."""
    v = v.astype(F32)
    for off in (16, 8, 4, 2, 1):
        v = (v + v[np.arange(32) ^ off]).astype(F32)
    return v


def rows_sum(a):
    """a: (32, R) float32 per lane and row -> (32,) as the kernel's rows_sum."""
    lanes = np.arange(32)
    R = a.shape[1]
    vals = a.astype(F32).copy()
    h, off = R // 2, 16
    while h >= 1:
        up = (lanes & off) != 0
        new = np.empty((32, h), dtype=F32)
        for i in range(h):
            lo, hi = vals[:, i], vals[:, i + h]
            send = np.where(up, lo, hi)
            keep = np.where(up, hi, lo)
            new[:, i] = (keep + send[lanes ^ off]).astype(F32)
        vals = new
        h //= 2
        off //= 2
    v = vals[:, 0]
    off = 16 // R
    while off >= 1:
        v = (v + v[lanes ^ off]).astype(F32)
        off //= 2
    return v


@pytest.mark.parametrize("R", [2, 4, 8])
def test_rows_sum_equals_per_row_warp_sums(R):
    rng = np.random.default_rng(R)
    for trial in range(200):
        scale = np.exp(rng.uniform(-30, 30, (1, R)))
        a = (rng.standard_normal((32, R)) * scale).astype(F32)
        got = rows_sum(a)
        for lane in range(32):
            row = lane >> (5 - int(np.log2(R)))
            want = warp_sum(a[:, row])[0]
            assert got[lane].tobytes() == F32(want).tobytes(), (R, trial, lane)


def kth_upper(v, kk):
    """block_kth_upper on uint32 keys v: two 11-bit radix passes."""
    prefix, mask = 0, 0
    for shift in (21, 10):
        sel = (v & mask) == prefix
        hist = np.bincount(((v[sel] >> shift) & 2047).astype(np.int64), minlength=2048)
        cum = np.cumsum(hist)
        b = int(np.searchsorted(cum, kk))  # first bin whose cumulative count reaches kk
        kk -= int(cum[b - 1]) if b > 0 else 0
        prefix |= b << shift
        mask |= 2047 << shift
    return prefix | 1023


@pytest.mark.parametrize("case", ["spread", "ties", "near_equal", "tiny_and_huge", "zeros"])
def test_kth_upper_bound(case):
    rng = np.random.default_rng(len(case))
    for trial in range(50):
        n = int(rng.integers(11, 4097))
        if case == "spread":
            x = np.exp(rng.uniform(-20, 20, n))
        elif case == "ties":
            x = rng.choice(np.exp(rng.uniform(-3, 3, 5)), n)
        elif case == "near_equal":
            x = 7.0 * (1 + rng.uniform(0, 1e-5, n))
        elif case == "tiny_and_huge":
            x = np.where(rng.random(n) < 0.5, 1e-30, 1e30) * rng.uniform(1, 2, n)
        else:
            x = np.where(rng.random(n) < 0.9, 0.0, rng.uniform(0, 1, n))
        f = x.astype(F32)
        keys = f.view(np.uint32).astype(np.uint64)
        kk = int(rng.integers(1, n + 1))
        U = kth_upper(keys, kk)
        assert int((keys <= U).sum()) >= kk
        kth = np.sort(f)[kk - 1]
        u = np.array([U], dtype=np.uint32).view(F32)[0]
        assert u >= kth
        if kth > 0:
            assert (float(u) - float(kth)) < 2.0 ** -13 * float(kth) * (1 + 1e-6)
        else:
            assert u < 1e-38  # the smallest bin above zero: a subnormal
