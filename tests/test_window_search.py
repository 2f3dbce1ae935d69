"""The dense generator's 32-bit boundary search, emulated on the CPU in the
same IEEE single-precision steps, against exact integer arithmetic.

Within a block's 32-column window [d, d + 31] (d >= 1024 columns from the
axis), the zone boundary with threshold S sits at a = d + k, k the smallest
k >= 0 with k (k + 2d) >= D, D = S - dj^2 - d^2 (Sec. 2.2: the boundary
radius is the smallest integer distance whose squared radius reaches the
threshold).  The kernel estimates k as ceil(fl(fl(D) * fl(0.5 / d))) and
corrects it by two steps up and one down in 32-bit integers.  This checks
that the correction always lands on the exact k over d from 1024 to 2^23 and
every k the window can hold."""
import math

import numpy as np


def window_k(D: np.ndarray, d: int) -> np.ndarray:
    inv2d = np.float32(0.5) / np.float32(d)            # 0.5f / (float)d, one rounding
    two_d = 2 * d
    k = np.ceil(D.astype(np.float32) * inv2d).astype(np.int64)  # __float2int_ru of a rounded product
    k = np.maximum(k, 0)
    k += (k * (k + two_d) < D).astype(np.int64)
    k += (k * (k + two_d) < D).astype(np.int64)
    k -= ((k > 0) & ((k - 1) * (k - 1 + two_d) >= D)).astype(np.int64)
    assert np.all(np.abs(k * (k + two_d)) < 2 ** 31)  # the kernel's products fit int32
    return k


def exact_k(D: int, d: int) -> int:
    if D <= 0:
        return 0
    k = math.isqrt(d * d + D) - d
    while k * (k + 2 * d) < D:
        k += 1
    while k > 0 and (k - 1) * (k - 1 + 2 * d) >= D:
        k -= 1
    return k


def test_window_search_is_exact():
    rng = np.random.default_rng(5)
    ds = sorted({1024, 1025, 2047, 4096, 65535, 1 << 20, (1 << 23) - 1}
                | {int(x) for x in rng.integers(1024, 1 << 23, 200)})
    checked = 0
    for d in ds:
        Ds = [-5, 0]
        for k in range(0, 32):
            lo = (k - 1) * (k - 1 + 2 * d) + 1 if k > 0 else -3
            hi = k * (k + 2 * d)
            Ds += [lo, hi, (lo + hi) // 2]
            Ds += [int(x) for x in rng.integers(lo, hi + 1, 8)]
        D = np.array(Ds, dtype=np.int64)
        got = window_k(D, d)
        want = np.array([exact_k(int(x), d) for x in Ds])
        assert np.array_equal(got, want), (d, D[got != want][:5], got[got != want][:5], want[got != want][:5])
        checked += len(Ds)
    assert checked > 50_000


def _ceil_sqrt46_from(a: np.ndarray, t: np.ndarray) -> np.ndarray:
    """The kernel's exact integer corrections after a = (uint32) r."""
    a = a.astype(np.int64)
    a += (a * a < t).astype(np.int64)
    a += (a * a < t).astype(np.int64)
    a += (a * a < t).astype(np.int64)
    a -= ((a > 0) & ((a - 1) * (a - 1) >= t)).astype(np.int64)
    return a


def test_ceil_sqrt46_corrections_cover_the_approximate_root():
    """The row walker (and the block generator near the axis) takes
    a = ceil(sqrt(t)), t < 2^46, from r = sqrt.approx(fl(t)) and three steps up
    and one down in integers.  fl(t) carries a relative error of 2^-24 (kept
    here: t goes through float32), the approximate root one below 2^-23; with
    r off by -2 or +1 units of 2^-23 relative (and rounded to float32), the
    corrections still give the exact ceiling up to t = 2^46, where a is near
    2^23.  (Off by +1.8 units they would not, for a few a near 2^23: the
    margin upward is below two units.)"""
    rng = np.random.default_rng(9)
    ts = np.concatenate([
        rng.integers(1, 1 << 46, 200_000, dtype=np.int64),
        np.array([1, 2, 3, 4, 5, (1 << 46) - 1], dtype=np.int64),
        np.array([x * x for x in rng.integers(1, 1 << 23, 20_000)] +
                 [x * x + 1 for x in rng.integers(1, 1 << 23, 20_000)] +
                 [x * x - 1 for x in rng.integers(2, 1 << 23, 20_000)], dtype=np.int64),
    ])
    want = np.array([math.isqrt(int(t) - 1) + 1 for t in ts])  # ceil(sqrt(t)) for t >= 1
    root = np.sqrt(ts.astype(np.float32).astype(np.float64))
    for rel in (-2.0 ** -22, -2.0 ** -23, 0.0, 2.0 ** -23):
        r = (root * (1 + rel)).astype(np.float32)
        got = _ceil_sqrt46_from(np.floor(r).astype(np.uint32), ts)
        assert np.array_equal(got, want), rel


def _zone_of(s: int, K64: int, thr, nthr: int) -> int:
    """The device's zone_of in exact integers: the high word of the 64 x 64-bit
    product s K64, and the threshold table where the product lies within 2^-17
    below or 2^-28 above an integer (the low word's window)."""
    prod = s * K64
    z, lo = prod >> 64, prod & ((1 << 64) - 1)
    if lo < (1 << 36) or lo >= 0xFFFF800000000000:
        if z >= 1 and thr[z - 1] > s:
            z -= 1
        elif z < nthr and thr[z] <= s:
            z += 1
    return z


def test_device_zone_rule_equals_the_ieee_rule():
    """Reading 2's exactness argument, checked on the CPU: the fixed-point
    product with its threshold-table window gives floor(fl(s kappa_L)) for
    every s tried -- random s over the disc and s at, just below and just
    above sampled thresholds, on config 1, the 5 m plate, and the grids of
    Table 1 (L = 16) and Table 5 (L = 2), up to s near 2^45.6.  The table is
    the library's own (fzp_zone_thresholds) and K64 = floor(kappa_L 2^64)."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import __graft_entry__
    __graft_entry__.build()
    import paper_2609_01978_gb300 as fzp
    rng = np.random.default_rng(3)
    lam1, lam2 = 632.8e-9, 532e-9
    cases = [
        dict(D=4e-3, f=20e-3, lam=lam1),
        dict(D=5.0, f=25.0, lam=lam1),
        dict(D=1.0, f=5.0, lam=lam2, levels=16, dx=lam2 * 5.0 / 0.5 / 64),
        dict(D=5.0, f=25.0, lam=lam2, levels=2, dx=lam2 * 25.0 / 2.5 / 16),
    ]
    for kw in cases:
        kw = dict(kw, M=256, pitch=kw["lam"] * 5 / 8)
        q = fzp.plan_query(**kw)
        thr = [int(x) for x in fzp.zone_thresholds(**kw)]
        L = kw.get("levels", 0)
        rate = q["kappa"] * (0.5 * L if L >= 2 else 1.0)
        K64 = math.floor(math.ldexp(rate, 64))
        dx2, R2 = q["dx"] ** 2, q["R"] ** 2
        sR = int(R2 // dx2)
        while float(sR + 1) * dx2 <= R2:
            sR += 1
        samples = [0, 1, sR, sR - 1] + [int(x) for x in rng.integers(0, sR, 20_000)]
        for m in rng.integers(1, len(thr) - 1, 5_000):
            S = thr[m - 1]
            samples += [S - 1, S, S + 1]
        in_window = 0
        for s in samples:
            if 0 <= s <= sR:
                assert _zone_of(s, K64, thr, len(thr)) == math.floor(float(s) * rate), (kw, s)
                lo = (s * K64) & ((1 << 64) - 1)
                in_window += lo < (1 << 36) or lo >= 0xFFFF800000000000
        assert in_window > 100, in_window  # the table's window was exercised
        assert sR > (1 << 40) or kw["D"] < 1
