"""The partitioned row pass's flat-plate generator (`chunk_bits`, form (a)),
emulated on the CPU in the same integer and IEEE single-precision steps,
against the zone rule evaluated column by column (Sec. 2.2: a sample is open
where its zone index is odd, or even for the positive-centred plate).

A thread makes the open bits of 16 neighbouring columns of a row.  Between
the chunk's two ends the zone index steps through the boundaries m in
(zn, zf]; boundary m lies at distance a_m = ceil(sqrt(S_m - dj^2)) from the
axis, found as a_m = d + k with k the smallest k with k (k + 2d) >= D,
D = S_m - dj^2 - d^2, from the FP32 estimate ceil(fl(fl(D) * fl(0.5 / d)))
and one integer step up and two down.  Checked here: that search against
exact integers for d from 128 to 2^23 and every k a chunk can hold, and the
whole chunk rule against the column-by-column zone parity on sampled rows of
four plates (the library's own threshold table, fzp_zone_thresholds), at the
sampling of Eq. 5 and at Eq. 6's limit of two samples per zone, including
chunks at the chord ends, next to the axis and on the positive-centred plate.
"""
import bisect
import math
import os
import sys

import numpy as np
import pytest


def window16(D: np.ndarray, d: int) -> np.ndarray:
    inv2d = np.float32(0.5) / np.float32(d)
    td = 2 * d
    k = np.ceil(D.astype(np.float32) * inv2d).astype(np.int64)
    k += (k * (k + td) < D).astype(np.int64)
    k -= ((k > 0) & ((k - 1) * (k - 1 + td) >= D)).astype(np.int64)
    k -= ((k > 0) & ((k - 1) * (k - 1 + td) >= D)).astype(np.int64)
    assert np.all(np.abs(k * (k + td)) < 2 ** 31) and np.all(np.abs(D) < 2 ** 31)
    return k


def exact_k(D: int, d: int) -> int:
    k = max(0, math.isqrt(d * d + D) - d)
    while k * (k + 2 * d) < D:
        k += 1
    while k > 0 and (k - 1) * (k - 1 + 2 * d) >= D:
        k -= 1
    return k


def test_window16_search_is_exact():
    rng = np.random.default_rng(11)
    ds = sorted({128, 129, 255, 1000, 4096, 65535, 1 << 20, (1 << 23) - 1}
                | {int(x) for x in rng.integers(128, 1 << 23, 300)})
    checked = 0
    for d in ds:
        Ds = []
        for k in range(1, 16):  # a boundary strictly inside the chunk
            lo, hi = (k - 1) * (k - 1 + 2 * d) + 1, k * (k + 2 * d)
            Ds += [lo, hi, (lo + hi) // 2] + [int(x) for x in rng.integers(lo, hi + 1, 6)]
        D = np.array(Ds, dtype=np.int64)
        got = window16(D, d)
        want = np.array([exact_k(int(x), d) for x in Ds])
        assert np.array_equal(got, want), (d, D[got != want][:4], got[got != want][:4])
        checked += len(Ds)
    assert checked > 20_000


def _chunk_bits(x, dj2, c, sR, thr, centre, zone):
    """The kernel's chunk rule, step for step."""
    dr, dl = x - c, c - (x + 15)
    if dr < 128 and dl < 128:
        bits = 0
        for p in range(16):
            s = dj2 + (x + p - c) ** 2
            if s <= sR and (zone(s) ^ centre) & 1:
                bits |= 1 << p
        return bits
    right = dr >= 128
    d = dr if right else dl
    sn, sf = dj2 + d * d, dj2 + (d + 15) ** 2
    zn, zf = zone(min(sn, sR)), zone(min(sf, sR))
    bits = 0xFFFF if ((zn if right else zf) ^ centre) & 1 else 0
    for m in range(zn + 1, zf + 1):
        D = thr[m - 1] - sn
        k = int(window16(np.array([D], dtype=np.int64), d)[0])
        bits ^= (0xFFFF << (k if right else 16 - k)) & 0xFFFF
    return bits


def _direct(x, dj2, c, sR, centre, zone):
    """Column by column; also the mask of the columns inside the disc."""
    bits = inside = 0
    for p in range(16):
        s = dj2 + (x + p - c) ** 2
        if s <= sR:
            inside |= 1 << p
            if (zone(s) ^ centre) & 1:
                bits |= 1 << p
    return bits, inside


@pytest.fixture(scope="module")
def fzp():
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import __graft_entry__
    __graft_entry__.build()
    import paper_2609_01978_gb300 as m
    return m


LAM = 632.8e-9
CASES = {
    "config1": dict(D=4e-3, f=20e-3, lam=LAM),
    "d0.25m": dict(D=0.25, f=1.25, lam=LAM),
    "d5m": dict(D=5.0, f=25.0, lam=LAM),
    "d0.25m_eq6_limit": dict(D=0.25, f=1.25, lam=LAM, dx=LAM * 1.25 / (2 * 0.25)),
    "d0.25m_positive_centred": dict(D=0.25, f=1.25, lam=LAM, centre_open=1),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_chunk_rule_equals_column_rule(fzp, case):
    kw = dict(CASES[case], M=512, pitch=LAM * 5 / 8)
    q = fzp.plan_query(**kw)
    thr = [int(x) for x in fzp.zone_thresholds(**kw)]
    c, sR, centre = q["c"], q["s_R"], kw.get("centre_open", 0)

    def zone(s):
        return bisect.bisect_right(thr, s)  # #{m : S_m <= s}

    rng = np.random.default_rng(sum(map(ord, case)))
    bmax0 = math.isqrt(sR)
    n_events = n_chunks = 0
    for dj in [0, 1, bmax0 // 2, bmax0 - 3] + [int(x) for x in rng.integers(-bmax0, bmax0, 40)]:
        dj2 = dj * dj
        if dj2 > sR:
            continue
        b = math.isqrt(sR - dj2)
        lo, hi = c - b, c + b
        xs = [lo - 7, lo, hi - 15, hi - 3, c - 15, c - 8, c + 1, c - 143, c + 128, c - 128 - 15]
        xs += [int(x) for x in rng.integers(lo, max(lo + 1, hi - 15), 60)]
        for x in xs:
            if x + 15 < lo or x > hi:
                continue
            want, inside = _direct(x, dj2, c, sR, centre, zone)
            got = _chunk_bits(x, dj2, c, sR, thr, centre, zone)
            assert (got & inside) == want, (case, dj, x, hex(got), hex(want), hex(inside))
            n_chunks += 1
            n_events += bin(want ^ (want << 1) & 0xFFFF).count("1")
    assert n_chunks > 1000 and n_events > 500, (n_chunks, n_events)

