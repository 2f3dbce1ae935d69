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



def _chunk_zones(x, dj2, c, sR, thr, zone):
    """The kernel's phase-plate chunk rule: (ok, z0, up, down)."""
    dr, dl = x - c, c - (x + 15)
    if dr < 128 and dl < 128:
        zp = zone(min(dj2 + dr * dr, sR))
        z0, up, dn = zp, 0, 0
        for p in range(1, 16):
            z = zone(min(dj2 + (dr + p) ** 2, sR))
            if z == zp + 1:
                up |= 1 << p
            elif z == zp - 1:
                dn |= 1 << p
            elif z != zp:
                return False, 0, 0, 0
            zp = z
        return True, z0, up, dn
    right = dr >= 128
    d = dr if right else dl
    sn, sf = dj2 + d * d, dj2 + (d + 15) ** 2
    zn, zf = zone(min(sn, sR)), zone(min(sf, sR))
    ev = 0
    for m in range(zn + 1, zf + 1):
        k = int(window16(np.array([thr[m - 1] - sn], dtype=np.int64), d)[0])
        ev |= 1 << (k if right else 16 - k)
    if bin(ev).count("1") != zf - zn:
        return False, 0, 0, 0
    return (True, zn, ev, 0) if right else (True, zf, 0, ev)


PHASE_CASES = {
    "table4_grid_L4": dict(D=4.0, f=20.0, lam=532e-9, levels=4, dx=532e-9 * 20.0 / 2.0 / 16),
    "d0.02m_L16": dict(D=0.02, f=0.1, lam=LAM, levels=16),
    "d0.05m_L8": dict(D=0.05, f=0.25, lam=LAM, levels=8),
    "d0.01m_L3": dict(D=0.01, f=0.05, lam=LAM, levels=3),
}


@pytest.mark.parametrize("case", sorted(PHASE_CASES))
def test_chunk_zone_steps_equal_column_zones(fzp, case):
    """Phase plates: the chunk's zone at its first column plus the up and down
    steps at or before each column (two popcounts) give the zone of every
    column inside the disc; then the level is z mod L, computed as
    z - L umulhi(z, ceil(2^32 / L))."""
    kw = dict(PHASE_CASES[case], M=512, pitch=LAM * 5 / 8)
    q = fzp.plan_query(**kw)
    thr = [int(x) for x in fzp.zone_thresholds(**kw)]
    c, sR, L = q["c"], q["s_R"], kw["levels"]
    magic = (0xFFFFFFFF // L) + 1

    def zone(s):
        return bisect.bisect_right(thr, s)

    rng = np.random.default_rng(sum(map(ord, case)))
    bmax0 = math.isqrt(sR)
    n_chunks = n_steps = 0
    for dj in [0, 5, bmax0 // 3, bmax0 - 2] + [int(x) for x in rng.integers(-bmax0, bmax0, 30)]:
        dj2 = dj * dj
        if dj2 > sR:
            continue
        b = math.isqrt(sR - dj2)
        lo, hi = c - b, c + b
        xs = [lo, hi - 15, c - 15, c - 7, c + 3, c - 143, c + 128]
        xs += [int(x) for x in rng.integers(lo, max(lo + 1, hi - 15), 40)]
        for x in xs:
            if x + 15 < lo or x > hi:
                continue
            ok, z0, up, dn = _chunk_zones(x, dj2, c, sR, thr, zone)
            assert ok, (case, dj, x)
            for p in range(16):
                s = dj2 + (x + p - c) ** 2
                if s > sR:
                    continue
                mp = (2 << p) - 1
                z = z0 + bin(up & mp).count("1") - bin(dn & mp).count("1")
                assert z == zone(s), (case, dj, x, p)
                lev = z - L * ((z * magic) >> 32)
                assert lev == z % L
            n_chunks += 1
            n_steps += bin(up | dn).count("1")
    assert n_chunks > 500 and n_steps > 200, (n_chunks, n_steps)


def test_level_remainder_by_multiply_high():
    rng = np.random.default_rng(9)
    zs = [0, 1, (1 << 24) - 1] + [int(x) for x in rng.integers(0, 1 << 24, 3000)]
    for L in range(2, 65):
        magic = (0xFFFFFFFF // L) + 1
        extra = [L * k + e for k in (1, 1000, (1 << 24) // L - 1) for e in (-1, 0, 1) if 0 <= L * k + e < (1 << 24)]
        for z in zs + extra:
            assert z - L * ((z * magic) >> 32) == z % L, (L, z)
