"""The SA-CZT residual phase without FP64 (k_sa_phase in saczt.cu), emulated
on the CPU in the same IEEE single-precision steps, against the phase of
Fig. 5 step 2 in extended precision.

For spectrum sample s = fa^2 + fb^2 (fa, fb the signed frequency indices of
the P x P grid), q = K^2 / k0^2 = eps s with eps = (lambda / (P dx))^2, and
the residual h = k_z - c k_max - d K^2 / k_max times f is, in turns,
-A z - C s with z = 1 - sqrt(1 - q), A = f / lambda, C = A (d k0 / k_max) eps.
The kernel forms z in float-float pairs and C s mod 1 in 64-bit fixed
point; this checks its error stays below 3e-7 turns over every region of
the spectrum the grid holds (up to the evanescent edge, where the phase's
sensitivity to q grows as 1 / sqrt(1 - q)), for the plates the SA-CZT form
runs."""
import math

import numpy as np
import pytest

f32 = np.float32


def fmaf(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def consts(lam, f, dx, P):
    """The host constants (FP64, as sa_phase_consts computes them)."""
    lr = lam / (P * dx)
    eps = lr * lr
    A = f / lam
    k0 = 2.0 * math.pi / lam
    kmax = 2.0 * k0 / 3.0
    d = (math.sqrt(k0 * k0 - kmax * kmax) - k0) / kmax
    C = A * (d * k0 / kmax) * eps
    eh = f32(eps)
    el = f32(eps - float(eh))
    ah = f32(A)
    al = f32(A - float(ah))
    cfix = int(math.ldexp(abs(C), 64))
    sev = math.ceil(1.0 / eps)
    while sev > 0 and eps * (sev - 1) >= 1.0:
        sev -= 1
    while eps * sev < 1.0:
        sev += 1
    return dict(eh=eh, el=el, ah=ah, al=al, cfix=cfix, cneg=C < 0, s_ev=sev, eps=eps, A=A, C=C)


def turns_kernel(c, s: int) -> float:
    """sa_turns, step by step in float32."""
    sh, sl = f32(s & ~0xFFF), f32(s & 0xFFF)
    p1, p2 = f32(c["eh"] * sh), f32(c["eh"] * sl)
    e1, e2 = fmaf(c["eh"], sh, -p1), fmaf(c["eh"], sl, -p2)
    xh, xl = two_sum(p1, p2)
    xl = fmaf(c["el"], f32(sh + sl), f32(xl + f32(e1 + e2)))
    xh, xl = fast_two_sum(xh, xl)
    wh, wl = two_sum(f32(1.0), f32(-xh))
    wl = f32(wl - xl)
    wh, wl = fast_two_sum(wh, wl)
    y0 = f32(np.sqrt(wh))
    y1 = f32(f32(fmaf(-y0, y0, wh) + wl) * f32(f32(1.0) / f32(y0 + y0)))
    zh, ze = two_sum(f32(1.0), f32(-y0))
    zl = f32(ze - y1)
    zh, zl = fast_two_sum(zh, zl)
    ph = f32(c["ah"] * zh)
    pl = f32(fmaf(c["ah"], zh, -ph) + fmaf(c["ah"], zl, f32(c["al"] * zh)))
    t1 = f32(f32(ph - f32(np.rint(ph))) + pl)
    prod = (c["cfix"] * s) % (1 << 64)
    t2 = f32(f32(prod >> 40) * f32(2.0 ** -24))
    t = f32(t2 - t1) if c["cneg"] else f32(f32(-t2) - t1)
    return float(f32(t - f32(np.rint(t))))


def turns_ref(c, s: int) -> float:
    """-A z - C s mod 1 in extended precision (z without cancellation)."""
    L = np.longdouble
    q = L(c["eps"]) * L(s)
    z = q / (L(1) + np.sqrt(L(1) - q))
    t = -L(c["A"]) * z - L(c["C"]) * L(s)
    return float(t - np.rint(t))


PLATES = [
    # (lambda, f, dx, P): the bench's 8 mm plate, the tests' 2 mm plate, and an
    # f/1.5 plate whose grid reaches the evanescent edge
    (632.8e-9, 40e-3, 632.8e-9 * 5 / 4, 16384),
    (632.8e-9, 10e-3, 632.8e-9 * 5 / 4, 4096),
    (450e-9, 3e-3, 450e-9 * 1.5 / 4, 8192),
]


@pytest.mark.skipif(np.finfo(np.longdouble).eps > 1e-18, reason="needs an extended-precision long double")
@pytest.mark.parametrize("plate", PLATES)
def test_phase_turns_error(plate):
    c = consts(*plate)
    P = plate[3]
    smax = 2 * (P // 2) ** 2
    rng = np.random.default_rng(7)
    fa = rng.integers(-P // 2, P // 2, 4000)
    fb = rng.integers(-P // 2, P // 2, 4000)
    ss = list((fa * fa + fb * fb).tolist()) + list(range(0, 300)) + [smax, smax - 1]
    ss += [c["s_ev"] - k for k in range(1, 50)]  # the evanescent edge, where the grid reaches it
    worst = 0.0
    for s in ss:
        if s >= c["s_ev"] or s > smax or s < 0:
            continue
        e = abs(turns_kernel(c, int(s)) - turns_ref(c, int(s)))
        e = min(e, 1 - e)
        worst = max(worst, e)
    assert worst < 3e-7, worst


def test_evanescent_edge():
    """s_ev is the first s with eps s >= 1 (K >= k0 is zeroed)."""
    for plate in PLATES:
        c = consts(*plate)
        assert c["eps"] * c["s_ev"] >= 1.0 > c["eps"] * (c["s_ev"] - 1)
