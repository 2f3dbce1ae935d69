"""Pins of the CPU FP64 oracle against things other than itself.

Each test ties a piece of the oracle to the mathematics or to a number the
paper prints: brute force, a library transform, closed forms of Sec. 2.3,
discrete identities (Parseval, Wiener-Khinchin), symmetries, and the grid rule
of Tables 1-5.  A plausible mistake in the oracle (dropped chirp, wrong sign,
transposed operand, wrong ROI origin, wrong zone rule) fails at least one.
"""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


# --------------------------------------------------------------------------
# Transforms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 11, 14])
def test_fft_matches_numpy(oracle_mod, k):
    rng = np.random.default_rng(k)
    L = 1 << k
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    assert rel(oracle_mod.fft(x), np.fft.fft(x)) < 1e-13
    assert rel(oracle_mod.fft(x, inverse=True), np.fft.ifft(x) * L) < 1e-13


@pytest.mark.parametrize("N,M", [(1, 1), (7, 3), (64, 64), (200, 37), (513, 256)])
def test_czt_bluestein_matches_eq9_direct_sum(oracle_mod, N, M):
    rng = np.random.default_rng(N * 1000 + M)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    alpha, omega = rng.uniform(-0.5, 0.5), rng.uniform(-0.01, 0.01)
    ref = np.array([np.sum(x * np.exp(-2j * np.pi * (alpha * np.arange(N) + omega * m * np.arange(N))))
                    for m in range(M)])
    assert rel(oracle_mod.czt(x, M, alpha, omega), ref) < 1e-12
    assert rel(oracle_mod.czt(x, M, alpha, omega, direct=True), ref) < 1e-12


@pytest.mark.parametrize("N", [16, 100, 257])
def test_czt_dft_special_case(oracle_mod, N):
    """A = 1, W = exp(-2 pi i / N), M = N recovers the DFT (Sec. 2.6)."""
    rng = np.random.default_rng(N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    assert rel(oracle_mod.czt(x, N, 0.0, 1.0 / N), np.fft.fft(x)) < 1e-12


# --------------------------------------------------------------------------
# Three evaluations of the field agree (brute force pins the CZT method)
# --------------------------------------------------------------------------

def _tiny(oracle_mod, **kw):
    base = dict(D=4e-3 / 8, f=20e-3 / 8, lam=632.8e-9, M=16, p=0.4e-6)
    base.update(kw)
    return oracle_mod.Geometry(**base)


@pytest.mark.parametrize("case", ["fzp", "fzp_oddM", "fzp_exact", "lens", "deform", "offaxis_pitch", "offaxis_roi"])
def test_o1_o2_o3_agree(oracle_mod, case):
    O = oracle_mod
    if case == "fzp":
        g = _tiny(O)
    elif case == "fzp_oddM":
        g = _tiny(O, M=15, p=0.31e-6)
    elif case == "fzp_exact":
        g = _tiny(O, kind=O.FZP_EXACT)
    elif case == "lens":
        g = _tiny(O, kind=O.LENS, M=12)
    elif case == "deform":
        d = O.Deform(amp=632.8e-9 / 4, period=1.3e-4, theta=0.7, taper=0.4,
                     ridges=[(1e-5, -2e-5, 0.3, 632.8e-9 / 8, 3e-5), (-4e-5, 0.0, 2.0, -632.8e-9 / 10, 5e-5)])
        g = _tiny(O, deform=d)
    elif case == "offaxis_pitch":
        g = _tiny(O, M=10, p=1.1e-6)
    else:  # ROI whose first sample is off the centred grid by 3.3 pitches on both axes
        g = _tiny(O, M=12, p=0.5e-6, x0=-2.7 * 0.5e-6)
        assert abs(g.coords_out()[0] + 2.7 * 0.5e-6) < 1e-20
    u1 = O.field_direct(g)
    assert rel(O.field_separable(g), u1) < 1e-12
    assert rel(O.field_czt(g), u1) < 1e-12
    # a sub-range of rows (stripe) as well
    j0, j1 = 37, 211
    u1s = O.field_direct(g, j0, j1)
    assert rel(O.field_czt(g, j0, j1), u1s) < 1e-12
    assert rel(O.field_separable(g, j0, j1), u1s) < 1e-12


def test_row_linearity(oracle_mod):
    """U is linear in aperture rows (Sec. 2.6: rows transformed in independent batches)."""
    O = oracle_mod
    g = _tiny(O, M=20)
    full = O.field_czt(g)
    a = 301
    assert rel(O.field_czt(g, 0, a) + O.field_czt(g, a, g.N), full) < 1e-12


# --------------------------------------------------------------------------
# Discrete identities on the full (SFFT-like) window
# --------------------------------------------------------------------------

def _full_window(O, N=101, kind=None):
    D, f, lam = 4e-3 / 40, 20e-3 / 40, 632.8e-9
    dx = D / N * 1.02
    p = lam * f / (N * dx)  # Eq. 8: dx_out = lambda z / (N dx_in)
    kw = dict(D=D, f=f, lam=lam, M=N, p=p, dx=dx, N=N)
    if kind is not None:
        kw["kind"] = kind
    return O.Geometry(**kw)


def test_parseval_full_window(oracle_mod):
    """With dx_out = lambda f/(N dx_in) and M = N the CZT is an N-point DFT, so
    sum |U|^2 dx_out^2 = sum |U0|^2 dx_in^2 exactly (energy conservation)."""
    O = oracle_mod
    g = _full_window(O)
    U = O.field_czt(g)
    U0 = O.aperture_rows(g, 0, g.N)
    lhs = np.sum(np.abs(U) ** 2) * g.p ** 2
    rhs = np.sum(np.abs(U0) ** 2) * g.dx ** 2
    assert abs(lhs / rhs - 1) < 1e-12


def test_wiener_khinchin_full_window(oracle_mod):
    """On the full window |fft2(I)| equals the modulus of the circular
    autocorrelation of the chirped aperture field (Sec. 2.3 MTF machinery)."""
    O = oracle_mod
    g = _full_window(O, N=61)
    U = O.field_czt(g)
    I = np.abs(U) ** 2
    U0 = O.aperture_rows(g, 0, g.N)
    u = (np.arange(g.N) - g.c) * g.dx
    a = U0 * np.exp(1j * np.pi * (u[None, :] ** 2 + u[:, None] ** 2) / (g.lam * g.f))
    Fa = np.fft.fft2(a)
    ac = np.fft.ifft2(np.abs(Fa) ** 2)  # circular autocorrelation of a
    lhs = np.abs(np.fft.fft2(I))
    rhs = np.abs(ac) * np.abs(lhs[0, 0]) / np.abs(ac[0, 0])
    assert rel(lhs, rhs) < 1e-10


# --------------------------------------------------------------------------
# Closed forms of Sec. 2.3 (ideal lens -> Airy; binary FZP -> 1/pi^2)
# --------------------------------------------------------------------------

def test_closed_forms_match_printed_values(oracle_mod):
    O = oracle_mod
    gold = json.load(open(os.path.join(GOLDEN, "airy_constants.json")))
    fw = O.airy_fwhm_factor()
    assert abs(fw - 1.028994) < 2e-6
    assert round(fw, 3) == gold["fwhm_factor_printed"][1]
    assert math.floor(fw * 1000) / 1000 == gold["fwhm_factor_printed"][0]
    assert round(100 * O.binary_fzp_efficiency(), 1) == gold["de_binary_printed_percent"]
    assert round(O.AIRY_NULL, 2) == gold["null_factor_printed"]
    assert abs(O.airy_encircled(O.AIRY_NULL) - 0.837785) < 2e-6
    assert abs(O.circ_mtf(0.5) - 0.391002) < 1e-6


def test_ideal_lens_gives_airy(oracle_mod):
    """A perfect thin lens (circ pupil, phase -pi r^2/(lambda f)) focuses to the
    Airy pattern: FWHM 1.028994 lambda f / D, EE(r_null) = 0.837785 and the
    circular-pupil MTF at nu_cut/2 (0.391002).  The ROI truncates the PSF tails,
    which raises the normalised MTF by the energy fraction that leaves the ROI;
    the pin multiplies that fraction back (bound measured: < 1e-3)."""
    O = oracle_mod
    D, f, lam = 4e-3, 20e-3, 632.8e-9
    N = 2001
    g = O.Geometry(D=D, f=f, lam=lam, M=512, p=lam * (f / D) / 8, dx=D / (N - 1) * 1.0000001, N=N, kind=O.LENS)
    m = O.metrics(g, O.field_czt(g))
    lfD = lam * f / (2 * g.R)
    assert abs(m["fwhm_x"] / (O.airy_fwhm_factor() * lfD) - 1) < 1e-4
    assert abs(m["fwhm_y"] / (O.airy_fwhm_factor() * lfD) - 1) < 1e-4
    assert abs(m["de_lobe"] / O.airy_encircled(O.AIRY_NULL) - 1) < 1e-4  # lens: all incident power in one order
    assert abs(m["mtf_half_cut"] * m["de_roi"] / O.circ_mtf(0.5) - 1) < 1e-3
    # MTF curve over the band, same correction
    nu = (np.arange(16) + 0.5) / 16
    ref = np.array([O.circ_mtf(v) for v in nu])
    assert np.max(np.abs(m["mtf16"] * m["de_roi"] - ref)) < 2.5e-3


@pytest.fixture(scope="module")
def config1(oracle_mod):
    O = oracle_mod
    g = O.Geometry(D=4e-3, f=20e-3, lam=632.8e-9, M=256, p=0.2e-6)
    U = O.field_czt(g)
    return g, U, O.metrics(g, U)


def test_config1_grid(config1, oracle_mod):
    g, _, _ = config1
    assert g.N == 5057 and g.c == 2528
    assert g.total_zones() == 315


def test_binary_fzp_efficiency_and_fwhm(config1, oracle_mod):
    """Binary amplitude FZP: first order carries 1/pi^2 of the incident power
    (Sec. 2.3), so the main lobe holds EE(r_null)/pi^2 = 0.084885; the other
    orders perturb it by O(1/zones) (315 zones here).  The focal spot is the
    Airy spot of the full aperture."""
    O = oracle_mod
    g, U, m = config1
    target = O.airy_encircled(O.AIRY_NULL) * O.binary_fzp_efficiency()
    assert abs(m["de_lobe"] / target - 1) < 1e-2
    airy = O.airy_fwhm_factor() * g.lam * g.f / (2 * g.R)
    assert abs(m["fwhm_x"] / airy - 1) < 5e-3
    assert abs(m["fwhm_x"] / m["fwhm_y"] - 1) < 1e-12
    assert abs(m["p_in"] / m["p_in_disc"] - 1) < 1e-3  # pixel count vs pi R^2 (reading 5)


def test_focal_plane_symmetry(config1):
    """Flat FZP on a centred grid: I is invariant under transpose and under the
    mirror n -> M - n about the on-axis sample M/2."""
    g, U, _ = config1
    I = np.abs(U) ** 2
    assert rel(I, I.T) < 1e-12
    M = g.M
    assert rel(I[1:, :], I[1:, :][::-1, :]) < 1e-12
    assert np.unravel_index(np.argmax(I), I.shape) == (M // 2, M // 2)


# --------------------------------------------------------------------------
# Mask and grid rule
# --------------------------------------------------------------------------

def test_mask_structure(oracle_mod):
    O = oracle_mod
    g = O.Geometry(D=4e-3 / 4, f=20e-3 / 4, lam=632.8e-9, M=8, p=1e-6)
    mask = O.mask_rows(g, 0, g.N).astype(np.int64)
    c = g.c
    assert mask[c, c] == 0  # negative-centred: zone 0 opaque (Sec. 4.1)
    assert np.array_equal(mask, mask.T) and np.array_equal(mask, mask[::-1, :])
    inside = O.count_aperture(g)
    # zones have equal area (r_m^2 = m lambda f), half of them open
    assert abs(mask.sum() / inside - 0.5) < 2.0 / g.total_zones()
    # zone boundaries along the centre row sit at r_m = sqrt(m lambda f) (Eq. 4)
    row = mask[c, c:]
    flips = np.nonzero(np.diff(row))[0] + 1  # first index of each new run
    r_flip = flips * g.dx
    r_m = np.sqrt(np.arange(1, len(flips) + 1) * g.lam * g.f)
    assert np.all(np.abs(r_flip - r_m) <= g.dx)


def _disc_limit_exact(dx, R):
    """Largest integer s with fl(s dx^2) <= fl(R^2): the disc rule of Fig. 2
    Stage 2 on squared sample distances, found from the exact quotient and
    settled by the same IEEE products (Python floats)."""
    from fractions import Fraction
    dx2, R2 = dx * dx, R * R
    s = int(Fraction(R2) / Fraction(dx2))
    while float(s + 1) * dx2 <= R2:
        s += 1
    while s > 0 and float(s) * dx2 > R2:
        s -= 1
    return s


@pytest.mark.parametrize("D,f,dx", [(4e-3, 20e-3, None), (0.02, 0.1, None), (0.05, 0.25, None),
                                    (2000 * 2.0 ** -20, 20e-3, 2.0 ** -20)])
def test_count_aperture_is_the_disc_lattice_count(oracle_mod, D, f, dx):
    """P_in = (samples inside R_eff) dx^2 (Fig. 2 Stage 2, reading 5).  The
    oracle counts by bisection on each row; the count must equal the number
    of lattice points (a, b) with a^2 + b^2 <= s_R (Gauss's circle count,
    summed row by row with exact integer square roots), and, on config 1's
    grid, the number of open samples of the clear pupil's per-sample mask.
    A count that drops the on-axis column of each row (2 lo instead of
    2 lo + 1) fails here; so does a strict inequality at the rim, on the grid
    with dx = 2^-20 m and R = 1000 dx, where R^2 / dx^2 = 10^6 exactly and
    samples such as (600, 800) lie on the rim."""
    O = oracle_mod
    g = O.Geometry(D=D, f=f, lam=632.8e-9, M=8, p=1e-6, dx=dx)
    sR = _disc_limit_exact(g.dx, g.R)
    b = math.isqrt(sR)
    lattice = sum(2 * math.isqrt(sR - a * a) + 1 for a in range(-b, b + 1))
    assert O.count_aperture(g) == lattice, (D, O.count_aperture(g), lattice)
    if D == 4e-3:
        gc = O.Geometry(D=D, f=f, lam=632.8e-9, M=8, p=1e-6, kind=O.CIRC)
        assert int(O.mask_rows(gc, 0, gc.N).sum(dtype=np.int64)) == lattice
        # the disc of Fig. 2 Stage 2 holds pi R^2 / dx^2 samples to O(R / dx)
        assert abs(lattice * g.dx ** 2 / (math.pi * g.R ** 2) - 1) < 4 * g.dx / g.R


def test_total_zones_eq3(oracle_mod):
    """Total_Zones = floor(n_exact) of Eq. 3, checked by counting exact radii
    r_n = sqrt(n lambda f + n^2 lambda^2 / 4) that fit inside R."""
    O = oracle_mod
    for D, f in [(4e-3, 20e-3), (0.08, 1.5), (0.25, 1.25)]:
        g = O.Geometry(D=D, f=f, lam=632.8e-9, M=8, p=1e-6)
        n = 0
        while (n + 1) * g.lam * g.f + ((n + 1) * g.lam) ** 2 / 4 <= g.R ** 2:
            n += 1
        assert g.total_zones() == n


def test_v8_grid_tables(oracle_mod):
    """Nx of Tables 1-5 from the Fig. 18 grid rule (ceil, forced odd)."""
    O = oracle_mod
    gold = json.load(open(os.path.join(GOLDEN, "v8_grid_tables.json")))
    lam = gold["lambda"]
    for row in gold["rows"]:
        R = row["D"] / 2
        edge = lam * row["f"] / R
        dx = edge / row["k"]
        assert abs(dx * 1e6 - row["dx_um_printed"]) < 5e-4 + 1e-9
        g = O.Geometry(D=row["D"], f=row["f"], lam=lam, M=8, p=1e-6, dx=dx)
        assert g.N == row["Nx"], row


# --------------------------------------------------------------------------
# Extractor pieces on synthetic inputs with known answers
# --------------------------------------------------------------------------

def test_fwhm_extractor_gaussian(oracle_mod):
    M, p, sigma = 256, 0.1e-6, 0.9e-6
    x = (np.arange(M) - M // 2) * p
    row = np.exp(-x ** 2 / (2 * sigma ** 2))
    fw = oracle_mod.fwhm_row(row, p)
    assert abs(fw / (2 * math.sqrt(2 * math.log(2)) * sigma) - 1) < 2e-4


@pytest.mark.parametrize("off", [0.3, 0.45])
def test_fwhm_extractor_off_sample_peak(oracle_mod, off):
    """A Gaussian whose peak falls between samples (0.3 and 0.45 of a sample
    from the on-axis one): the 3-point parabola (Fig. 18 'parabolic peak')
    recovers the peak height, so the spline crossings give the FWHM within
    1e-4; taking the on-axis sample as the peak would widen it by 1-3e-3."""
    M, sigma = 128, 5.0
    x = np.arange(M) - M // 2 - off
    fw = oracle_mod.fwhm_row(np.exp(-x ** 2 / (2 * sigma ** 2)), 1.0)
    assert abs(fw / (2 * math.sqrt(2 * math.log(2)) * sigma) - 1) < 1e-4


def test_mtf_extractor_gaussian(oracle_mod):
    """A Gaussian PSF has a Gaussian OTF, exp(-2 pi^2 sigma^2 nu^2); each radial
    bin must hold the mean of that closed form over the FFT samples whose
    radial frequency falls in the bin (bins of nu_Nyq / 200)."""
    M, p, sigma = 256, 0.1e-6, 0.5e-6
    x = (np.arange(M) - M // 2) * p
    I = np.exp(-(x[None, :] ** 2 + x[:, None] ** 2) / (2 * sigma ** 2))
    c, mean = oracle_mod.mtf_radial(I, p)
    fu = np.fft.fftfreq(M, d=p)
    nu = np.hypot(fu[None, :], fu[:, None])
    # bin of each sample: largest b with b <= 200 |k| / (M/2), by exact integer search
    kk = [int(round(v)) for v in np.fft.fftfreq(M) * M]
    b = np.array([[max(t for t in range(0, 300) if (t * M) ** 2 <= 160000 * (kv * kv + ku * ku))
                   for ku in kk] for kv in kk])
    ok = b < 200
    ref = np.bincount(b[ok], weights=np.exp(-2 * np.pi ** 2 * sigma ** 2 * nu[ok] ** 2), minlength=200)
    cnt = np.bincount(b[ok], minlength=200)
    has = cnt > 0
    assert np.array_equal(np.isfinite(mean), has)
    assert np.max(np.abs(mean[has] - ref[has] / cnt[has])) < 1e-10
    # the first sample off DC lands in bin floor(200 * 2 p / (M p)) = 1
    assert np.isfinite(mean[0]) and mean[0] == 1.0


@pytest.mark.parametrize("L", [2, 4, 8])
def test_phase_fzp_efficiency_ladder(oracle_mod, L):
    """L-level phase FZP (Fig. 18, Stage 3 "L-level phase"; the DE ladder of its
    report): the first order carries sinc^2(1/L) of the incident power
    (0.405 / 0.811 / 0.950), so the main lobe holds EE(r_null) sinc^2(1/L); the
    focal spot is the Airy spot.  Grid of Fig. 18 Stage 1 (S_samp = 4):
    dx = lambda f / (2 D max(L, 2)).  Measured deviations are about 1e-4."""
    O = oracle_mod
    lam = 632.8e-9
    g = O.Geometry(D=2e-3, f=10e-3, lam=lam, M=256, p=lam * 5 / 8, kind=O.FZP_PHASE, levels=L)
    assert g.N == {2: 2529, 4: 5057, 8: 10115}[L]
    m = O.metrics(g, O.field_czt(g))
    target = O.airy_encircled(O.AIRY_NULL) * O.phase_fzp_efficiency(L)
    assert abs(m["de_lobe"] / target - 1) < 5e-4
    airy = O.airy_fwhm_factor() * g.lam * g.f / (2 * g.R)
    assert abs(m["fwhm_x"] / airy - 1) < 3e-4


def test_binary_phase_is_disc_minus_twice_amplitude(oracle_mod):
    """For L = 2 the level steps are the zones of the amplitude rule (kappa_L =
    kappa), so the transmission is +1 on even and -1 on odd zones: T_phase =
    circ - 2 T_amplitude exactly, and the fields obey the same identity (the
    propagation is linear)."""
    O = oracle_mod
    lam = 632.8e-9
    kw = dict(D=1e-3, f=5e-3, lam=lam, M=64, p=lam * 5 / 8)
    gp = O.Geometry(kind=O.FZP_PHASE, levels=2, **kw)
    ga = O.Geometry(kind=O.FZP_PARAXIAL, **kw)
    gc = O.Geometry(kind=O.CIRC, **kw)
    assert gp.N == ga.N == gc.N and gp.dx == ga.dx
    Up, Ua, Uc = O.field_czt(gp), O.field_czt(ga), O.field_czt(gc)
    assert rel(Up, Uc - 2 * Ua) < 1e-12
    # the exported level map: 1 + q inside the aperture, q = zone parity here
    lev = O.mask_rows(gp, 0, gp.N)
    amp = O.mask_rows(ga, 0, ga.N)
    disc = O.mask_rows(gc, 0, gc.N)
    assert np.array_equal(lev, disc * (1 + amp))


def test_phase_fzp_direct_equals_czt(oracle_mod):
    """O1 (Eq. 1 summed literally) and O3 (the Bluestein method) agree for a
    4-level phase plate on a small grid."""
    O = oracle_mod
    lam = 632.8e-9
    g = O.Geometry(D=0.15e-3, f=0.75e-3, lam=lam, M=24, p=lam * 5 / 8, kind=O.FZP_PHASE, levels=4)
    assert g.N < 400
    assert rel(O.field_direct(g), O.field_czt(g)) < 1e-10


@pytest.mark.parametrize("nz", [7, 8])
def test_centre_configurations_on_axis(oracle_mod, nz):
    """The two centre configurations of the binary plate (Fig. 18 engine).  On
    the axis each paraxial zone k contributes the closed form
    e^{ikf}/(i lambda f) * (lambda f / i)(e^{i pi (k+1)} - e^{i pi k}) = 2 (-1)^k e^{ikf}
    (the zone integral of the Eq. 2 chirp over r_k^2 = k lambda f .. (k+1) lambda f),
    so with nz zones inside R the negative-centred plate (odd zones open) gives
    -2 floor(nz/2) e^{ikf} and the positive-centred one (even zones, the centre
    among them) +2 ceil(nz/2) e^{ikf}: opposite signs, and a magnitude ratio
    that tells an odd zone count from an even one.  The two masks are
    complements inside the aperture disc, so their fields sum to the clear
    pupil's exactly.  16 samples per outermost zone width keep the
    discretisation error near 1e-3 of a zone's contribution."""
    O = oracle_mod
    lam, f = 500e-9, 0.02
    D = 2 * math.sqrt(nz * lam * f)
    kw = dict(D=D, f=f, lam=lam, M=16, p=lam * f / D / 8, dx=lam * f / (16 * D))
    gn = O.Geometry(kind=O.FZP_PARAXIAL, **kw)
    gp = O.Geometry(kind=O.FZP_POSITIVE, **kw)
    gc = O.Geometry(kind=O.CIRC, **kw)
    Un, Up, Uc = O.field_separable(gn), O.field_separable(gp), O.field_separable(gc)
    assert rel(Un + Up, Uc) < 1e-12
    ikf = np.exp(2j * math.pi * f / lam)
    c = gn.M // 2
    assert abs(Un[c, c] / ikf - (-2 * (nz // 2))) < 0.02
    assert abs(Up[c, c] / ikf - 2 * ((nz + 1) // 2)) < 0.02
    assert abs(Uc[c, c] / ikf - 2 * (nz % 2)) < 0.02
    # the exported masks: complements inside the disc, the centre pixel open
    mn, mp, mc = (O.mask_rows(g, 0, g.N) for g in (gn, gp, gc))
    assert np.array_equal(mn + mp, mc)
    assert mp[gp.c, gp.c] == 1 and mn[gn.c, gn.c] == 0


# --------------------------------------------------------------------------
# Membrane deformation (config 4's model; reading of the wrinkle and ridges)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("theta,axis", [(0.0, 1), (math.pi / 2, 0)])
def test_wrinkle_tilt_shifts_the_focus(oracle_mod, theta, axis):
    """A wrinkle whose period is 1000 R is a tilt over the aperture:
    phi = (4 pi / lambda) A 2 pi (u cos theta + v sin theta) / period, and a
    linear aperture phase shifts the focal intensity by (4 pi A f / period)
    (cos theta, sin theta) exactly (the Eq. 2 output chirp has unit modulus).
    A is chosen for a shift of 3 ROI samples, so the deformed lens's
    intensity is the flat lens's moved by 3 samples along x (theta = 0) or y
    (theta = pi/2).  The sine's curvature costs about 1e-5."""
    O = oracle_mod
    lam, f, D = 632.8e-9, 2.5e-3, 0.5e-3
    p = 0.4e-6
    period = 1000 * D / 2
    A = 3 * p * period / (4 * math.pi * f)
    kw = dict(D=D, f=f, lam=lam, M=32, p=p, kind=O.LENS)
    I0 = np.abs(O.field_separable(O.Geometry(**kw))) ** 2
    I1 = np.abs(O.field_separable(O.Geometry(deform=O.Deform(amp=A, period=period, theta=theta), **kw))) ** 2
    if axis == 1:
        a, b = I1[:, 3:], I0[:, :-3]
    else:
        a, b = I1[3:, :], I0[:-3, :]
    assert rel(a, b) < 1e-4
    # and not the unshifted pattern (the test would pass trivially for A = 0)
    assert rel(I1, I0) > 0.1


def _centre_row_phase(O, g):
    a = O.aperture_rows(g, g.c, g.c + 1)[0]
    u = (np.arange(g.N) - g.c) * g.dx
    inside = np.abs(a) > 0
    return u[inside], np.angle(a[inside])


def test_ridge_profile_height_width_and_orientation(oracle_mod):
    """A crease ridge at alpha = pi/2 (the line runs along v through px): along
    the centre row the aperture phase is a bump of peak (4 pi / lambda) h at
    u = px whose half-maximum points lie width/2 on either side (width is the
    FWHM, reading 10); along v it is constant (the row 40 samples below gives
    the same profile).  A clear pupil, so the phase is the deformation's."""
    O = oracle_mod
    lam = 632.8e-9
    D, f = 4e-3, 20e-3
    R = D / 2
    px, width, h = R / 4, R / 3, lam / 8
    g = O.Geometry(D=D, f=f, lam=lam, M=16, p=1e-6, kind=O.CIRC,
                   deform=O.Deform(ridges=[(px, 0.3 * R, math.pi / 2, h, width)]))
    u, ph = _centre_row_phase(O, g)
    k = int(np.argmax(ph))
    assert abs(ph[k] - 4 * math.pi / lam * h) < 1e-6
    assert abs(u[k] - px) <= g.dx
    half = ph[k] / 2
    # half-maximum crossings by linear interpolation on each flank
    left = np.where((ph[:-1] < half) & (ph[1:] >= half))[0][0]
    right = np.where((ph[:-1] >= half) & (ph[1:] < half))[0][-1]
    ul = u[left] + (half - ph[left]) / (ph[left + 1] - ph[left]) * g.dx
    ur = u[right] + (half - ph[right]) / (ph[right + 1] - ph[right]) * g.dx
    assert abs((ur - ul) / width - 1) < 1e-4
    assert abs((ur + ul) / 2 - px) < 1e-3 * width
    # constant along the crease direction
    b = O.aperture_rows(g, g.c - 40, g.c - 39)[0]
    a = O.aperture_rows(g, g.c, g.c + 1)[0]
    both = (np.abs(a) > 0) & (np.abs(b) > 0)
    assert np.max(np.abs(np.angle(a[both]) - np.angle(b[both]))) < 1e-12


def test_wrinkle_profile_period_amplitude_and_taper(oracle_mod):
    """A wrinkle at theta = 0 with taper tau: along the centre row the phase
    is a sine of period `period` (zeros every period/2 from the axis), whose
    envelope is (4 pi / lambda) A at the axis and (1 - tau) of that at the rim
    (reading 10's taper 1 - tau (r/R)^2); along v it is constant up to the
    taper."""
    O = oracle_mod
    lam = 632.8e-9
    D, f = 4e-3, 20e-3
    R = D / 2
    A, period, tau = lam / 16, R / 2.5, 0.5
    g = O.Geometry(D=D, f=f, lam=lam, M=16, p=1e-6, kind=O.CIRC,
                   deform=O.Deform(amp=A, period=period, theta=0.0, taper=tau))
    u, ph = _centre_row_phase(O, g)
    amp0 = 4 * math.pi / lam * A
    # zeros: sign changes of the phase, interpolated, at multiples of period/2
    s = np.where(np.sign(ph[:-1]) * np.sign(ph[1:]) < 0)[0]
    zeros = u[s] - ph[s] / (ph[s + 1] - ph[s]) * g.dx
    half = period / 2
    assert len(zeros) >= 8
    assert np.max(np.abs(zeros / half - np.round(zeros / half))) < 1e-3
    # the crest nearest the axis (u = period/4) carries the axis envelope, the
    # outermost samples the rim envelope
    crest = np.argmin(np.abs(u - period / 4))
    assert abs(ph[crest] / amp0 - 1) < 0.02 + (period / 4 / R) ** 2 * tau
    # envelope |phi| / |sin|: (1 - tau) at the rim, 1 - tau/4 at half the
    # radius (a taper linear in r would give 1 - tau/2 there)
    sn = np.abs(np.sin(2 * math.pi * u / period))
    env = np.abs(ph) / sn.clip(1e-3)
    for lo, hi, target, tol in [(0.97, 1.0, 1 - tau, 0.04), (0.45, 0.55, 1 - tau / 4, 0.03)]:
        ok = (np.abs(u) >= lo * R) & (np.abs(u) <= hi * R) & (sn > 0.3)
        assert ok.sum() > 2
        assert np.max(np.abs(env[ok] / amp0 - target)) < tol, (lo, hi)


@pytest.mark.parametrize("kind,L", [("amp", 0), ("pos", 0), ("phase", 4), ("phase", 8)])
def test_mask_rule_against_exact_arithmetic(oracle_mod, kind, L):
    """The mask rule against exact rational arithmetic on the same doubles:
    a sample is inside iff s dx^2 <= R^2 and its zone (level step) is
    floor(s dx^2 / (lambda f)) (times L/2 for an L-level plate, Fig. 18
    Stage 3).  Rounding of the oracle's IEEE products may decide only samples
    within 1e-9 of a boundary; every other sample must agree exactly."""
    from fractions import Fraction
    O = oracle_mod
    kw = dict(D=0.5e-3, f=2.5e-3, lam=632.8e-9, M=8, p=1e-6)
    if kind == "amp":
        g = O.Geometry(kind=O.FZP_PARAXIAL, **kw)
    elif kind == "pos":
        g = O.Geometry(kind=O.FZP_POSITIVE, **kw)
    else:
        g = O.Geometry(kind=O.FZP_PHASE, levels=L, **kw)
    mask = O.mask_rows(g, 0, g.N)
    d = np.arange(g.N, dtype=np.int64) - g.c
    S = d[:, None] ** 2 + d[None, :] ** 2
    uniq, inv = np.unique(S, return_inverse=True)
    dx2, R2 = Fraction(g.dx) ** 2, Fraction(g.R) ** 2
    rate = dx2 / (Fraction(g.lam) * Fraction(g.f)) * (Fraction(L, 2) if kind == "phase" else 1)
    eps = Fraction(1, 10 ** 9)
    expect = np.full(len(uniq), -1, dtype=np.int64)  # -1: within eps of a boundary
    for k, s in enumerate(uniq.tolist()):
        a = s * dx2
        if abs(a - R2) <= R2 * eps:
            continue
        z = s * rate
        step = z.numerator // z.denominator
        if z - step < eps or z - step > 1 - eps:
            continue
        if a > R2:
            expect[k] = 0
        elif kind == "amp":
            expect[k] = step % 2
        elif kind == "pos":
            expect[k] = 1 - step % 2
        else:
            expect[k] = 1 + step % L
    e = expect[inv.reshape(S.shape)]
    decided = e >= 0
    assert decided.mean() > 0.99
    assert np.array_equal(mask[decided].astype(np.int64), e[decided]), (kind, L)
