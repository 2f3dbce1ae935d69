"""CPU FP64 oracle for the Fresnel zone plate propagator.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
library (``paper_2609_01978_gb300``) never imports it, and this package never
imports the product: the two share no code.

What lives here
---------------
* ``Geometry`` -- the sampling grids of Fig. 2, Stage 1 (dx_in, N forced odd,
  centred input grid, ROI grid) and the zone count of Eq. 3; the aperture
  kinds: binary plate (negative- or positive-centred), exact-radius plate,
  L-level phase plate, ideal lens, clear pupil, each with an optional
  membrane deformation ``Deform``.
* ``field_direct`` (O1, Eq. 1 literally), ``field_separable`` (O2, Eq. 2 as
  K T K^T) and ``field_czt`` (O3, Bluestein CZT rows then columns, Fig. 2) --
  thin ctypes wrappers over ``fzp_oracle.c``.
* ``metrics`` -- the shared metric extractor of Fig. 2, Stage 4 / Fig. 18,
  Stage 5: FWHM of the centre row by cubic spline, main-lobe diffraction
  efficiency, MTF by |fft2(I)| radially averaged (numpy / scipy primitives).
* closed forms used as pins: Airy FWHM and encircled energy (Sec. 2.3), the
  circular-pupil MTF, binary-FZP efficiency 1/pi^2 (Sec. 2.3).

Every function cites the passage it follows.  Readings of passages that are
ambiguous are stated where they are taken.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fzp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

# Aperture kinds (match the enum in fzp_oracle.c).
FZP_PARAXIAL = 0
LENS = 1
FZP_EXACT = 2
CIRC = 3
FZP_PHASE = 4  # L-level phase FZP (Fig. 18): transmission e^{-2 pi i q / L}
FZP_POSITIVE = 5  # binary amplitude FZP with the centre zone open (even zones open)

# First zero of J1 divided by pi: Airy null radius in units of lambda f / D.
AIRY_NULL = 3.8317059702075125 / math.pi  # 1.2196698...


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, OpenMP).  Returns the library path."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", _LIB_PATH, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB_PATH


class _Deform(ctypes.Structure):
    _fields_ = [("amp", ctypes.c_double), ("period", ctypes.c_double), ("theta", ctypes.c_double),
                ("taper", ctypes.c_double), ("n_ridges", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("ridge_px", ctypes.c_double * 3), ("ridge_py", ctypes.c_double * 3),
                ("ridge_alpha", ctypes.c_double * 3), ("ridge_h", ctypes.c_double * 3),
                ("ridge_width", ctypes.c_double * 3)]


class _Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("dx", ctypes.c_double), ("lam", ctypes.c_double),
                ("f", ctypes.c_double), ("R", ctypes.c_double), ("M", ctypes.c_int32),
                ("kind", ctypes.c_int32), ("p", ctypes.c_double), ("x0", ctypes.c_double),
                ("deform", ctypes.POINTER(_Deform)), ("levels", ctypes.c_int32), ("pad2_", ctypes.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        i64 = ctypes.c_int64
        for name, args in {
            "orc_mask_rows": [pp, i64, i64, ctypes.POINTER(ctypes.c_uint8)],
            "orc_aperture_rows": [pp, i64, i64, dp, dp],
            "orc_fft": [i64, dp, dp, ctypes.c_int],
            "orc_czt": [i64, dp, dp, i64, ctypes.c_double, ctypes.c_double, dp, dp],
            "orc_czt_direct": [i64, dp, dp, i64, ctypes.c_double, ctypes.c_double, dp, dp],
            "orc_field_direct": [pp, i64, i64, dp, dp],
            "orc_field_separable": [pp, i64, i64, dp, dp],
            "orc_field_czt": [pp, i64, i64, ctypes.c_int, dp, dp],
        }.items():
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _lib.orc_count_aperture.argtypes = [pp]
        _lib.orc_count_aperture.restype = ctypes.c_int64
        _lib.orc_max_threads.argtypes = []
        _lib.orc_max_threads.restype = ctypes.c_int
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------------------
# Geometry (Fig. 2, Stage 1; Eq. 5-7; Eq. 3 for the zone count)
# ---------------------------------------------------------------------------

@dataclass
class Deform:
    """Membrane deformation w(u,v) [m]; phase phi = (4 pi / lambda) w.

    w = amp sin(2 pi (u cos theta + v sin theta)/period) (1 - taper (r/R)^2)
        + sum_k h_k exp(-d_k^2 / (2 sigma_k^2)),  sigma_k = width_k / 2.3548,
    d_k the distance to the crease line through (px_k, py_k) at angle alpha_k.
    """
    amp: float = 0.0
    period: float = 1e-2
    theta: float = 0.0
    taper: float = 0.0
    ridges: list = field(default_factory=list)  # [(px, py, alpha, h, width), ...] up to 3

    def to_c(self) -> _Deform:
        d = _Deform()
        d.amp, d.period, d.theta, d.taper = self.amp, self.period, self.theta, self.taper
        d.n_ridges = len(self.ridges)
        for k, (px, py, al, h, w) in enumerate(self.ridges[:3]):
            d.ridge_px[k], d.ridge_py[k], d.ridge_alpha[k], d.ridge_h[k], d.ridge_width[k] = px, py, al, h, w
        return d


@dataclass
class Geometry:
    """Sampling grids.

    Input plane (Fig. 2, Stage 1): dx_in defaults to lambda f / (4 D), i.e. four
    samples across the outermost zone width Delta r_N = lambda f / D (Eq. 5),
    twice the Nyquist bound of Eq. 6; N = ceil(D / dx_in), forced odd, so that
    pixel c = (N-1)/2 sits on the optical axis.  Aperture radius
    R_eff = min(D/2, lambda f / (2 dx_in)) (Fig. 2, Stage 2).
    ROI (Fig. 2, Stage 1, decoupled): M samples at pitch p; reading taken here:
    x_m = (m - M/2) p so that sample M/2 is on the axis, unless ``x0`` gives
    the first ROI coordinate (the same on both axes: x_m = x0 + m p,
    y_n = x0 + n p, the A of Eq. 10 taken from the first ROI coordinate).
    """
    D: float
    f: float
    lam: float
    M: int
    p: float
    dx: Optional[float] = None
    N: Optional[int] = None
    kind: int = FZP_PARAXIAL
    deform: Optional[Deform] = None
    levels: int = 0  # FZP_PHASE: phase levels L (>= 2)
    x0: Optional[float] = None  # first ROI coordinate, both axes (None: centred on the focus)

    def __post_init__(self):
        if self.kind == FZP_PHASE and self.levels < 2:
            raise ValueError("a phase FZP needs levels >= 2")
        if self.dx is None:
            # Fig. 18 Stage 1: dx_in = Lambda_edge / (S_samp max(L, 2)), Lambda_edge =
            # lambda f / R, S_samp = 4; for the amplitude plate (and L = 2) this is
            # lambda f / (4 D)
            mult = max(self.levels, 2) if self.kind == FZP_PHASE else 2
            self.dx = self.lam * self.f / (2.0 * mult * self.D)
        if self.N is None:
            n = int(math.ceil(self.D / self.dx))
            self.N = n + 1 if n % 2 == 0 else n
        if self.N % 2 == 0:
            raise ValueError("N must be odd (centred grid)")
        self.R = min(self.D / 2.0, self.lam * self.f / (2.0 * self.dx))
        if self.x0 is None:
            self.x0 = -(self.M // 2) * self.p
        self._deform_c = self.deform.to_c() if self.deform is not None else None

    @property
    def c(self) -> int:
        return (self.N - 1) // 2

    @property
    def fnum(self) -> float:
        return self.f / self.D

    def total_zones(self) -> int:
        """Total_Zones = floor(n_exact), n_exact solving (lambda^2/4) n^2 + lambda f n = R^2 (Eq. 3)."""
        a, b, c = self.lam ** 2 / 4.0, self.lam * self.f, -self.R ** 2
        n = (-b + math.sqrt(b * b - 4 * a * c)) / (2 * a)
        return int(math.floor(n))

    def params(self) -> _Params:
        P = _Params()
        P.N, P.dx, P.lam, P.f, P.R = self.N, self.dx, self.lam, self.f, self.R
        P.M, P.kind, P.p, P.x0 = self.M, self.kind, self.p, self.x0
        P.levels = self.levels
        P.deform = ctypes.pointer(self._deform_c) if self._deform_c is not None else None
        return P

    def coords_out(self) -> np.ndarray:
        return self.x0 + np.arange(self.M) * self.p

    def r_null(self) -> float:
        """First Airy null, 1.21967 lambda f / D (the paper rounds it to 1.22, Fig. 2)."""
        return AIRY_NULL * self.lam * self.f / (2.0 * self.R)


# ---------------------------------------------------------------------------
# Aperture and field
# ---------------------------------------------------------------------------

def mask_rows(g: Geometry, j0: int, j1: int) -> np.ndarray:
    out = np.zeros((j1 - j0, g.N), dtype=np.uint8)
    P = g.params()
    rc = lib().orc_mask_rows(ctypes.byref(P), j0, j1, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    assert rc == 0
    return out


def aperture_rows(g: Geometry, j0: int, j1: int) -> np.ndarray:
    re = np.zeros((j1 - j0, g.N))
    im = np.zeros_like(re)
    P = g.params()
    assert lib().orc_aperture_rows(ctypes.byref(P), j0, j1, _dptr(re), _dptr(im)) == 0
    return re + 1j * im


def count_aperture(g: Geometry) -> int:
    P = g.params()
    return int(lib().orc_count_aperture(ctypes.byref(P)))


def _field(fn: str, g: Geometry, j0: int, j1: int, *extra) -> np.ndarray:
    re = np.zeros((g.M, g.M))
    im = np.zeros_like(re)
    P = g.params()
    rc = getattr(lib(), fn)(ctypes.byref(P), j0, j1, *extra, _dptr(re), _dptr(im))
    if rc != 0:
        raise RuntimeError(f"{fn} failed with code {rc}")
    return re + 1j * im


def field_direct(g: Geometry, j0: int = 0, j1: Optional[int] = None) -> np.ndarray:
    """O1: Eq. 1 summed literally over aperture rows [j0, j1).  out[n, m] at (x_m, y_n)."""
    return _field("orc_field_direct", g, j0, g.N if j1 is None else j1)


def field_separable(g: Geometry, j0: int = 0, j1: Optional[int] = None) -> np.ndarray:
    """O2: Eq. 2 as Pre * chirp_out * (K T K^T) over aperture rows [j0, j1)."""
    return _field("orc_field_separable", g, j0, g.N if j1 is None else j1)


def field_czt(g: Geometry, j0: int = 0, j1: Optional[int] = None, threads: int = 0) -> np.ndarray:
    """O3: Bluestein CZT rows then columns (Fig. 2, Stage 3; Eq. 9-10; Sec. 2.6)."""
    return _field("orc_field_czt", g, j0, g.N if j1 is None else j1, int(threads))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def fft(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    re = np.ascontiguousarray(x.real, dtype=np.float64).copy()
    im = np.ascontiguousarray(x.imag, dtype=np.float64).copy()
    assert lib().orc_fft(len(re), _dptr(re), _dptr(im), 1 if inverse else 0) == 0
    return re + 1j * im


def czt(x: np.ndarray, M: int, alpha: float, omega: float, direct: bool = False) -> np.ndarray:
    """Eq. 9 with A = exp(2 pi i alpha), W = exp(-2 pi i omega)."""
    xr = np.ascontiguousarray(x.real, dtype=np.float64)
    xi = np.ascontiguousarray(x.imag, dtype=np.float64)
    Xr = np.zeros(M)
    Xi = np.zeros(M)
    fn = lib().orc_czt_direct if direct else lib().orc_czt
    assert fn(len(xr), _dptr(xr), _dptr(xi), M, alpha, omega, _dptr(Xr), _dptr(Xi)) == 0
    return Xr + 1j * Xi


# ---------------------------------------------------------------------------
# Metric extractor (Fig. 2 Stage 4; Fig. 18 Stage 5)
# ---------------------------------------------------------------------------

MTF_BINS = 200  # Fig. 18: 200 radial bins


def fwhm_row(row: np.ndarray, p: float) -> float:
    """FWHM of a centre row through the focus (Fig. 2 Stage 4, Fig. 18 Stage 5).

    Peak: 3-point parabola through the on-axis sample and its neighbours
    (Fig. 18 'parabolic peak').  Half-maximum crossings: roots of the
    not-a-knot cubic spline of the row (MATLAB 'spline' default) on either side
    of the peak, solved to 1e-12 px instead of the x100 / x16 upsampling.
    """
    from scipy.interpolate import CubicSpline
    from scipy.optimize import brentq

    M = len(row)
    k = M // 2
    ym, y0, yp = row[k - 1], row[k], row[k + 1]
    den = ym - 2 * y0 + yp
    peak = y0 - 0.125 * (yp - ym) ** 2 / den if den != 0 else y0
    half = 0.5 * peak
    cs = CubicSpline(np.arange(M, dtype=np.float64), row, bc_type="not-a-knot")
    m = k
    while m > 0 and row[m] >= half:
        m -= 1
    xl = brentq(lambda t: cs(t) - half, m, m + 1, xtol=1e-13)
    m = k
    while m < M - 1 and row[m] >= half:
        m += 1
    xr = brentq(lambda t: cs(t) - half, m - 1, m, xtol=1e-13)
    return (xr - xl) * p


def mtf_radial(I: np.ndarray, p: float, bins: int = MTF_BINS):
    """OTF = |fft2(I)| normalised at DC, radially averaged in `bins` equal bins
    over [0, nu_Nyq], nu_Nyq = 1/(2p) (Fig. 2 Stage 4, Fig. 18 Stage 5).

    Reading: FFT sample (ku, kv) (integer frequency indices, numpy fftfreq
    order) has radial frequency |k| / (M p) and falls in bin
    floor(bins |k| / (M/2)), evaluated exactly in integers so that samples on a
    bin edge have a well-defined bin.  Returns (bin centres [cycles/m], means).
    """
    M = I.shape[0]
    otf = np.abs(np.fft.fft2(I))
    otf = otf / otf[0, 0]
    k = np.rint(np.fft.fftfreq(M) * M).astype(np.int64)
    r2 = k[None, :] ** 2 + k[:, None] ** 2
    q = (4 * bins * bins * r2) // (M * M)
    b = np.floor(np.sqrt(q.astype(np.float64))).astype(np.int64)
    b -= (b * b > q).astype(np.int64)
    b += ((b + 1) * (b + 1) <= q).astype(np.int64)
    ok = b < bins
    s = np.bincount(b[ok], weights=otf[ok], minlength=bins)
    n = np.bincount(b[ok], minlength=bins)
    nyq = 1.0 / (2.0 * p)
    centres = (np.arange(bins) + 0.5) * nyq / bins
    with np.errstate(invalid="ignore"):
        mean = s / n
    return centres, mean


def mtf_at(centres: np.ndarray, mean: np.ndarray, nu: float) -> float:
    ok = np.isfinite(mean)
    return float(np.interp(nu, centres[ok], mean[ok]))


def metrics(g: Geometry, U: np.ndarray, p_in_count: Optional[int] = None) -> dict:
    """All metrics of the extractor for a ROI field U[n, m]."""
    I = np.abs(U) ** 2
    M, p = g.M, g.p
    k = M // 2
    x = g.coords_out()
    r = np.hypot(x[None, :], x[:, None])
    if p_in_count is None:
        p_in_count = count_aperture(g)
    P_in = p_in_count * g.dx ** 2
    lobe = I[r <= g.r_null()].sum() * p * p
    nu_cut = 2.0 * g.R / (g.lam * g.f)
    centres, mean = mtf_radial(I, p)
    return {
        "fwhm_x": fwhm_row(I[k, :], p),
        "fwhm_y": fwhm_row(I[:, k], p),
        "de_lobe": lobe / P_in,
        "de_roi": I.sum() * p * p / P_in,
        "p_in": P_in,
        "p_in_disc": math.pi * g.R ** 2,
        "peak": float(I[k, k]),
        "strehl": float(I[k, k]) / (math.pi * g.R ** 2 / (g.lam * g.f)) ** 2,
        "mtf_half_cut": mtf_at(centres, mean, 0.5 * nu_cut),
        "mtf16": np.array([mtf_at(centres, mean, (q + 0.5) * nu_cut / 16) for q in range(16)]),
    }


# ---------------------------------------------------------------------------
# Closed forms (Sec. 2.3)
# ---------------------------------------------------------------------------

def airy_fwhm_factor() -> float:
    """FWHM of |2 J1(x)/x|^2 in units of lambda f / D: 1.028994 (Sec. 2.3 prints 1.028 / 1.029)."""
    from scipy.optimize import brentq
    from scipy.special import j1

    def h(v):
        t = math.pi * v
        return (2 * j1(t) / t) ** 2 - 0.5

    return 2.0 * brentq(h, 0.3, 0.7, xtol=1e-15)


def airy_encircled(r_over_lfD: float) -> float:
    """Encircled energy of the Airy pattern, 1 - J0^2 - J1^2 at x = pi r D/(lambda f)."""
    from scipy.special import j0, j1
    t = math.pi * r_over_lfD
    return 1.0 - j0(t) ** 2 - j1(t) ** 2


def circ_mtf(nu_over_cut: float) -> float:
    """Diffraction-limited MTF of a clear circular pupil, (2/pi)(acos v - v sqrt(1 - v^2))."""
    v = nu_over_cut
    return (2.0 / math.pi) * (math.acos(v) - v * math.sqrt(1.0 - v * v))


def phase_fzp_efficiency(levels: int) -> float:
    """First-order efficiency of an L-level phase kinoform, sinc^2(1/L) =
    (sin(pi/L) / (pi/L))^2 (textbook value for a staircase approximation of a
    blazed profile; 4/pi^2 = 0.405 for L = 2)."""
    x = math.pi / levels
    return (math.sin(x) / x) ** 2


def binary_fzp_efficiency() -> float:
    """First-order efficiency of a binary amplitude FZP, 1/pi^2 (Sec. 2.3)."""
    return 1.0 / math.pi ** 2
