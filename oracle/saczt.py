"""Oracle of the semi-analytical chirp-z transform (SA-CZT, Sec. 3.6, Fig. 5).

TEST INFRASTRUCTURE ONLY (see the package docstring): only the tests,
``__graft_entry__.smoke()`` and bench.py's CPU legs may use it.

The SA-CZT propagates the binary amplitude FZP with the exact zone radii of
Eq. 3 by angular-spectrum propagation without the paraxial approximation,
split into an exact residual applied on the padded grid and a quadratic part
evaluated semi-analytically as a Fresnel integral with a CZT zoom onto the
ROI.  In the paper's order (Fig. 5, Stage 3):

  1  A = fft2 of the mask, zero-padded to P x P (no input chirp)
  2  A *= exp(i h(K) f), h(K) = k_z(K) - c k_max - d K^2 / k_max,
     k_z = sqrt(k0^2 - K^2); evanescent components (K^2 > k0^2) zeroed
  3-4 U1 = ifft2(A), times the separable chirp exp(i k0 (u^2 + v^2) / (2 z_F))
  5  the Fourier sum of step 4 at the ROI frequencies x / (lambda z_F) (the
     CZT zoom: frequency step dx_out k_max / |4 pi d f|), times dx_in^2 and
     the prefactor alpha and the output chirp exp(i k0 (x^2 + y^2) / (2 z_F)).

Readings taken here (the figure gives the fit only by its anchor):
  * the quadratic c k_max + d K^2 / k_max matches k_z at K = 0 and at
    K = k_max = 2 k0 / 3: c = k0 / k_max, d = (sqrt(k0^2 - k_max^2) - k0) / k_max;
  * the quadratic part exp(i d f K^2 / k_max) is the Fresnel transfer function
    of the distance z_F = -2 k0 d f / k_max without its constant phase
    exp(i k0 z_F) (so the zoom step dx_out / (lambda z_F) equals the figure's
    dx_out k_max / |4 pi d f|); with the constant phases of both parts,
    alpha = exp(i c k_max f) / (i lambda z_F) = exp(i k0 f) / (i lambda z_F);
  * the padded grid is P x P (P a power of two >= 1.5 N, the figure's 1.5 N
    rounded up for radix-2 transforms) with the mask's centre sample at index
    P/2, so that u_p = (p - P/2) dx_in;
  * the figure's empirical (2 pi)^2 division of the lobe power belongs to its
    own extractor's normalisation; this library's extractor (Fig. 2 Stage 4)
    is applied unchanged.
``paraxial=True`` replaces k_z by its paraxial form, so that h = 0 and
z_F = f: the method then reduces to Eq. 2's Fresnel sum, the oracle's O1-O3
(a pin).
"""
from __future__ import annotations

import math

import numpy as np


def pad_size(N: int) -> int:
    """Smallest power of two >= 1.5 N."""
    P = 1
    while P < 1.5 * N:
        P *= 2
    return P


def fit(k0: float):
    """(k_max, c, d) of the quadratic fit of k_z (reading above)."""
    kmax = 2.0 * k0 / 3.0
    c = k0 / kmax
    d = (math.sqrt(k0 * k0 - kmax * kmax) - k0) / kmax
    return kmax, c, d


def angular_residual(g, P: int, paraxial: bool = False, mask=None) -> np.ndarray:
    """Steps 1-4 without the chirp: U1 = ifft2(fft2(T) exp(i h f)) on the P x P
    padded grid (mask centred at P/2)."""
    from . import mask_rows
    T = mask_rows(g, 0, g.N).astype(np.float64) if mask is None else mask
    G = np.zeros((P, P), dtype=np.complex128)
    o = P // 2 - g.c
    G[o:o + g.N, o:o + g.N] = T
    A = np.fft.fft2(G)
    if paraxial:
        return np.fft.ifft2(A)
    k0 = 2.0 * math.pi / g.lam
    kf = 2.0 * math.pi * np.fft.fftfreq(P, d=g.dx)
    K2 = kf[None, :] ** 2 + kf[:, None] ** 2
    prop = K2 < k0 * k0
    kz = np.sqrt(np.where(prop, k0 * k0 - K2, 0.0))
    kmax, c, d = fit(k0)
    h = kz - c * kmax - d * K2 / kmax
    return np.fft.ifft2(np.where(prop, A * np.exp(1j * h * g.f), 0.0))


def z_fresnel(g, paraxial: bool = False) -> float:
    """Distance of the Fresnel part, z_F = -2 k0 d f / k_max (f when paraxial)."""
    if paraxial:
        return g.f
    k0 = 2.0 * math.pi / g.lam
    kmax, _, d = fit(k0)
    return -2.0 * k0 * d * g.f / kmax


def field_saczt(g, P: int = 0, paraxial: bool = False, mask=None) -> np.ndarray:
    """U[n, m] at (x_m, y_n) by the SA-CZT (Fig. 5), in FP64.  `g` is an
    oracle Geometry (kind FZP_EXACT for the exact radii of Eq. 3); `mask`
    overrides the aperture (N x N)."""
    P = P or pad_size(g.N)
    U1 = angular_residual(g, P, paraxial, mask)
    zF = z_fresnel(g, paraxial)
    k0 = 2.0 * math.pi / g.lam
    u = (np.arange(P) - P // 2) * g.dx
    x = g.coords_out()
    chirp = np.exp(1j * k0 * u * u / (2.0 * zF))
    # the Fourier sum at the ROI frequencies x / (lambda z_F), rows then columns
    Kx = np.exp(-1j * k0 * np.outer(x, u) / zF) * chirp[None, :]
    S = Kx @ U1 @ Kx.T  # S[n, m] = sum_{q,p} Kx[n, q] U1[q, p] Kx[m, p]
    alpha = np.exp(1j * k0 * g.f) / (1j * g.lam * zF)
    return alpha * g.dx * g.dx * np.exp(1j * k0 * (x[None, :] ** 2 + x[:, None] ** 2) / (2.0 * zF)) * S
