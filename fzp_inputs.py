"""Seeded synthetic inputs shared by the library's workloads and the tests.

Only random draws live here -- no optical arithmetic: the deformation
parameters of config 4 (batched membranes) and of the surrogate's training set
(8-vector: wrinkle amplitude, period, orientation, taper, three crease-ridge
heights, wavelength).  Both the product path and the oracle consume these
draws; neither imports the other.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Ridge geometry of the surrogate set, fixed across the dataset (only the heights
# vary): crease lines through (px, py) * R at angle alpha, full width `width_frac`
# times the wrinkle-period scale.
RIDGES = [(0.30, -0.20, 0.35, 0.075), (-0.40, 0.10, 1.60, 0.125), (0.10, 0.45, 2.70, 0.175)]


@dataclass
class Membrane:
    amp: float          # wrinkle amplitude [m]
    period: float       # wrinkle period [m]
    theta: float        # wrinkle orientation [rad]
    taper: float        # radial taper coefficient
    ridges: list        # [(px, py, alpha, height, width)] in metres / radians
    lam: float          # wavelength [m]
    D: float            # aperture diameter [m]


def surrogate_draws(n: int, seed: int, D: float, lam_range=(450e-9, 650e-9), period_range=None):
    """n membranes for the surrogate: A ~ U[0, lambda/4], log-uniform period in
    [1, 20] mm scaled by D / 0.2 m, theta ~ U[0, pi), taper ~ U[0, 1], heights
    ~ U[0, lambda/8], lambda ~ U[lam_range].  Returns (list[Membrane], X[n, 8]) with X
    the raw 8-vector (A/lambda, log10 period, theta, taper, h1/lambda, h2/lambda,
    h3/lambda, lambda)."""
    rng = np.random.default_rng(seed)
    scale = D / 0.2
    pr = period_range or (1e-3 * scale, 20e-3 * scale)
    lam = rng.uniform(*lam_range, n)
    amp = rng.uniform(0, 0.25, n) * lam
    period = np.exp(rng.uniform(np.log(pr[0]), np.log(pr[1]), n))
    theta = rng.uniform(0, np.pi, n)
    taper = rng.uniform(0, 1, n)
    h = rng.uniform(0, 0.125, (n, 3)) * lam[:, None]
    R = D / 2
    out = []
    for k in range(n):
        ridges = [(px * R, py * R, al, h[k, q], wf * 10e-3 * scale) for q, (px, py, al, wf) in enumerate(RIDGES)]
        out.append(Membrane(amp[k], period[k], theta[k], taper[k], ridges, lam[k], D))
    X = np.stack([amp / lam, np.log10(period), theta, taper, h[:, 0] / lam, h[:, 1] / lam, h[:, 2] / lam, lam], 1)
    return out, X


def batch_draws(n: int, seed: int):
    """Config 4: D ~ U[0.05, 0.30] m, lambda in {450, 550, 650} nm, A ~ U[0, lambda/4],
    period ~ U[1, 20] mm, theta ~ U[0, pi), taper ~ U[0, 1], 0-3 ridges with heights
    U[0, lambda/8], widths U[0.5, 5] mm, lines through uniform points of the disc at
    uniform angles."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        D = rng.uniform(0.05, 0.30)
        lam = float(rng.choice([450e-9, 550e-9, 650e-9]))
        R = D / 2
        ridges = []
        for _ in range(int(rng.integers(0, 4))):
            rr, ph = R * np.sqrt(rng.uniform()), rng.uniform(0, 2 * np.pi)
            ridges.append((rr * np.cos(ph), rr * np.sin(ph), rng.uniform(0, np.pi), rng.uniform(0, lam / 8),
                           rng.uniform(0.5e-3, 5e-3)))
        out.append(Membrane(rng.uniform(0, lam / 4), rng.uniform(1e-3, 20e-3), rng.uniform(0, np.pi),
                            rng.uniform(0, 1), ridges, lam, D))
    return out
