"""Pins of the SA-CZT oracle (Sec. 3.6, Fig. 5) against things other than itself:
the paraxial limit, where the method is Eq. 2's Fresnel sum (the O1-O3
oracles); energy conservation of the angular-spectrum step; and the physics
the exact radii of Eq. 3 are for: under the exact propagator the exact-radii
plate focuses to the Airy spot with the binary-FZP efficiency, while the
paraxial-radii plate is aberrated (reading 1)."""
import math

import numpy as np
import pytest


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def sa(oracle_mod):
    from oracle import saczt
    return saczt


def test_paraxial_limit_is_the_fresnel_sum(oracle_mod, sa):
    """With k_z paraxial (h = 0, z_F = f) the SA-CZT evaluates Eq. 2's sum:
    equal to O3 (Bluestein rows then columns) and O1 (Eq. 1 literally)."""
    O = oracle_mod
    g = O.Geometry(D=0.5e-3, f=2.5e-3, lam=632.8e-9, M=16, p=0.4e-6)
    U = sa.field_saczt(g, paraxial=True)
    assert rel(U, O.field_czt(g)) < 1e-10
    assert rel(U, O.field_direct(g)) < 1e-10
    # off-axis origin and an odd ROI side through the same sum
    g2 = O.Geometry(D=0.5e-3, f=2.5e-3, lam=632.8e-9, M=11, p=0.5e-6, x0=-3.3e-6)
    assert rel(sa.field_saczt(g2, paraxial=True), O.field_czt(g2)) < 1e-10


def test_paraxial_limit_asymmetric_aperture(oracle_mod, sa):
    """The same limit on a seeded random aperture (no symmetry, so a mirrored
    or transposed zoom fails), against Eq. 2 summed directly here."""
    O = oracle_mod
    g = O.Geometry(D=41 * 1e-6, f=2e-3, lam=632.8e-9, M=9, p=3e-6, dx=1e-6, N=41, x0=-7e-6)
    T = (np.random.default_rng(5).uniform(size=(g.N, g.N)) < 0.4).astype(np.float64)
    U = sa.field_saczt(g, paraxial=True, mask=T)
    lf, k = g.lam * g.f, 2 * math.pi / g.lam
    u = (np.arange(g.N) - g.c) * g.dx
    x = g.x0 + np.arange(g.M) * g.p
    ref = np.zeros((g.M, g.M), complex)
    for n in range(g.M):
        for m in range(g.M):
            ph = np.exp(1j * math.pi * (u[None, :] ** 2 + u[:, None] ** 2) / lf
                        - 2j * math.pi * (x[m] * u[None, :] + x[n] * u[:, None]) / lf)
            ref[n, m] = np.sum(T * ph)
    ref *= np.exp(1j * k * g.f) * np.exp(1j * math.pi * (x[None, :] ** 2 + x[:, None] ** 2) / lf) * g.dx ** 2 / (1j * lf)
    assert rel(U, ref) < 1e-10


def test_angular_step_conserves_energy(oracle_mod, sa):
    """exp(i h f) has unit modulus and no component is evanescent at dx > lambda / 2,
    so the residual step keeps sum |U1|^2 = sum |T|^2 (Parseval)."""
    O = oracle_mod
    g = O.Geometry(D=0.5e-3, f=2.5e-3, lam=632.8e-9, M=8, p=0.4e-6, kind=O.FZP_EXACT)
    assert g.dx > g.lam / 2
    T = O.mask_rows(g, 0, g.N).astype(np.float64)
    U1 = sa.angular_residual(g, sa.pad_size(g.N))
    assert abs(np.sum(np.abs(U1) ** 2) / np.sum(T ** 2) - 1) < 1e-12
    # and h vanishes at the fit's anchors K = 0 and K = k_max (reading of Fig. 5)
    k0 = 2 * math.pi / g.lam
    kmax, c, d = sa.fit(k0)
    assert abs(k0 - c * kmax) < 1e-9 * k0
    assert abs(math.sqrt(k0 ** 2 - kmax ** 2) - (c * kmax + d * kmax)) < 1e-9 * k0


def f5_fields_of(O, sa):
    """A 2 mm plate at f/5 (N = 2529, 158 zones, NA 0.1) under the exact
    propagator, with exact and with paraxial radii."""
    kw = dict(D=2e-3, f=10e-3, lam=632.8e-9, M=128, p=632.8e-9 * 5 / 8)
    ge = O.Geometry(kind=O.FZP_EXACT, **kw)
    gp = O.Geometry(kind=O.FZP_PARAXIAL, **kw)
    return ge, sa.field_saczt(ge), gp, sa.field_saczt(gp)


@pytest.fixture(scope="module")
def f5_fields(oracle_mod, sa):
    return f5_fields_of(oracle_mod, sa)


def test_exact_radii_focus_under_the_exact_propagator(oracle_mod, f5_fields):
    """The exact-radii plate (Eq. 3) focuses to the Airy spot: FWHM within 1 %
    of 1.028994 lambda f / D, main-lobe DE within 2 % of EE(r_null) / pi^2."""
    O = oracle_mod
    ge, Ue, _, _ = f5_fields
    m = O.metrics(ge, Ue)
    airy = O.airy_fwhm_factor() * ge.lam * ge.f / (2 * ge.R)
    assert abs(m["fwhm_x"] / airy - 1) < 1e-2
    assert abs(m["de_lobe"] / (O.airy_encircled(O.AIRY_NULL) * O.binary_fzp_efficiency()) - 1) < 2e-2


def test_paraxial_radii_are_aberrated_under_the_exact_propagator(oracle_mod, f5_fields):
    """Reading 1: the paraxial radii under the exact kernel carry spherical
    aberration (about 1.2 rad at this plate's edge): a lower peak than the
    exact-radii plate by several per cent, the same disc and zone count."""
    O = oracle_mod
    ge, Ue, gp, Up = f5_fields
    pe = np.abs(Ue[ge.M // 2, ge.M // 2]) ** 2
    pp = np.abs(Up[gp.M // 2, gp.M // 2]) ** 2
    assert pp < 0.95 * pe  # measured 0.877
