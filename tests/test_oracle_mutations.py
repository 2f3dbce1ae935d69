"""Planted mistakes in the oracle, on the CPU, in a scratch copy of it.

Each mutation is a plausible error in a part of the oracle that the GPU path
is compared against (a sign, a factor, a dropped square, a swapped axis, a
wrong parity); each must make at least one of the oracle's pins fail.  This
shows that the pins tie the oracle to the paper and to the mathematics, not
only to itself.  The unmutated copy passes the same pins (the harness works).
"""
import importlib.util
import os
import shutil
import sys

import pytest

import test_oracle_pins as pins
import test_oracle_saczt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle")

def _sa_paraxial_limit(mod):
    test_oracle_saczt.test_paraxial_limit_is_the_fresnel_sum(mod, mod.saczt)
    test_oracle_saczt.test_paraxial_limit_asymmetric_aperture(mod, mod.saczt)


def _sa_exact_focus(mod):
    test_oracle_saczt.test_exact_radii_focus_under_the_exact_propagator(
        mod, test_oracle_saczt.f5_fields_of(mod, mod.saczt))


# (file, name, exact source text, replacement, pins that must catch it): "c" is
# fzp_oracle.c, "py" the extractor and closed forms in __init__.py, "sa" the
# SA-CZT oracle saczt.py
MUTATIONS = [
    ("c", "negative plate opens even zones",
     "    return ((int64_t)zone & 1) ? 1 : 0;\n  }\n  if (P->kind == ORC_FZP_POSITIVE)",
     "    return ((int64_t)zone & 1) ? 0 : 1;\n  }\n  if (P->kind == ORC_FZP_POSITIVE)",
     [(pins.test_mask_structure, ()), (pins.test_centre_configurations_on_axis, (7,))]),
    ("c", "positive plate equals the negative one",
     "    return ((int64_t)zone & 1) ? 0 : 1;",
     "    return ((int64_t)zone & 1) ? 1 : 0;",
     [(pins.test_centre_configurations_on_axis, (7,))]),
    ("c", "level rate kappa L instead of kappa L / 2",
     "const double kL = orc_kappa(P) * (0.5 * (double)P->levels);",
     "const double kL = orc_kappa(P) * ((double)P->levels);",
     [(pins.test_binary_phase_is_disc_minus_twice_amplitude, ()), (pins.test_phase_fzp_efficiency_ladder, (4,))]),
    ("c", "phase plate focuses the -1 order",
     "a = cexp(-I * 2.0 * M_PI * (double)orc_level(P, j, i) / (double)P->levels);",
     "a = cexp(I * 2.0 * M_PI * (double)orc_level(P, j, i) / (double)P->levels);",
     [(pins.test_phase_fzp_efficiency_ladder, (4,))]),
    ("c", "lens phase of the wrong sign",
     "if (P->kind == ORC_LENS) a = cexp(-I * M_PI",
     "if (P->kind == ORC_LENS) a = cexp(I * M_PI",
     [(pins.test_ideal_lens_gives_airy, ())]),
    ("c", "Bluestein pre-chirp of the wrong sign",
     "cexp(-I * M_PI * omega * (double)n * (double)n);",
     "cexp(I * M_PI * omega * (double)n * (double)n);",
     [(pins.test_o1_o2_o3_agree, ("fzp",)), (pins.test_czt_dft_special_case, (16,))]),
    ("c", "output chirp dropped from O2",
     "      acc *= pre * cexp(I * M_PI * (x * x + y * y) / lf);",
     "      acc *= pre;",
     [(pins.test_o1_o2_o3_agree, ("fzp",))]),
    ("c", "deformation phase 2 pi / lambda instead of 4 pi / lambda",
     "a *= cexp(I * (4.0 * M_PI / P->lambda)",
     "a *= cexp(I * (2.0 * M_PI / P->lambda)",
     [(pins.test_wrinkle_tilt_shifts_the_focus, (0.0, 1)),
      (pins.test_ridge_profile_height_width_and_orientation, ())]),
    ("c", "deformation phase of the wrong sign",
     "a *= cexp(I * (4.0 * M_PI / P->lambda)",
     "a *= cexp(-I * (4.0 * M_PI / P->lambda)",
     [(pins.test_wrinkle_tilt_shifts_the_focus, (0.0, 1))]),
    ("c", "crease normal along the line",
     "double nx = -sin(d->ridge_alpha[k]), ny = cos(d->ridge_alpha[k]);",
     "double nx = cos(d->ridge_alpha[k]), ny = sin(d->ridge_alpha[k]);",
     [(pins.test_ridge_profile_height_width_and_orientation, ())]),
    ("c", "ridge sigma = width / 2",
     "double sigma = d->ridge_width[k] / (2.0 * sqrt(2.0 * log(2.0)));",
     "double sigma = d->ridge_width[k] / 2.0;",
     [(pins.test_ridge_profile_height_width_and_orientation, ())]),
    ("c", "taper linear in r",
     "(1.0 - d->taper * r2);",
     "(1.0 - d->taper * sqrt(r2));",
     [(pins.test_wrinkle_profile_period_amplitude_and_taper, ())]),
    ("c", "wrinkle axes swapped",
     "(u * cos(d->theta) + v * sin(d->theta))",
     "(u * sin(d->theta) + v * cos(d->theta))",
     [(pins.test_wrinkle_tilt_shifts_the_focus, (0.0, 1))]),
    ("c", "aperture count drops the on-axis sample of each row",
     "    total += 2 * lo + 1;",
     "    total += 2 * lo;",
     [(pins.test_count_aperture_is_the_disc_lattice_count, (4e-3, 20e-3, None))]),
    ("c", "aperture count with a strict rim inequality",
     "if ((double)(dj * dj + mid * mid) * dx2 <= R2) lo = mid;",
     "if ((double)(dj * dj + mid * mid) * dx2 < R2) lo = mid;",
     [(pins.test_count_aperture_is_the_disc_lattice_count, (2000 * 2.0 ** -20, 20e-3, 2.0 ** -20))]),
    ("sa", "SA-CZT residual phase of the wrong sign",
     "A * np.exp(1j * h * g.f)",
     "A * np.exp(-1j * h * g.f)",
     [(_sa_exact_focus, ())]),
    ("sa", "SA-CZT Fresnel part over f instead of z_F",
     "return -2.0 * k0 * d * g.f / kmax",
     "return g.f",
     [(_sa_exact_focus, ())]),
    ("sa", "SA-CZT zoom kernel of the wrong sign",
     "np.exp(-1j * k0 * np.outer(x, u) / zF)",
     "np.exp(1j * k0 * np.outer(x, u) / zF)",
     [(_sa_paraxial_limit, ())]),
    ("sa", "SA-CZT mask not centred on the padded grid",
     "o = P // 2 - g.c",
     "o = 0",
     [(_sa_paraxial_limit, ())]),
    ("py", "FWHM peak taken as the on-axis sample (no parabola)",
     "peak = y0 - 0.125 * (yp - ym) ** 2 / den if den != 0 else y0",
     "peak = y0",
     [(pins.test_fwhm_extractor_off_sample_peak, (0.45,))]),
    ("py", "MTF samples at q nu_cut / 16 instead of (q + 1/2) nu_cut / 16",
     "mtf_at(centres, mean, (q + 0.5) * nu_cut / 16)",
     "mtf_at(centres, mean, q * nu_cut / 16)",
     [(pins.test_ideal_lens_gives_airy, ())]),
    ("py", "main-lobe energy with p instead of p^2",
     "lobe = I[r <= g.r_null()].sum() * p * p",
     "lobe = I[r <= g.r_null()].sum() * p",
     [(pins.test_ideal_lens_gives_airy, ()), (pins.test_phase_fzp_efficiency_ladder, (2,))]),
    ("py", "incident power with dx instead of dx^2",
     "P_in = p_in_count * g.dx ** 2",
     "P_in = p_in_count * g.dx",
     [(pins.test_ideal_lens_gives_airy, ())]),
    ("py", "cut-off frequency R / (lambda f)",
     "nu_cut = 2.0 * g.R / (g.lam * g.f)",
     "nu_cut = g.R / (g.lam * g.f)",
     [(pins.test_ideal_lens_gives_airy, ())]),
    ("py", "MTF bins spread over twice the Nyquist frequency",
     "q = (4 * bins * bins * r2) // (M * M)",
     "q = (bins * bins * r2) // (M * M)",
     [(pins.test_mtf_extractor_gaussian, ())]),
    ("py", "Airy FWHM closed form without pi",
     "        t = math.pi * v\n        return (2 * j1(t) / t) ** 2 - 0.5",
     "        t = v\n        return (2 * j1(t) / t) ** 2 - 0.5",
     [(pins.test_closed_forms_match_printed_values, ())]),
    ("py", "circular-pupil MTF with a dropped square root",
     "(math.acos(v) - v * math.sqrt(1.0 - v * v))",
     "(math.acos(v) - v * (1.0 - v * v))",
     [(pins.test_ideal_lens_gives_airy, ())]),
]


def _copy(tmp_path, tag, which=None, old=None, new=None):
    d = tmp_path / f"oracle_{tag}"
    d.mkdir()
    for fn, key in (("__init__.py", "py"), ("fzp_oracle.c", "c"), ("saczt.py", "sa")):
        src = open(os.path.join(SRC, fn)).read()
        if which == key:
            assert src.count(old) == 1, f"mutation target not unique: {old!r}"
            src = src.replace(old, new)
        (d / fn).write_text(src)
    spec = importlib.util.spec_from_file_location(f"oracle_{tag}", d / "__init__.py",
                                                  submodule_search_locations=[str(d)])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod  # dataclasses look their module up here
    spec.loader.exec_module(mod)
    mod.build(force=True)
    mod.saczt = importlib.import_module(f"oracle_{tag}.saczt")
    return mod


def _fails(fn, mod, args):
    """The pin does not pass: an assertion fails, or the mutated oracle's
    output is so far off that the pin's extractor cannot run (a FWHM with no
    half-maximum crossing).  The control copy shows the pins run cleanly."""
    try:
        fn(mod, *args)
    except (AssertionError, ValueError, RuntimeError, FloatingPointError):
        return True
    return False


def test_unmutated_copy_passes(tmp_path):
    mod = _copy(tmp_path, "control")
    for _, _, _, _, checks in MUTATIONS:
        for fn, args in checks:
            assert not _fails(fn, mod, args), fn.__name__


@pytest.mark.parametrize("k", range(len(MUTATIONS)), ids=[m[1] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, k):
    which, name, old, new, checks = MUTATIONS[k]
    mod = _copy(tmp_path, f"m{k}", which, old, new)
    caught = [fn.__name__ for fn, args in checks if _fails(fn, mod, args)]
    assert caught, f"no pin caught: {name}"


# The FP64 surrogate reference (oracle/surrogate.py) against its pins in
# test_oracle_surrogate.py, which read the module through their global `S`.
SURROGATE_MUTATIONS = [
    ("BF16 rounding by truncation",
     "rounded = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000",
     "rounded = u & 0xFFFF0000",
     ["test_bf16_rounding_matches_torch"]),
    ("SiLU derivative taken as the sigmoid's",
     "return s * (1.0 + z * (1.0 - s))",
     "return s * (1.0 - s)",
     ["test_silu_and_its_derivative", "test_gradients_match_central_differences"]),
    ("MSE gradient without its factor 2",
     "G = 2.0 * (yhat - Y) / (B * n_out)",
     "G = (yhat - Y) / (B * n_out)",
     ["test_gradients_match_central_differences"]),
    ("bias gradient averaged over the batch",
     "grads[l] = (r(G).T @ r(H[l]), G.sum(axis=0))",
     "grads[l] = (r(G).T @ r(H[l]), G.mean(axis=0))",
     ["test_gradients_match_central_differences"]),
    ("AdamW without bias correction",
     "c1, c2 = 1 - b1 ** t, 1 - b2 ** t",
     "c1, c2 = 1.0, 1.0",
     ["test_adamw_matches_torch"]),
    ("AdamW without weight decay",
     "(np.sqrt(vW / c2) + eps) + wd * W)",
     "(np.sqrt(vW / c2) + eps))",
     ["test_adamw_matches_torch"]),
]


def _surrogate_copy(tmp_path, tag, old=None, new=None):
    src = open(os.path.join(SRC, "surrogate.py")).read()
    if old is not None:
        assert src.count(old) == 1, f"mutation target not unique: {old!r}"
        src = src.replace(old, new)
    f = tmp_path / f"surrogate_{tag}.py"
    f.write_text(src)
    spec = importlib.util.spec_from_file_location(f"surrogate_{tag}", f)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    return mod


def _run_with(tos, mod, name):
    saved = tos.S
    tos.S = mod
    try:
        getattr(tos, name)()
    except (AssertionError, ValueError, FloatingPointError):
        return True
    finally:
        tos.S = saved
    return False


def test_surrogate_unmutated_copy_passes(tmp_path):
    import test_oracle_surrogate as tos
    mod = _surrogate_copy(tmp_path, "control")
    for _, _, _, names in SURROGATE_MUTATIONS:
        for name in names:
            assert not _run_with(tos, mod, name), name


@pytest.mark.parametrize("k", range(len(SURROGATE_MUTATIONS)), ids=[m[0] for m in SURROGATE_MUTATIONS])
def test_surrogate_planted_mistake_fails_a_pin(tmp_path, k):
    import test_oracle_surrogate as tos
    name, old, new, names = SURROGATE_MUTATIONS[k]
    mod = _surrogate_copy(tmp_path, f"m{k}", old, new)
    assert any(_run_with(tos, mod, n) for n in names), f"no pin caught: {name}"
