"""Form (a), the Bluestein row/column CZT (Sec. 2.6, Fig. 2), against the CPU
FP64 oracle through the C ABI.  Tolerances: relative L2 error of the ROI
intensity <= 1e-6 (FP64) and <= 1e-4 (FP32); FWHM within 0.01 %; DE within
0.01 percentage points."""
import numpy as np
import pytest

from gpu_util import rel_l2, run_plan

pytestmark = pytest.mark.gpu

TOL = {0: 1e-6, 1: 1e-4}  # PREC_FP64, PREC_FP32


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2609_01978_gb300 as fzp
    return fzp, torch, oracle


def _plan(fzp, g, precision, **kw):
    return fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, dx=g.dx, N=g.N, form=fzp.FORM_BLUESTEIN,
                    precision=precision, **kw)


@pytest.fixture(scope="module")
def config1(env):
    fzp, torch, O = env
    g = O.Geometry(D=4e-3, f=20e-3, lam=632.8e-9, M=256, p=0.2e-6)
    U = O.field_czt(g)
    return g, U, O.metrics(g, U)


@pytest.mark.parametrize("precision,conv", [(0, 0), (1, 1), (1, 2)])
def test_config1_full_aperture(env, config1, precision, conv):
    """Config 1: D = 4 mm, f/# = 5, 632.8 nm, N = 5057 (FP64 runs the four-step
    split L = 2 x 4096, FP32 the single 8192-point pass or two partitioned
    blocks of 3840 columns), 256^2 ROI at 0.2 um."""
    fzp, torch, O = env
    g, Uref, mref = config1
    with _plan(fzp, g, precision, conv=conv) as plan:
        info = plan.info
        assert info["N"] == g.N == 5057 and info["total_zones"] == g.total_zones()
        assert info["fft_length"] == 8192
        assert info["conv"] == (2 if conv == 2 else 1)
        U, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
        Iref = np.abs(Uref) ** 2
        assert rel_l2(I, Iref) <= TOL[precision]
        assert rel_l2(U, Uref) <= TOL[precision]
        dev = torch.from_numpy(U).to("cuda:0")
        m = plan.metrics(dev)
    assert abs(m["fwhm_x"] / mref["fwhm_x"] - 1) < 1e-4
    assert abs(m["fwhm_y"] / mref["fwhm_y"] - 1) < 1e-4
    assert abs(m["de_lobe"] - mref["de_lobe"]) < 1e-4
    assert abs(m["de_roi"] - mref["de_roi"]) < 1e-4
    assert m["aperture_count"] == O.count_aperture(g)


def test_metrics_extractor_on_oracle_field(env, config1):
    """The device extractor applied to the oracle's own field reproduces the
    oracle's metrics (isolates Stage 4 from the propagation)."""
    fzp, torch, O = env
    g, Uref, mref = config1
    with _plan(fzp, g, 1) as plan:
        m = plan.metrics(torch.from_numpy(Uref).to("cuda:0"))
    for k in ("fwhm_x", "fwhm_y", "de_lobe", "de_roi", "p_in", "peak", "strehl", "mtf_half_cut"):
        assert abs(m[k] / mref[k] - 1) < 1e-9, (k, m[k], mref[k])
    assert np.max(np.abs(np.array(m["mtf16"]) - mref["mtf16"])) < 1e-9


@pytest.mark.parametrize("conv", [1, 2])
def test_four_step_fp32_and_ragged_rows(env, conv):
    """FP32 with L = 16384 = 2 x 8192 (four-step path) or three partitioned
    blocks, odd row ranges, a single row on the axis."""
    fzp, torch, O = env
    g = O.Geometry(D=4e-3 * 9001 / 5057, f=20e-3 * 9001 / 5057, lam=632.8e-9, M=128, p=0.3e-6, N=9001)
    with _plan(fzp, g, 1, conv=conv) as plan:
        assert plan.info["fft_length"] == 16384
        for (j0, j1) in [(0, g.N), (4321, 4321 + 777), (g.c, g.c + 1)]:
            _, I = run_plan(fzp, torch, plan, g.M, j0, j1)
            Iref = np.abs(O.field_czt(g, j0, j1)) ** 2
            assert rel_l2(I, Iref) <= 1e-4, (j0, j1)


def test_row_range_linearity_and_empty(env):
    fzp, torch, O = env
    g = O.Geometry(D=4e-3 / 2, f=20e-3 / 2, lam=632.8e-9, M=64, p=0.4e-6)
    with _plan(fzp, g, 0) as plan:
        Ufull, _ = run_plan(fzp, torch, plan, g.M, 0, g.N)
        dev = torch.device("cuda:0")
        U = torch.zeros((g.M, g.M), dtype=torch.complex128, device=dev)
        for (a, b) in [(0, 700), (700, 1300), (1300, g.N)]:
            plan.propagate_roi(a, b, U, accumulate=True)
        torch.cuda.synchronize()
        assert rel_l2(U.cpu().numpy(), Ufull) < 1e-12
        Uz, Iz = run_plan(fzp, torch, plan, g.M, 17, 17)  # empty range: zero field
        assert np.all(Uz == 0)
        with pytest.raises(fzp.FzpError):
            plan.propagate_roi(0, g.N + 1, U)
        with pytest.raises(fzp.FzpError):
            plan.propagate_roi(5, 4, U)


@pytest.mark.parametrize("precision,conv", [(0, 0), (1, 1), (1, 2)])
def test_deformed_membrane(env, precision, conv):
    """Membrane deformation phase (4 pi / lambda) w with a sine wrinkle, taper
    and two crease ridges (config 4's model) against the oracle."""
    fzp, torch, O = env
    lam = 550e-9
    d = dict(amp=lam / 4, period=2.1e-4, theta=0.6, taper=0.3,
             ridges=[(5e-5, -1e-4, 0.4, lam / 8, 8e-5), (-2e-4, 3e-5, 2.2, lam / 10, 1.2e-4)])
    g = O.Geometry(D=2e-3, f=1e-2, lam=lam, M=128, p=lam * 5 / 8, deform=O.Deform(**d))
    with fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, dx=g.dx, N=g.N, form=fzp.FORM_BLUESTEIN,
                  precision=precision, deform=fzp.make_deform(**d), conv=conv) as plan:
        _, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
    Iref = np.abs(O.field_czt(g)) ** 2
    assert rel_l2(I, Iref) <= TOL[precision]


@pytest.mark.parametrize("conv", [1, 2])
def test_config2_sampled_stripes(env, conv):
    """Config 2 (D = 0.25 m, N = 316,057, L = 2^19, 512^2 ROI at lambda f/#/8):
    the field is linear in rows, so 1024-row stripes at random offsets are
    compared with the oracle on the same rows (single convolution, or 89
    partitioned blocks of 3584 columns)."""
    fzp, torch, O = env
    lam, F = 632.8e-9, 5.0
    g = O.Geometry(D=0.25, f=1.25, lam=lam, M=512, p=lam * F / 8)
    assert g.N == 316057
    rng = np.random.default_rng(1)
    with _plan(fzp, g, 1, conv=conv) as plan:
        assert plan.info["fft_length"] == 1 << 19
        for j0 in [g.c - 512, int(rng.integers(0, g.N - 1024))]:
            _, I = run_plan(fzp, torch, plan, g.M, j0, j0 + 1024)
            Iref = np.abs(O.field_czt(g, j0, j0 + 1024)) ** 2
            assert rel_l2(I, Iref) <= 1e-4, j0
