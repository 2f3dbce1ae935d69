"""Off-axis ROI (fzp_params.roi_origin = 1, x0 = y0): the first ROI sample at
(x0, x0), so that x_m = x0 + m p on both axes and Eq. 10's A is taken from
the first ROI coordinate (Sec. 2.6).  Every form against the oracle's O3 on
the same grids (relative L2 of I <= 1e-6 FP64, <= 1e-4 FP32 and split-BF16),
through the C ABI."""
import numpy as np
import pytest

from gpu_util import rel_l2, run_plan

pytestmark = pytest.mark.gpu

LAM = 632.8e-9


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


FORMS = [("fp64", 1, 0, 1e-6), ("fp32", 1, 1, 1e-4), ("dense", 2, 2, 1e-4)]
_REF = {}


CASES = [(f, s) for s in (37.3, -100.0) for f in FORMS] + [(FORMS[0], 200.5)]


@pytest.mark.parametrize("form,shift", CASES, ids=[f"{f[0]}-{s}" for f, s in CASES])
def test_offaxis_roi_config1(env, form, shift):
    """Config 1's plate (D = 4 mm, N = 5057, ROI 256^2 at 0.2 um) with the ROI
    origin moved by `shift` pitches from the centred one: windows that hold
    the focus off their centre (37.3 and -100 pitches, every form), and one
    200.5 pitches away that holds only side lobes, four orders of magnitude
    below the peak (FP64 form: the FP32 forms' error is set by the aperture's
    whole sum, not by the weak local field)."""
    fzp, torch, O = env
    name, form_id, prec, tol = form
    p = 0.2e-6
    x0 = -(256 // 2) * p + shift * p
    g = O.Geometry(D=4e-3, f=20e-3, lam=LAM, M=256, p=p, x0=x0)
    if shift not in _REF:
        _REF[shift] = O.field_czt(g)
    Uref = _REF[shift]
    with fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, dx=g.dx, N=g.N, form=form_id, precision=prec,
                  x0=x0) as plan:
        assert plan.info["x0"] == x0
        U, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
    err = rel_l2(I, np.abs(Uref) ** 2)
    print(f"off-axis {name} shift {shift}: rel L2 of I {err:.3e}")
    assert err <= tol, (name, shift, err)
    # the complex field as well (the output chirp and Pre depend on x0)
    assert rel_l2(U, Uref) <= 10 * tol


def test_offaxis_stripe_config2_dense(env):
    """The 0.25 m plate's dense plan with an off-axis ROI, on a stripe of 512
    rows through the axis, against the oracle's same rows."""
    fzp, torch, O = env
    p = LAM * 5 / 8
    x0 = -256 * p + 64.25 * p
    g = O.Geometry(D=0.25, f=1.25, lam=LAM, M=512, p=p, x0=x0)
    j0 = g.c - 256
    Iref = np.abs(O.field_czt(g, j0, j0 + 512)) ** 2
    with fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, form=fzp.FORM_DENSE, precision=fzp.PREC_SPLIT_BF16,
                  x0=x0) as plan:
        _, I = run_plan(fzp, torch, plan, g.M, j0, j0 + 512)
    assert rel_l2(I, Iref) <= 1e-4


def test_offaxis_metrics_rejected(env):
    """The extractor reads the focus at the ROI centre, so an off-axis plan's
    fzp_metrics returns FZP_E_UNSUPPORTED."""
    fzp, torch, O = env
    with fzp.Plan(D=1e-3, f=5e-3, lam=LAM, M=64, pitch=0.4e-6, precision=fzp.PREC_FP32, x0=1e-6) as plan:
        U = torch.zeros((64, 64), dtype=torch.complex128, device="cuda")
        with pytest.raises(fzp.FzpError) as e:
            plan.metrics(U)
        assert e.value.status == fzp.FZP_E_UNSUPPORTED
