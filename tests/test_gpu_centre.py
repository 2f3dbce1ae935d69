"""The positive-centred binary plate (centre zone open, even zones open; the
centre configuration of the Fig. 18 engine) through the C ABI against the
oracle: the exported mask bit for bit in both forms, the field in FP64 / FP32
(Bluestein form) and split-BF16 (dense form, one level-mode pass, 1-, 2- and
4-CTA clusters), sampled rows of the D = 0.25 m workload, the autotuned plan
and the metric extractor."""
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


def _geom(O, D, f, M, **kw):
    return O.Geometry(D=D, f=f, lam=LAM, M=M, p=LAM * (f / D) / 8, kind=O.FZP_POSITIVE, **kw)


def _plan(fzp, g, form, prec, **kw):
    return fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, dx=g.dx, N=g.N, form=form, precision=prec,
                    centre_open=1, **kw)


def _mask(fzp, torch, plan, j0, j1, N):
    out = torch.empty(((j1 - j0) * N,), dtype=torch.uint8, device="cuda")
    plan.aperture_mask(j0, j1, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(j1 - j0, N)


def test_mask_bit_exact_both_forms(env):
    fzp, torch, O = env
    g = _geom(O, 4e-3, 20e-3, 64)
    for form, prec in [(fzp.FORM_BLUESTEIN, fzp.PREC_FP32), (fzp.FORM_DENSE, fzp.PREC_SPLIT_BF16)]:
        with _plan(fzp, g, form, prec) as plan:
            assert plan.info["centre_open"] == 1
            for j0 in [g.c - 2, 0, g.N - 5, g.N // 3]:
                got = _mask(fzp, torch, plan, j0, j0 + 5, g.N)
                assert np.array_equal(got, O.mask_rows(g, j0, j0 + 5)), (form, j0)
            assert _mask(fzp, torch, plan, g.c, g.c + 1, g.N)[0, g.c] == 1  # the centre zone is open


def test_field_parity(env):
    fzp, torch, O = env
    g = _geom(O, 1e-3, 5e-3, 64)
    Uref = O.field_czt(g)
    Iref = np.abs(Uref) ** 2
    cases = [(fzp.FORM_BLUESTEIN, fzp.PREC_FP64, 1e-6), (fzp.FORM_BLUESTEIN, fzp.PREC_FP32, 1e-4),
             (fzp.FORM_DENSE, fzp.PREC_SPLIT_BF16, 1e-4)]
    for form, prec, tol in cases:
        with _plan(fzp, g, form, prec) as plan:
            U, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
            assert rel_l2(I, Iref) <= tol, (form, prec, rel_l2(I, Iref))
            assert rel_l2(U, Uref) <= 10 * tol, (form, prec)


@pytest.mark.parametrize("cluster", [1, 2, 4])
def test_dense_clusters(env, cluster):
    """M = 256: two kernel-tile pairs, so 4-CTA clusters pad with zero tiles;
    a ragged last stripe (N = 2529 rows is not a multiple of 256)."""
    fzp, torch, O = env
    g = _geom(O, 2e-3, 10e-3, 256)
    assert g.N % 256 != 0
    Iref = np.abs(O.field_czt(g)) ** 2
    with _plan(fzp, g, fzp.FORM_DENSE, fzp.PREC_SPLIT_BF16, cluster=cluster) as plan:
        assert plan.info["passes"] == 1
        _, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
        assert rel_l2(I, Iref) <= 1e-4, (cluster, rel_l2(I, Iref))


def test_d025_sampled_rows(env):
    """The D = 0.25 m workload (N = 316,057, ROI 512^2), positive-centred,
    dense split-BF16 on sampled row ranges against the oracle's rows."""
    fzp, torch, O = env
    g = _geom(O, 0.25, 1.25, 512)
    assert g.N == 316057
    with _plan(fzp, g, fzp.FORM_DENSE, fzp.PREC_SPLIT_BF16) as plan:
        for (j0, j1) in [(g.c - 4, g.c + 4), (g.N // 5, g.N // 5 + 6)]:
            _, I = run_plan(fzp, torch, plan, g.M, j0, j1)
            Iref = np.abs(O.field_czt(g, j0, j1)) ** 2
            assert rel_l2(I, Iref) <= 1e-4, (j0, rel_l2(I, Iref))


def test_autotuned_plan_and_metrics(env):
    """FZP_PREC_AUTO_1E4 picks a form for the positive-centred plate; its field
    meets 1e-4 and the device extractor equals the oracle's (0.01 pp, 0.01 %)."""
    fzp, torch, O = env
    g = _geom(O, 2e-3, 10e-3, 256)
    Uref = O.field_czt(g)
    mref = O.metrics(g, Uref)
    with _plan(fzp, g, fzp.FORM_AUTO, fzp.PREC_AUTO_1E4) as plan:
        U = torch.empty((g.M, g.M), dtype=torch.complex128, device="cuda")
        plan.propagate_roi(0, g.N, U)
        m = plan.metrics(U)
        torch.cuda.synchronize()
        I = np.abs(U.cpu().numpy()) ** 2
    assert rel_l2(I, np.abs(Uref) ** 2) <= 1e-4
    assert abs(m["de_lobe"] - mref["de_lobe"]) < 1e-4
    assert abs(m["fwhm_x"] / mref["fwhm_x"] - 1) < 1e-4
    assert m["aperture_count"] == O.count_aperture(g)


def test_rejected_for_phase_plates(env):
    fzp, torch, O = env
    with pytest.raises(fzp.FzpError) as ei:
        fzp.Plan(D=1e-3, f=5e-3, lam=LAM, M=64, pitch=LAM * 5 / 8, levels=4, centre_open=1)
    assert ei.value.status == fzp.FZP_E_INVALID
