"""fzp_metrics_noalloc: the metric extractor for callers that cannot allocate
device memory (their device memory belongs to another allocator, or they run a
loop that must not allocate once started).  It takes the problem parameters
instead of a plan and keeps its scratch in a static device array (M <= 512).

Checked against the plan-based fzp_metrics on the same field, on two calls in a
row (the array keeps the previous call's contents, so the second call shows
that everything that must start at zero is cleared)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2609_01978_gb300 as fzp
    return fzp, torch


KEYS = ("fwhm_x", "fwhm_y", "de_lobe", "de_roi", "p_in", "p_in_disc", "peak", "strehl", "mtf_half_cut")


def test_noalloc_matches_plan_metrics_twice(env):
    fzp, torch = env
    kw = dict(D=4e-3, f=20e-3, lam=632.8e-9, M=256, pitch=0.2e-6)
    with fzp.Plan(form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP32, **kw) as plan:
        N = plan.info["N"]
        U = torch.empty((256, 256), dtype=torch.complex128, device="cuda:0")
        plan.propagate_roi(0, N, U)
        ref = plan.metrics(U)
    # a second, different field so that a call that failed to clear its scratch
    # would carry the first field's sums into the next result
    with fzp.Plan(form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP32, **kw) as plan:
        V = torch.empty_like(U)
        plan.propagate_roi(0, N // 2, V)
        ref_v = plan.metrics(V)
    first = fzp.metrics_noalloc(U, **kw)
    free0 = torch.cuda.mem_get_info()[0]
    second = fzp.metrics_noalloc(U, **kw)
    third = fzp.metrics_noalloc(V, **kw)
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0  # no device memory taken by the calls after set-up
    for got in (first, second):
        for k in KEYS:
            assert abs(got[k] / ref[k] - 1) < 1e-9, (k, got[k], ref[k])
        assert np.max(np.abs(np.array(got["mtf16"]) - np.array(ref["mtf16"]))) < 1e-9
        assert got["aperture_count"] == ref["aperture_count"]
    for k in KEYS:
        assert abs(third[k] / ref_v[k] - 1) < 1e-9, (k, third[k], ref_v[k])


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    fzp, torch = env
    U = torch.zeros((1024, 1024), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(fzp.FzpError) as ei:
        fzp.metrics_noalloc(U, D=4e-3, f=20e-3, lam=632.8e-9, M=1024, pitch=0.2e-6)
    assert ei.value.status == fzp.FZP_E_INVALID and "static scratch" in str(ei.value)


@pytest.mark.parametrize("levels,centre_open", [(4, 0), (0, 1)])
def test_noalloc_phase_and_positive_plates(env, levels, centre_open):
    """A 4-level phase plate (default dx = lambda f / (2 D L), Fig. 18 Stage 1)
    and a positive-centred plate: the same grid and aperture count as the plan,
    so the same metrics."""
    fzp, torch = env
    kw = dict(D=2e-3, f=10e-3, lam=632.8e-9, M=128, pitch=632.8e-9 * 5 / 8, levels=levels, centre_open=centre_open)
    with fzp.Plan(form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP32, **kw) as plan:
        U = torch.empty((128, 128), dtype=torch.complex128, device="cuda:0")
        plan.propagate_roi(0, plan.info["N"], U)
        ref = plan.metrics(U)
    got = fzp.metrics_noalloc(U, **kw)
    assert got["aperture_count"] == ref["aperture_count"]
    for k in KEYS:
        assert abs(got[k] / ref[k] - 1) < 1e-9, (k, got[k], ref[k])
