"""Edge cases of the propagation through the C ABI, for both forms: empty and
off-aperture row ranges, accumulation over row ranges, row passes split into
many chunks (chunk starts not aligned to 32 rows), and the smallest and
largest ROI sizes (M = 64: single-CTA dense kernel and CUDA-core column pass;
M = 1024: eight kernel tile pairs)."""
import numpy as np
import pytest

from gpu_util import rel_l2, run_plan

pytestmark = pytest.mark.gpu

FORMS = [("dense", 2, 1e-4), ("bluestein", 1, 1e-4), ("bluestein", 0, 1e-6)]


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


def _plan(fzp, g, form, prec, **kw):
    f = fzp.FORM_DENSE if form == "dense" else fzp.FORM_BLUESTEIN
    return fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, dx=g.dx, N=g.N, form=f, precision=prec, **kw)


@pytest.mark.parametrize("form,prec,tol", FORMS)
def test_empty_and_off_aperture_ranges(env, form, prec, tol):
    fzp, torch, O = env
    # a grid 200 samples wider than the aperture: its first rows miss the disc
    g = O.Geometry(D=4e-3, f=20e-3, lam=632.8e-9, M=128, p=0.3e-6, N=5257)
    with _plan(fzp, g, form, prec) as plan:
        Uz, _ = run_plan(fzp, torch, plan, g.M, 100, 100)
        assert np.all(Uz == 0)
        # rows outside the aperture disc: no open sample, zero field
        assert O.mask_rows(g, 0, 3).sum() == 0
        Uo, _ = run_plan(fzp, torch, plan, g.M, 0, 3)
        assert np.all(Uo == 0)
        U1, _ = run_plan(fzp, torch, plan, g.M, g.c, g.c + 1)  # one row
        ref = O.field_czt(g, g.c, g.c + 1)
        assert rel_l2(np.abs(U1) ** 2, np.abs(ref) ** 2) <= tol


@pytest.mark.parametrize("form,prec,tol", FORMS)
def test_many_chunks_and_accumulation(env, form, prec, tol):
    """stripe_rows = 512 splits config 1's 5057 rows into 10 chunks whose starts
    (disc edge c - b plus multiples of 512) are not multiples of 32; three
    accumulated row ranges give the one-pass field."""
    fzp, torch, O = env
    g = O.Geometry(D=4e-3, f=20e-3, lam=632.8e-9, M=256, p=0.2e-6)
    Iref = np.abs(O.field_czt(g)) ** 2
    with _plan(fzp, g, form, prec, stripe_rows=512) as plan:
        assert plan.info["chunk_rows"] == 512
        U, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
        assert rel_l2(I, Iref) <= tol
        dev = torch.device("cuda:0")
        Ua = torch.zeros((g.M, g.M), dtype=torch.complex128, device=dev)
        for (a, b) in [(0, 1777), (1777, 3001), (3001, g.N)]:
            plan.propagate_roi(a, b, Ua, accumulate=True)
        torch.cuda.synchronize()
        assert rel_l2(Ua.cpu().numpy(), U) <= (1e-12 if prec == 0 else 1e-5)


@pytest.mark.parametrize("M", [64, 1024])
def test_roi_extremes_dense(env, M):
    fzp, torch, O = env
    g = O.Geometry(D=2e-3, f=10e-3, lam=632.8e-9, M=M, p=632.8e-9 * 5 / 8 * (512 / M))
    Iref = np.abs(O.field_czt(g)) ** 2
    with _plan(fzp, g, "dense", 2) as plan:
        assert plan.info["cluster"] == (1 if M == 64 else 4)
        _, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
        assert rel_l2(I, Iref) <= 1e-4
