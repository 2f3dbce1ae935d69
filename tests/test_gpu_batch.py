"""Batched apertures (uneven D, wavelength, deformation, form) replayed as one
CUDA graph, and the autotuner that picks the form per (N, M)."""
import numpy as np
import pytest

from gpu_util import rel_l2, run_plan

pytestmark = pytest.mark.gpu


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


def _problems(fzp):
    lam1, lam2, lam3 = 632.8e-9, 450e-9, 550e-9
    d = dict(amp=lam3 / 4, period=2.1e-4, theta=0.6, taper=0.3,
             ridges=[(5e-5, -1e-4, 0.4, lam3 / 8, 8e-5), (-2e-4, 3e-5, 2.2, lam3 / 10, 1.2e-4)])
    return [
        dict(D=4e-3, f=20e-3, lam=lam1, M=256, pitch=0.2e-6, form=fzp.FORM_DENSE, precision=fzp.PREC_SPLIT_BF16),
        dict(D=5e-3, f=25e-3, lam=lam2, M=128, pitch=lam2 * 5 / 8, form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP32),
        dict(D=3e-3, f=15e-3, lam=lam3, M=128, pitch=lam3 * 5 / 8, precision=fzp.PREC_AUTO_1E4,
             deform=fzp.make_deform(**d), _deform_kw=d),
        dict(D=2e-3, f=10e-3, lam=lam1, M=64, pitch=lam1 * 5 / 8, form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP64),
    ]


def test_batch_graph_matches_single_plans_and_oracle(env):
    fzp, torch, O = env
    probs = _problems(fzp)
    b = fzp.Batch([{k: v for k, v in p.items() if not k.startswith("_")} for p in probs])
    dev = torch.device("cuda:0")
    fields = [torch.empty((p["M"], p["M"]), dtype=torch.complex128, device=dev) for p in probs]
    b.propagate(fields)
    torch.cuda.synchronize()
    first = [f.cpu().numpy() for f in fields]
    for f in fields:
        f.zero_()
    b.propagate(fields)  # graph replay
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        again = fields[i].cpu().numpy()
        assert rel_l2(again, first[i]) < 1e-12, i
        info = b.info(i)
        kw = {k: v for k, v in p.items() if not k.startswith("_") and k not in ("form", "precision")}
        with fzp.Plan(form=info["form"], precision=info["precision"], promote=info["promote"], **kw) as plan:
            U, _ = run_plan(fzp, torch, plan, p["M"], 0, info["N"])
        assert rel_l2(first[i], U) < 1e-6, i
        g = O.Geometry(D=p["D"], f=p["f"], lam=p["lam"], M=p["M"], p=p["pitch"],
                       deform=O.Deform(**p["_deform_kw"]) if "_deform_kw" in p else None)
        Iref = np.abs(O.field_czt(g)) ** 2
        tol = 1e-6 if info["precision"] == fzp.PREC_FP64 else 1e-4
        assert rel_l2(np.abs(first[i]) ** 2, Iref) <= tol, (i, info["form"], info["precision"])
    # deformed binary plate: both forms are candidates; the autotuner keeps the faster
    assert b.info(2)["form"] in (fzp.FORM_BLUESTEIN, fzp.FORM_DENSE)
    m = b.metrics(0, fields[0])
    assert m["aperture_count"] > 0
    b.close()


def test_autotune_picks_dense_for_large_flat_aperture(env):
    """At D = 0.25 m the split-BF16 dense form is faster than the FP32
    Bluestein form (partitioned convolution: about 1.5x) on the probe stripe."""
    fzp, torch, O = env
    lam = 632.8e-9
    with fzp.Plan(D=0.25, f=1.25, lam=lam, M=512, pitch=lam * 5 / 8, precision=fzp.PREC_AUTO_1E4) as plan:
        info = plan.info
        assert info["form"] == fzp.FORM_DENSE and info["precision"] == fzp.PREC_SPLIT_BF16
        assert info["promote"] in (128, 256)
        g = O.Geometry(D=0.25, f=1.25, lam=lam, M=512, p=lam * 5 / 8)
        j0 = g.c + 777
        _, I = run_plan(fzp, torch, plan, 512, j0, j0 + 512)
    assert rel_l2(I, np.abs(O.field_czt(g, j0, j0 + 512)) ** 2) <= 1e-4


def test_autotune_picks_partitioned_fp32_for_sixteen_levels(env):
    """A 16-level phase plate (D = 0.02 m at f/5 on Fig. 18 Stage 1's grid,
    N = 202,277): the dense form takes L/2 = 8 signed-mask passes, the
    partitioned FP32 Bluestein form one pass whatever L, so the autotuner,
    which times both on its probe stripe, keeps the FP32 form; the tuned plan
    matches the oracle on 64 rows at v = R/3."""
    fzp, torch, O = env
    lam = 632.8e-9
    with fzp.Plan(D=0.02, f=0.1, lam=lam, M=256, pitch=lam * 5 / 8, levels=16,
                  precision=fzp.PREC_AUTO_1E4) as plan:
        info = plan.info
        assert info["form"] == fzp.FORM_BLUESTEIN and info["precision"] == fzp.PREC_FP32
        assert info["conv"] == 2
        g = O.Geometry(D=0.02, f=0.1, lam=lam, M=256, p=lam * 5 / 8, kind=O.FZP_PHASE, levels=16)
        assert info["N"] == g.N
        j0 = g.c + int(g.R / g.dx / 3)
        _, I = run_plan(fzp, torch, plan, 256, j0, j0 + 64)
    assert rel_l2(I, np.abs(O.field_czt(g, j0, j0 + 64)) ** 2) <= 1e-4
