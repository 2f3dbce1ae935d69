"""Run outputs of the engine (Fig. 18, RETURN: result, text report, JSON
sidecar in a run folder) through fzp_report_write: the stored intensity
against the oracle's field, the sidecar's metrics against the oracle's
extractor, and its analytic references against the oracle's closed forms."""
import json
import os

import numpy as np
import pytest

from gpu_util import rel_l2

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


CASES = [("binary-dense", 0, 2, 2), ("phase4-fp32", 4, 1, 1)]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_report_files(env, tmp_path, case):
    fzp, torch, O = env
    name, levels, form, prec = case
    kw = dict(D=4e-3, f=20e-3, lam=632.8e-9, M=256, p=0.2e-6)
    g = O.Geometry(kind=O.FZP_PHASE, levels=levels, **kw) if levels else O.Geometry(**kw)
    Uref = O.field_czt(g)
    mref = O.metrics(g, Uref)
    with fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, dx=g.dx, N=g.N, form=form, precision=prec,
                  levels=levels) as plan:
        U = torch.empty((g.M, g.M), dtype=torch.complex128, device="cuda:0")
        plan.propagate_roi(0, g.N, U)
        m = plan.report(U, str(tmp_path), name, t_propagate_s=0.5)
    I = np.load(tmp_path / f"result_{name}.npy")
    assert I.shape == (g.M, g.M) and I.dtype == np.float64
    assert rel_l2(I, np.abs(Uref) ** 2) <= 1e-4
    side = json.load(open(tmp_path / f"result_{name}.json"))
    assert side["result"] == f"result_{name}.npy" and side["config"]["N"] == g.N
    assert side["metrics"]["fwhm_x"] == m["fwhm_x"]
    assert abs(side["metrics"]["fwhm_x"] / mref["fwhm_x"] - 1) < 1e-4
    assert abs(side["metrics"]["de_lobe"] - mref["de_lobe"]) < 1e-4
    assert side["metrics"]["aperture_count"] == O.count_aperture(g)
    ref = side["references"]
    assert abs(ref["fwhm_airy"] / (O.airy_fwhm_factor() * g.lam * g.f / (2 * g.R)) - 1) < 1e-6
    eta = O.phase_fzp_efficiency(levels) if levels else O.binary_fzp_efficiency()
    assert abs(ref["de_lobe_ladder"] / (O.airy_encircled(O.AIRY_NULL) * eta) - 1) < 1e-6
    assert abs(ref["mtf_half_cut_clear_pupil"] - O.circ_mtf(0.5)) < 1e-6
    assert abs(side["timing"]["gsamples_per_s"] - g.N ** 2 / 0.5 / 1e9) < 1e-6 * side["timing"]["gsamples_per_s"]
    txt = open(tmp_path / f"report_{name}.txt").read()
    assert "FWHM x" in txt and "DE lobe" in txt and "Strehl" in txt and str(g.N) in txt


def test_report_rejects_bad_tag(env, tmp_path):
    fzp, torch, O = env
    with fzp.Plan(D=1e-3, f=5e-3, lam=632.8e-9, M=64, pitch=0.4e-6, precision=fzp.PREC_FP32) as plan:
        U = torch.zeros((64, 64), dtype=torch.complex128, device="cuda:0")
        for tag in ("", "../x", "a b"):
            with pytest.raises(fzp.FzpError) as e:
                plan.report(U, str(tmp_path), tag)
            assert e.value.status == fzp.FZP_E_INVALID
        with pytest.raises(fzp.FzpError) as e:
            plan.report(U, os.path.join(str(tmp_path), "missing_dir"), "t")
        assert e.value.status == fzp.FZP_E_INVALID
