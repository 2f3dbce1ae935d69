"""The dense tensor-core form for deformed membranes (complex transmission
T e^{i phi}, phi = (4 pi / lambda) w with the wrinkle, taper and crease
ridges of the membrane model): two membrane passes with the split masks
T cos(phi) and T sin(phi), against the oracle's O3 evaluation of the same
deformed aperture (relative L2 of I <= 1e-4), through the C ABI."""
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


def _scaled(m, D):
    """A config-4 membrane draw moved onto a plate of diameter D (lengths of the
    wrinkle and the ridges scaled with D / D_draw, heights kept)."""
    k = D / m.D
    ridges = [(px * k, py * k, al, h, w * k) for (px, py, al, h, w) in m.ridges]
    return dict(amp=m.amp, period=m.period * k, theta=m.theta, taper=m.taper, ridges=ridges)


@pytest.mark.parametrize("k", range(4))
@pytest.mark.parametrize("cluster", [0, 1])
def test_dense_membrane_small_plates(env, k, cluster):
    """Four seeded config-4 draws on 2-5 mm plates (their wavelengths, ROI
    256^2 at lambda f/# / 8), the plan's own cluster (2 CTAs) and the
    single-CTA kernel."""
    fzp, torch, O = env
    import fzp_inputs
    m = fzp_inputs.batch_draws(8, seed=0)[k]
    D = (2e-3, 3e-3, 4e-3, 5e-3)[k]
    d = _scaled(m, D)
    g = O.Geometry(D=D, f=5 * D, lam=m.lam, M=256, p=m.lam * 5 / 8, deform=O.Deform(**d))
    Iref = np.abs(O.field_czt(g)) ** 2
    with fzp.Plan(D=D, f=5 * D, lam=m.lam, M=256, pitch=m.lam * 5 / 8, form=fzp.FORM_DENSE,
                  precision=fzp.PREC_SPLIT_BF16, cluster=cluster, deform=fzp.make_deform(**d)) as plan:
        assert plan.info["passes"] == 2
        _, I = run_plan(fzp, torch, plan, 256, 0, g.N)
    err = rel_l2(I, Iref)
    print(f"dense membrane draw {k} D = {D} m cluster {cluster}: rel L2 of I {err:.3e}")
    assert err <= 1e-4


@pytest.mark.parametrize("M,cluster", [(512, 0), (128, 4)])
def test_dense_membrane_roi_and_clusters(env, M, cluster):
    """ROI 512^2 (4-CTA clusters) and 128^2 padded into a 4-CTA cluster, with a
    strong wrinkle (a quarter wave), three ridges and the positive-centred
    plate for the latter."""
    fzp, torch, O = env
    lam = 550e-9
    D = 4e-3
    d = dict(amp=lam / 4, period=3.1e-4, theta=2.2, taper=0.7,
             ridges=[(3e-4, -2e-4, 0.4, lam / 8, 2e-4), (-5e-4, 1e-4, 1.9, lam / 9, 3e-4),
                     (1e-4, 6e-4, 2.8, lam / 10, 1.5e-4)])
    centre_open = 1 if M == 128 else 0
    g = O.Geometry(D=D, f=5 * D, lam=lam, M=M, p=lam * 5 / 8, deform=O.Deform(**d),
                   kind=O.FZP_POSITIVE if centre_open else O.FZP_PARAXIAL)
    Iref = np.abs(O.field_czt(g)) ** 2
    with fzp.Plan(D=D, f=5 * D, lam=lam, M=M, pitch=lam * 5 / 8, form=fzp.FORM_DENSE,
                  precision=fzp.PREC_SPLIT_BF16, cluster=cluster, centre_open=centre_open,
                  deform=fzp.make_deform(**d)) as plan:
        _, I = run_plan(fzp, torch, plan, M, 0, g.N)
    err = rel_l2(I, Iref)
    print(f"dense membrane M = {M} cluster {cluster}: rel L2 of I {err:.3e}")
    assert err <= 1e-4


def test_dense_membrane_config4_stripes(env):
    """A seeded config-4 membrane at its own size (D = 0.3 m class, N ~ 5e5)
    on two 256-row stripes (through the centre and at v = -0.6 R), dense form
    and FP32 Bluestein form against the oracle's same rows."""
    fzp, torch, O = env
    import fzp_inputs
    draws = fzp_inputs.batch_draws(256, seed=0)
    m = max(draws[:16], key=lambda x: x.D)
    d = dict(amp=m.amp, period=m.period, theta=m.theta, taper=m.taper, ridges=m.ridges)
    g = O.Geometry(D=m.D, f=5 * m.D, lam=m.lam, M=256, p=m.lam * 5 / 8, deform=O.Deform(**d))
    rows = [g.c - 128, g.c - int(0.6 * g.R / g.dx)]
    refs = [np.abs(O.field_czt(g, j0, j0 + 256)) ** 2 for j0 in rows]
    for form, prec in [(fzp.FORM_DENSE, fzp.PREC_SPLIT_BF16), (fzp.FORM_BLUESTEIN, fzp.PREC_FP32)]:
        with fzp.Plan(D=m.D, f=5 * m.D, lam=m.lam, M=256, pitch=m.lam * 5 / 8, form=form, precision=prec,
                      deform=fzp.make_deform(**d)) as plan:
            assert plan.info["N"] == g.N
            for j0, Iref in zip(rows, refs):
                _, I = run_plan(fzp, torch, plan, 256, j0, j0 + 256)
                err = rel_l2(I, Iref)
                print(f"config-4 membrane D = {m.D:.4f} m form {form} rows {j0}: rel L2 of I {err:.3e}")
                assert err <= 1e-4, (form, j0, err)


def test_autotune_on_a_large_membrane(env):
    """A deformed 0.15 m plate: the autotuner times the dense membrane passes
    (1-, 2- and 4-CTA clusters) and the FP32 Bluestein form (partitioned
    convolution) on its probe stripe and keeps the faster -- the two are
    within about 10 % of each other here (at D = 0.05 m, 184 against 194
    Gsamples/s) -- and the tuned plan matches the oracle on a stripe."""
    fzp, torch, O = env
    import fzp_inputs
    m = fzp_inputs.batch_draws(8, seed=0)[0]
    d = _scaled(m, 0.15)
    with fzp.Plan(D=0.15, f=0.75, lam=m.lam, M=256, pitch=m.lam * 5 / 8, precision=fzp.PREC_AUTO_1E4,
                  deform=fzp.make_deform(**d)) as plan:
        info = plan.info
        assert (info["form"], info["precision"]) in ((fzp.FORM_DENSE, fzp.PREC_SPLIT_BF16),
                                                     (fzp.FORM_BLUESTEIN, fzp.PREC_FP32)), info
        if info["form"] == fzp.FORM_BLUESTEIN:
            assert info["conv"] == 2
        g = O.Geometry(D=0.15, f=0.75, lam=m.lam, M=256, p=m.lam * 5 / 8, deform=O.Deform(**d))
        j0 = g.c + 300
        _, I = run_plan(fzp, torch, plan, 256, j0, j0 + 256)
    assert rel_l2(I, np.abs(O.field_czt(g, j0, j0 + 256)) ** 2) <= 1e-4


def test_dense_membrane_rejects_phase_plates(env):
    fzp, torch, O = env
    with pytest.raises(fzp.FzpError) as e:
        fzp.Plan(D=2e-3, f=10e-3, lam=550e-9, M=128, pitch=0.4e-6, form=fzp.FORM_DENSE,
                 precision=fzp.PREC_SPLIT_BF16, levels=4, deform=fzp.make_deform(amp=1e-7))
    assert e.value.status == fzp.FZP_E_UNSUPPORTED
