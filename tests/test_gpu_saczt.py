"""The SA-CZT form (Sec. 3.6, Fig. 5: exact-radii plate, angular-spectrum
residual on a padded grid, Fresnel chirp and CZT zoom onto the ROI) against
the oracle's FP64 evaluation of the same steps (oracle/saczt.py), through
the C ABI: relative L2 of I <= 1e-4 (FP32 form)."""
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
    from oracle import saczt
    import paper_2609_01978_gb300 as fzp
    return fzp, torch, oracle, saczt


def _plan(fzp, g, exact, x0=None):
    return fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, dx=g.dx, N=g.N, form=fzp.FORM_SACZT,
                    precision=fzp.PREC_FP32, exact_radii=exact, x0=x0)


@pytest.mark.parametrize("exact", [1, 0])
@pytest.mark.parametrize("D,M", [(2e-3, 128), (4e-3, 256)])
def test_saczt_matches_oracle(env, exact, D, M):
    """2 mm (N = 2529, P = 4096) and 4 mm (config 1's plate, N = 5057,
    P = 8192) at f/5, exact and paraxial zone radii."""
    fzp, torch, O, SA = env
    g = O.Geometry(D=D, f=5 * D, lam=LAM, M=M, p=LAM * 5 / 8, kind=O.FZP_EXACT if exact else O.FZP_PARAXIAL)
    Uref = SA.field_saczt(g)
    with _plan(fzp, g, exact) as plan:
        assert plan.info["fft_length"] == SA.pad_size(g.N)
        U, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
    err = rel_l2(I, np.abs(Uref) ** 2)
    print(f"SA-CZT D = {D} m exact = {exact}: rel L2 of I {err:.3e}, of U {rel_l2(U, Uref):.3e}")
    assert err <= 1e-4
    assert rel_l2(U, Uref) <= 1e-3


@pytest.mark.parametrize("M", [64, 128])
def test_saczt_rows_add_and_offaxis(env, M):
    """Row ranges are linear (two ranges accumulate to the whole plate), and an
    off-axis ROI origin matches the oracle's; M = 64 takes the CUDA-core zoom,
    M = 128 the tensor-core one."""
    fzp, torch, O, SA = env
    g = O.Geometry(D=2e-3, f=10e-3, lam=LAM, M=M, p=LAM * 5 / 8, kind=O.FZP_EXACT)
    with _plan(fzp, g, 1) as plan:
        U1, _ = run_plan(fzp, torch, plan, g.M, 0, g.N)
        dev = torch.device("cuda:0")
        acc = torch.zeros((g.M, g.M), dtype=torch.complex128, device=dev)
        a = g.c - 333
        plan.propagate_roi(0, a, acc, accumulate=True)
        plan.propagate_roi(a, g.N, acc, accumulate=True)
        torch.cuda.synchronize()
        assert rel_l2(acc.cpu().numpy(), U1) < 1e-5
    x0 = -(g.M // 2) * g.p + 17.5 * g.p
    g2 = O.Geometry(D=2e-3, f=10e-3, lam=LAM, M=M, p=LAM * 5 / 8, kind=O.FZP_EXACT, x0=x0)
    with _plan(fzp, g2, 1, x0=x0) as plan:
        _, I = run_plan(fzp, torch, plan, g2.M, 0, g2.N)
    assert rel_l2(I, np.abs(SA.field_saczt(g2)) ** 2) <= 1e-4


def test_saczt_mask_and_metrics(env):
    """The exported exact-radii mask equals the oracle's except on samples whose
    zone index lies within 1e-9 of an integer; the plan's metrics read the
    exact plate's Airy focus and binary-FZP efficiency."""
    fzp, torch, O, SA = env
    g = O.Geometry(D=2e-3, f=10e-3, lam=LAM, M=128, p=LAM * 5 / 8, kind=O.FZP_EXACT)
    ref = O.mask_rows(g, 0, g.N)
    with _plan(fzp, g, 1) as plan:
        out = torch.empty((g.N, g.N), dtype=torch.uint8, device="cuda:0")
        plan.aperture_mask(0, g.N, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        U = torch.empty((g.M, g.M), dtype=torch.complex128, device="cuda:0")
        plan.propagate_roi(0, g.N, U)
        m = plan.metrics(U)
    diff = np.argwhere(got != ref)
    d = np.arange(g.N) - g.c
    for j, i in diff:
        r2 = float(d[j] ** 2 + d[i] ** 2) * g.dx ** 2
        n = 2 * r2 / (g.lam * (np.sqrt(g.f ** 2 + r2) + g.f))
        assert abs(n - round(n)) < 1e-9, (j, i, n)
    assert len(diff) <= 8
    airy = O.airy_fwhm_factor() * g.lam * g.f / (2 * g.R)
    assert abs(m["fwhm_x"] / airy - 1) < 1e-2
    assert abs(m["de_lobe"] / (O.airy_encircled(O.AIRY_NULL) * O.binary_fzp_efficiency()) - 1) < 2e-2


def test_saczt_rejects(env):
    fzp, torch, O, SA = env
    base = dict(D=2e-3, f=10e-3, lam=LAM, M=64, pitch=0.4e-6)
    for kw, status in [(dict(form=fzp.FORM_SACZT, precision=fzp.PREC_FP64), fzp.FZP_E_UNSUPPORTED),
                       (dict(form=fzp.FORM_SACZT, precision=fzp.PREC_FP32, levels=4), fzp.FZP_E_UNSUPPORTED),
                       (dict(form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP32, exact_radii=1), fzp.FZP_E_UNSUPPORTED)]:
        with pytest.raises(fzp.FzpError) as e:
            fzp.Plan(**base, **kw)
        assert e.value.status == status, kw


def test_saczt_bench_plate_vs_stored_oracle(env):
    """The SA-CZT bench workload in the bench's launch configuration: the
    8 mm exact-radii plate (N = 10,115, padded grid 16,384^2, ROI 512^2,
    tensor-core zoom) against the oracle's FP64 SA-CZT field of the whole
    plate (tests/golden/saczt_d8mm_field.npy, written by
    tests/golden/make_saczt_oracle.py): relative L2 of I <= 1e-4, FWHM within
    0.01 % and lobe DE within 0.01 percentage points of the oracle's extractor
    on the oracle's field."""
    import json
    import os
    fzp, torch, O, SA = env
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    meta = json.load(open(os.path.join(golden, "saczt_d8mm.json")))
    Uref = np.load(os.path.join(golden, meta["field_file"])).astype(np.complex128)
    mref = meta["metrics_fp64"]
    g = O.Geometry(D=8e-3, f=40e-3, lam=LAM, M=512, p=LAM * 5 / 8, kind=O.FZP_EXACT)
    with _plan(fzp, g, 1) as plan:
        assert plan.info["fft_length"] == meta["geometry"]["P"] == 16384
        U, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
        m = plan.metrics(torch.from_numpy(U).to("cuda:0"))
    err = rel_l2(I, np.abs(Uref) ** 2)
    print(f"SA-CZT 8 mm plate: rel L2 of I {err:.3e}, of U {rel_l2(U, Uref):.3e}, "
          f"FWHM {m['fwhm_x'] / mref['fwhm_x'] - 1:.2e}, DE {m['de_lobe'] - mref['de_lobe']:.2e}")
    assert err <= 1e-4
    assert abs(m["fwhm_x"] / mref["fwhm_x"] - 1) < 1e-4
    assert abs(m["de_lobe"] - mref["de_lobe"]) < 1e-4
