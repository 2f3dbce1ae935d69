"""Binary zone-plate mask generators (Fig. 2 Stage 2) against the oracle, bit
for bit: the Bluestein form evaluates every sample, the dense form walks zone
thresholds along each row; both must equal floor(fl(s kappa)) odd, s <= s_R."""
import hashlib

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
    import oracle
    import paper_2609_01978_gb300 as fzp
    return fzp, torch, oracle


def _gpu_mask(fzp, torch, g, form, prec, j0, j1):
    with fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, dx=g.dx, N=g.N, form=form, precision=prec) as plan:
        out = torch.empty((j1 - j0, g.N), dtype=torch.uint8, device="cuda:0")
        plan.aperture_mask(j0, j1, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()


@pytest.mark.parametrize("form,prec", [(1, 1), (2, 2)])
def test_mask_full_config1(env, form, prec):
    fzp, torch, O = env
    g = O.Geometry(D=4e-3, f=20e-3, lam=632.8e-9, M=256, p=0.2e-6)
    ref = O.mask_rows(g, 0, g.N)
    got = _gpu_mask(fzp, torch, g, form, prec, 0, g.N)
    assert hashlib.sha256(got.tobytes()).hexdigest() == hashlib.sha256(ref.tobytes()).hexdigest()


@pytest.mark.parametrize("form,prec", [(1, 1), (2, 2)])
def test_mask_sampled_rows_large_apertures(env, form, prec):
    """D = 0.25 m and D = 1 m (N = 316,057 / 1,264,223): sampled rows, including
    the centre row, the aperture edge rows and random rows."""
    fzp, torch, O = env
    lam = 632.8e-9
    for D in (0.25, 1.0):
        g = O.Geometry(D=D, f=5 * D, lam=lam, M=512, p=lam * 5 / 8)
        rng = np.random.default_rng(int(D * 100))
        starts = [g.c - 2, 0, g.N - 5, int(rng.integers(0, g.N - 5)), int(rng.integers(0, g.N - 5))]
        for j0 in starts:
            ref = O.mask_rows(g, j0, j0 + 4)
            got = _gpu_mask(fzp, torch, g, form, prec, j0, j0 + 4)
            assert np.array_equal(got, ref), (D, j0, int(np.sum(got != ref)))
