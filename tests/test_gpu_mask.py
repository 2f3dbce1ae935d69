"""Zone-plate mask generators (Fig. 2 Stage 2; Fig. 18 Stage 3 for level maps)
against the oracle, bit for bit: the Bluestein form evaluates every sample;
the dense form exports through the generator its row pass launches -- the
row walker (single-CTA launches), the block-wise generator (2- and 4-CTA
clusters) or the level mode (phase plates with L >= 4) -- and each must equal
floor(fl(s kappa)) odd, s <= s_R (level q = floor(fl(s kappa_L)) mod L)."""
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


def _export(fzp, torch, plan, j0, j1, N):
    out = torch.empty((j1 - j0, N), dtype=torch.uint8, device="cuda:0")
    plan.aperture_mask(j0, j1, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def config1(env):
    fzp, torch, O = env
    g = O.Geometry(D=4e-3, f=20e-3, lam=632.8e-9, M=256, p=0.2e-6)
    return g, O.mask_rows(g, 0, g.N)


@pytest.mark.parametrize("cluster", [1, 2, 4])
def test_dense_export_each_generator(env, config1, cluster):
    """Config 1 (N = 5057) through the walker (1 CTA) and the block-wise
    generator (2 and 4 CTAs): the whole mask, and a ragged range of 37 rows
    about the axis (a partly filled warp)."""
    fzp, torch, O = env
    g, ref = config1
    with fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, form=fzp.FORM_DENSE, precision=fzp.PREC_SPLIT_BF16,
                  cluster=cluster) as plan:
        assert plan.info["cluster"] == cluster and plan.info["N"] == g.N
        got = _export(fzp, torch, plan, 0, g.N, g.N)
        assert np.array_equal(got, ref), (cluster, int(np.sum(got != ref)))
        got = _export(fzp, torch, plan, g.c - 17, g.c + 20, g.N)
        assert np.array_equal(got, ref[g.c - 17:g.c + 20]), cluster


@pytest.mark.parametrize("L,cluster", [(2, 1), (2, 4), (4, 1), (4, 4), (8, 2), (16, 4)])
def test_dense_level_maps(env, L, cluster):
    """Phase plates in the dense form: L = 2 through the signed walker or the
    block-wise generator, L >= 4 through the level mode (every level q read
    back from the generator's level sets), bit for bit on a 200-row band
    through the axis and ragged ranges at both edges (N = 1505 ... 12,031)."""
    fzp, torch, O = env
    lam = 532e-9
    g = O.Geometry(D=1e-3, f=5e-3, lam=lam, M=256, p=lam * 5 / 8, kind=O.FZP_PHASE, levels=L)
    with fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, form=fzp.FORM_DENSE, precision=fzp.PREC_SPLIT_BF16,
                  cluster=cluster, levels=L) as plan:
        assert plan.info["N"] == g.N and plan.info["passes"] == (1 if L == 2 else L // 2)
        for (j0, j1) in [(g.c - 100, g.c + 100), (0, 45), (g.N - 37, g.N)]:
            got = _export(fzp, torch, plan, j0, j1, g.N)
            ref = O.mask_rows(g, j0, j1)
            assert np.array_equal(got, ref), (L, cluster, j0, int(np.sum(got != ref)))


@pytest.mark.parametrize("table", [4, 5])
def test_dense_level_maps_table_grids(env, table):
    """The paper's grids: Table 4 (D = 4 m, L = 4, Nx = 12,030,077, level mode)
    and Table 5 (D = 5 m, L = 2, Nx = 15,037,595, block-wise generator of a
    cluster launch); rows through the axis, at the aperture edge and in
    between.  M = 64 in 2-CTA clusters keeps the kernel matrix at 25-31 GB; the
    generators depend on neither."""
    fzp, torch, O = env
    lam = 532e-9
    D, L = (4.0, 4) if table == 4 else (5.0, 2)
    f = 5 * D
    g = O.Geometry(D=D, f=f, lam=lam, M=64, p=lam * 5 / 8, dx=lam * f / (D / 2) / 16, kind=O.FZP_PHASE, levels=L)
    assert g.N == {4: 12030077, 5: 15037595}[table]
    with fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, dx=g.dx, N=g.N, form=fzp.FORM_DENSE,
                  precision=fzp.PREC_SPLIT_BF16, cluster=2, levels=L) as plan:
        for j0 in [g.c - 1, 3, g.N // 7, g.N - 4]:
            got = _export(fzp, torch, plan, j0, j0 + 3, g.N)
            ref = O.mask_rows(g, j0, j0 + 3)
            assert np.array_equal(got, ref), (table, j0, int(np.sum(got != ref)))


@pytest.mark.parametrize("D", [1.0, 5.0])
def test_dense_walker_export_large_grids(env, D):
    """The row walker of single-CTA launches (the automatic choice for M <= 128)
    far from the axis, where the boundary distances reach a ~ N/2 and its
    approximate square root needs its full correction range: D = 1 m at
    f/# = 5 (N = 1,264,223) and Table 5's grid (N = 15,037,595, L = 2 level
    map), rows through the axis, at mid radius and near the edge."""
    fzp, torch, O = env
    if D == 1.0:
        lam = 632.8e-9
        g = O.Geometry(D=D, f=5 * D, lam=lam, M=64, p=lam * 5 / 8)
        extra = {}
    else:
        lam, f = 532e-9, 25.0
        g = O.Geometry(D=D, f=f, lam=lam, M=64, p=lam * 5 / 8, dx=lam * f / (D / 2) / 16, kind=O.FZP_PHASE,
                       levels=2)
        extra = dict(dx=g.dx, levels=2)
    with fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, N=g.N, form=fzp.FORM_DENSE,
                  precision=fzp.PREC_SPLIT_BF16, cluster=1, **extra) as plan:
        assert plan.info["cluster"] == 1 and plan.info["N"] == g.N
        for j0 in [g.c - 1, g.c // 2, g.N // 50]:
            got = _export(fzp, torch, plan, j0, j0 + 3, g.N)
            ref = O.mask_rows(g, j0, j0 + 3)
            assert np.array_equal(got, ref), (D, j0, int(np.sum(got != ref)))
