"""Form (a) with the partitioned row convolution (fzp_params.conv = 2, the FP32
default): each row's chirp convolution (Sec. 2.6) summed over blocks of S
columns, every block a 4096-point product with the precomputed spectrum of its
chirp piece, one inverse transform per row.  Against the CPU FP64 oracle (O3)
at FP32's tolerance, relative L2 of I <= 1e-4: block sizes at both ends of the
M range (S = 3840 at M = 64, 3072 at M = 1024), an aperture narrower than one
block, rows whose disc chord is shorter than a block, blocks that straddle the
chord ends, a phase plate and an off-axis ROI; and the two convolutions of the
form against each other on the same rows."""
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


def _plan(fzp, g, conv=2, **kw):
    return fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, dx=g.dx, N=g.N, form=fzp.FORM_BLUESTEIN,
                    precision=fzp.PREC_FP32, conv=conv, **kw)


@pytest.mark.parametrize("M,S", [(64, 3840), (1024, 3072)])
def test_block_size_ends_of_the_roi_range(env, M, S):
    """D = 4 mm at f/5 (N = 5057): two blocks of 3840 columns at M = 64, two of
    3072 at M = 1024 (S + M - 1 <= 4096 at both ends)."""
    fzp, torch, O = env
    g = O.Geometry(D=4e-3, f=20e-3, lam=LAM, M=M, p=0.2e-6 * 256 / M)
    with _plan(fzp, g) as plan:
        assert plan.info["conv"] == 2 and plan.info["fft_inner"] == 4096
        U, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
    Uref = O.field_czt(g)
    err = rel_l2(I, np.abs(Uref) ** 2)
    print(f"partitioned M = {M} (S = {S}): rel L2 of I {err:.3e}")
    assert err <= 1e-4
    assert rel_l2(U, Uref) <= 1e-3


def test_aperture_narrower_than_one_block(env):
    """D = 1 mm at f/5: N = 1265 < S, one block per row."""
    fzp, torch, O = env
    g = O.Geometry(D=1e-3, f=5e-3, lam=LAM, M=128, p=LAM * 5 / 8)
    assert g.N < 3840
    with _plan(fzp, g) as plan:
        _, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
    assert rel_l2(I, np.abs(O.field_czt(g)) ** 2) <= 1e-4


def test_rim_rows_and_straddling_blocks(env):
    """Config 2's plate (N = 316,057, 89 blocks of 3584): the first 48 rows of
    the grid (the disc's top rows: chords far shorter than a block), and 64
    rows at v = -R/3, whose chord ends fall inside blocks."""
    fzp, torch, O = env
    g = O.Geometry(D=0.25, f=1.25, lam=LAM, M=512, p=LAM * 5 / 8)
    with _plan(fzp, g) as plan:
        for j0, n in [(0, 48), (g.c - g.N // 6, 64)]:
            _, I = run_plan(fzp, torch, plan, g.M, j0, j0 + n)
            Iref = np.abs(O.field_czt(g, j0, j0 + n)) ** 2
            err = rel_l2(I, Iref)
            print(f"rows [{j0}, {j0 + n}): rel L2 of I {err:.3e}")
            assert err <= 1e-4, (j0, err)


def test_phase_plate_and_offaxis_roi(env):
    """An L = 4 phase plate (D = 2 mm, f/5), and a binary plate with its ROI
    shifted off axis by 100.5 pitches on both axes."""
    fzp, torch, O = env
    g = O.Geometry(D=2e-3, f=10e-3, lam=LAM, M=128, p=LAM * 5 / 8, kind=O.FZP_PHASE, levels=4)
    with _plan(fzp, g, levels=4) as plan:
        _, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
    assert rel_l2(I, np.abs(O.field_czt(g)) ** 2) <= 1e-4
    p = 0.2e-6
    x0 = -128 * p + 100.5 * p
    g = O.Geometry(D=4e-3, f=20e-3, lam=LAM, M=256, p=p, x0=x0)
    with _plan(fzp, g, x0=x0) as plan:
        _, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
    assert rel_l2(I, np.abs(O.field_czt(g)) ** 2) <= 1e-4


def test_partitioned_equals_single(env):
    """Both convolutions of the FP32 form on config 1's whole aperture and on
    256 rows through the centre of the 1 m plate agree far inside the form's
    tolerance."""
    fzp, torch, O = env
    g1 = O.Geometry(D=4e-3, f=20e-3, lam=LAM, M=256, p=0.2e-6)
    g2 = O.Geometry(D=1.0, f=5.0, lam=LAM, M=512, p=LAM * 5 / 8)
    for g, a, b in [(g1, 0, g1.N), (g2, g2.c - 128, g2.c + 128)]:
        out = {}
        for conv in (1, 2):
            with _plan(fzp, g, conv=conv) as plan:
                U, _ = run_plan(fzp, torch, plan, g.M, a, b)
            out[conv] = U
        err = rel_l2(out[2], out[1])
        print(f"N = {g.N}: single vs partitioned, rel L2 of U {err:.3e}")
        assert err <= 2e-5


def test_grid_narrower_than_the_disc(env):
    """N = 4801 samples for a plate that needs 5057 (config 1's geometry): the
    grid cuts the disc, so row chords are clipped to [0, N) on both sides."""
    fzp, torch, O = env
    g = O.Geometry(D=4e-3, f=20e-3, lam=LAM, M=256, p=0.2e-6, N=4801)
    assert g.R / g.dx > g.c  # the disc reaches past the grid's edges
    with _plan(fzp, g) as plan:
        _, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
    assert rel_l2(I, np.abs(O.field_czt(g)) ** 2) <= 1e-4


@pytest.mark.parametrize("L,D,rows", [(3, 2e-3, None), (5, 1e-3, None), (16, 4e-3, 96)])
def test_phase_plates_any_level_count(env, L, D, rows):
    """Phase plates on the partitioned form's zone-step path (the dense form
    takes even L only): L = 3 and 5 whole, L = 16 on rows at v = R/3 of a
    plate of N = 40,457 (level steps four samples wide at the rim, the
    grid of Fig. 18 Stage 1)."""
    fzp, torch, O = env
    g = O.Geometry(D=D, f=5 * D, lam=LAM, M=64 if rows is None else 128, p=LAM * 5 / 8, kind=O.FZP_PHASE,
                   levels=L)
    a, b = (0, g.N) if rows is None else (g.c + int(g.R / g.dx / 3), g.c + int(g.R / g.dx / 3) + rows)
    with _plan(fzp, g, levels=L) as plan:
        _, I = run_plan(fzp, torch, plan, g.M, a, b)
    err = rel_l2(I, np.abs(O.field_czt(g, a, b)) ** 2)
    print(f"partitioned phase plate L = {L}, N = {g.N}, rows [{a}, {b}): rel L2 of I {err:.3e}")
    assert err <= 1e-4
