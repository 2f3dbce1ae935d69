"""The library's host logic on the CPU (no GPU): the plan description that
fzp_plan_query derives (grids of Fig. 2 / Fig. 18 Stage 1, the Eq. 3 zone
count, chunking) against the oracle's geometry and the Nx the paper prints
for Tables 1-5, and the zone-threshold table fzp_zone_thresholds exports
(the table every device mask generator reads) against its definition
S_m = min{s : floor(fl(s kappa_L)) >= m} evaluated in IEEE doubles."""
import json
import math
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")
LAM = 632.8e-9


@pytest.fixture(scope="module")
def fzp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2609_01978_gb300 as m
    return m


CASES = [
    dict(D=4e-3, f=20e-3, M=256, p=0.2e-6),                       # config 1
    dict(D=0.25, f=1.25, M=512, p=LAM * 5 / 8),                   # config 2
    dict(D=1.0, f=5.0, M=512, p=LAM * 5 / 8),                     # config 3, D = 1 m
    dict(D=5.0, f=25.0, M=512, p=LAM * 5 / 8),                    # config 3, D = 5 m
    dict(D=2e-3, f=10e-3, M=128, p=LAM * 5 / 8, levels=4),        # phase plates, default dx
    dict(D=2e-3, f=10e-3, M=128, p=LAM * 5 / 8, levels=16),
    dict(D=1e-3, f=5e-3, M=64, p=LAM * 5 / 8, centre_open=1),     # positive-centred
]


@pytest.mark.parametrize("case", CASES, ids=[str(i) for i in range(len(CASES))])
def test_query_matches_oracle_geometry(fzp, oracle_mod, case):
    O = oracle_mod
    levels = case.get("levels", 0)
    kind = O.FZP_PHASE if levels else (O.FZP_POSITIVE if case.get("centre_open") else O.FZP_PARAXIAL)
    g = O.Geometry(D=case["D"], f=case["f"], lam=LAM, M=case["M"], p=case["p"], kind=kind, levels=levels)
    q = fzp.plan_query(D=case["D"], f=case["f"], lam=LAM, M=case["M"], pitch=case["p"], levels=levels,
                       centre_open=case.get("centre_open", 0), form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP32)
    assert q["N"] == g.N and q["c"] == g.c
    assert q["dx"] == pytest.approx(g.dx, rel=1e-15) and q["R"] == pytest.approx(g.R, rel=1e-15)
    assert q["x0"] == pytest.approx(g.x0, rel=1e-15)
    assert q["total_zones"] == g.total_zones()
    assert q["levels"] == (levels if levels >= 2 else 0) and q["centre_open"] == case.get("centre_open", 0)
    # Bluestein length L = 2^ceil(log2(N + M - 1)) (Sec. 2.6)
    assert q["fft_length"] == 1 << math.ceil(math.log2(g.N + g.M - 1))
    # the threshold count: the last zone step inside the disc, plus two
    dx2, R2 = q["dx"] ** 2, q["R"] ** 2
    sR = int(R2 // dx2)
    while float(sR + 1) * dx2 <= R2:
        sR += 1
    while float(sR) * dx2 > R2:
        sR -= 1
    rate = q["kappa"] * (0.5 * levels if levels >= 2 else 1.0)
    assert q["n_thresholds"] == math.floor(float(sR) * rate) + 2


def test_query_tables_1_to_5_nx(fzp):
    """Nx of Tables 1-5 through the library's own grid rule (dx given as
    Lambda_edge / k, forced odd), and the dense form's pass count per L."""
    gold = json.load(open(os.path.join(GOLDEN, "v8_grid_tables.json")))
    lam = gold["lambda"]
    for row in gold["rows"]:
        dx = lam * row["f"] / (row["D"] / 2) / row["k"]
        q = fzp.plan_query(D=row["D"], f=row["f"], lam=lam, M=512, pitch=lam * 5 / 8, dx=dx, levels=row["L"],
                           form=fzp.FORM_DENSE, precision=fzp.PREC_SPLIT_BF16)
        assert q["N"] == row["Nx"], row
        assert q["passes"] == (1 if row["L"] == 2 else row["L"] // 2)
        assert q["promote"] == 128 and q["form"] == fzp.FORM_DENSE


def test_query_chunking_and_rejections(fzp):
    """Chunks: as many rows as an 8 GiB row intermediate holds (M = 512 in FP32:
    2^21 rows), at most the grid rounded up to 256; a requested stripe height
    is kept.  Invalid parameters are rejected as fzp_plan rejects them."""
    kw = dict(D=5.0, f=25.0, lam=LAM, M=512, pitch=LAM * 5 / 8)
    q = fzp.plan_query(form=fzp.FORM_DENSE, precision=fzp.PREC_SPLIT_BF16, **kw)
    assert q["chunk_rows"] == 1 << 21
    q = fzp.plan_query(form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP64, **kw)
    assert q["chunk_rows"] == 1 << 20  # FP64 intermediate: half the rows
    q = fzp.plan_query(form=fzp.FORM_DENSE, precision=fzp.PREC_SPLIT_BF16, stripe_rows=4096, **kw)
    assert q["chunk_rows"] == 4096
    q = fzp.plan_query(D=4e-3, f=20e-3, lam=LAM, M=256, pitch=0.2e-6)
    assert q["chunk_rows"] == 5120  # N = 5057 rounded up to 256
    q = fzp.plan_query(precision=fzp.PREC_AUTO_1E4, **kw)
    assert q["form"] == fzp.FORM_AUTO and q["fft_length"] == 0
    for bad in (dict(levels=65), dict(centre_open=1, levels=4), dict(N=1000), dict(M=100)):
        with pytest.raises(fzp.FzpError) as e:
            fzp.plan_query(**dict(kw, **bad))
        assert e.value.status == fzp.FZP_E_INVALID
    with pytest.raises(fzp.FzpError) as e:
        fzp.plan_query(form=fzp.FORM_DENSE, precision=fzp.PREC_SPLIT_BF16, levels=3, **kw)
    assert e.value.status == fzp.FZP_E_UNSUPPORTED


@pytest.mark.parametrize("case", [
    dict(D=4e-3, f=20e-3, levels=0),                  # config 1, zone rate kappa
    dict(D=2e-3, f=10e-3, levels=4),                  # kappa_L = kappa L / 2
    dict(D=5.0, f=25.0, levels=2, table5=True),       # Table 5 grid, 470k steps
])
def test_zone_thresholds_definition(fzp, case):
    lam = 532e-9 if case.get("table5") else LAM
    kw = dict(D=case["D"], f=case["f"], lam=lam, M=256, pitch=lam * 5 / 8, levels=case["levels"])
    if case.get("table5"):
        kw["dx"] = lam * case["f"] / (case["D"] / 2) / 16
    q = fzp.plan_query(**kw)
    S = fzp.zone_thresholds(**kw)
    assert len(S) == q["n_thresholds"]
    rate = q["kappa"] * (0.5 * case["levels"] if case["levels"] >= 2 else 1.0)
    m = np.arange(1, len(S) + 1)
    # numpy converts each s to double and rounds one product, as fl(s kappa) does
    assert np.all(np.floor(S.astype(np.float64) * rate) >= m)
    assert np.all(np.floor((S - 1).astype(np.float64) * rate) < m)
    assert np.all(np.diff(S) > 0)
    if case.get("table5"):
        assert q["N"] == 15037595 and len(S) > 400_000


def test_threshold_export_buffer_rules(fzp):
    import ctypes
    L = fzp.lib()
    p = fzp._params(D=4e-3, f=20e-3, lam=LAM, M=256, pitch=0.2e-6)
    n = ctypes.c_int64(-1)
    assert L.fzp_zone_thresholds(ctypes.byref(p), None, 0, ctypes.byref(n)) == fzp.FZP_OK and n.value > 0
    assert L.fzp_zone_thresholds(ctypes.byref(p), None, 4, ctypes.byref(n)) == fzp.FZP_E_INVALID
    assert L.fzp_zone_thresholds(ctypes.byref(p), None, 0, None) == fzp.FZP_E_INVALID
    buf = (ctypes.c_int64 * 3)()
    assert L.fzp_zone_thresholds(ctypes.byref(p), buf, 3, ctypes.byref(n)) == fzp.FZP_OK
    full = fzp.zone_thresholds(D=4e-3, f=20e-3, lam=LAM, M=256, pitch=0.2e-6)
    assert list(buf) == list(full[:3]) and n.value == len(full)


def test_query_size_limits(fzp):
    """The zone rule's s_R < 2^46 and the Bluestein FFT length <= 2^24: a
    5 m plate sampled to N = 16,700,001 passes, N = 16,800,001 does not (s_R
    above 2^46); N = 16,777,001 (N + M - 1 above 2^24, s_R still below 2^46)
    is refused to the Bluestein form but not to the dense one."""
    lam, D, f = 532e-9, 5.0, 25.0
    kw = dict(D=D, f=f, lam=lam, M=512, pitch=lam * 5 / 8)
    ok = fzp.plan_query(dx=D / 16_700_001, form=fzp.FORM_DENSE, precision=fzp.PREC_SPLIT_BF16, **kw)
    assert ok["N"] == 16_700_001
    with pytest.raises(fzp.FzpError) as e:
        fzp.plan_query(dx=D / 16_800_001, form=fzp.FORM_DENSE, precision=fzp.PREC_SPLIT_BF16, **kw)
    assert e.value.status == fzp.FZP_E_UNSUPPORTED and "zone rule" in str(e.value)
    big = fzp.plan_query(dx=D / 16_777_001, form=fzp.FORM_DENSE, precision=fzp.PREC_SPLIT_BF16, **kw)
    assert big["N"] == 16_777_001
    with pytest.raises(fzp.FzpError) as e:
        fzp.plan_query(dx=D / 16_777_001, form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP32, **kw)
    assert e.value.status == fzp.FZP_E_UNSUPPORTED and "FFT length" in str(e.value)


def test_query_random_geometries(fzp, oracle_mod):
    """200 random plates (D from 1 mm to 5 m, f/# from 2 to 20, 450-700 nm,
    levels 0-16, optional explicit dx at 1-8x the Nyquist spacing): the
    library's grid and zone count equal the oracle's."""
    O = oracle_mod
    rng = np.random.default_rng(2026)
    for _ in range(200):
        D = float(10 ** rng.uniform(-3, math.log10(5.0)))
        fnum = float(rng.uniform(2, 20))
        lam = float(rng.uniform(450e-9, 700e-9))
        L = int(rng.choice([0, 0, 2, 3, 4, 8, 16]))
        f = fnum * D
        dx = 0.0
        if rng.uniform() < 0.5:
            dx = lam * f / (2 * D) / float(rng.uniform(1.0, 8.0))
        N_est = D / (dx if dx else lam * f / (2 * D * max(L, 2)))
        if N_est > 3e6:
            continue  # keep the oracle's own grid arithmetic quick
        kind = O.FZP_PHASE if L >= 2 else O.FZP_PARAXIAL
        g = O.Geometry(D=D, f=f, lam=lam, M=64, p=lam * fnum / 8, dx=dx or None, kind=kind, levels=L)
        q = fzp.plan_query(D=D, f=f, lam=lam, M=64, pitch=lam * fnum / 8, dx=dx, levels=L)
        assert q["N"] == g.N and q["c"] == g.c, (D, fnum, lam, L, dx)
        assert q["dx"] == pytest.approx(g.dx, rel=1e-15) and q["R"] == pytest.approx(g.R, rel=1e-15)
        assert q["total_zones"] == g.total_zones()
