"""The benchmark's contract pieces that run without a GPU: the reference arm
(the oracle on the host cores) prints one JSON line with the required keys and
the same workload description as the GPU arm, and the helpers that the GPU arm
uses for its roofline (flop model, captured traffic keyed to the sources)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "fzp-d0.05m", "--steps", "1", "--warmup", "0", "--ref-rows", "4"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == bench.UNIT
    assert d["metric"] == bench.METRIC and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"] == "fzp-d0.05m" and d["config"]["N"] == 63213
    assert d["config"]["rows_per_step"] == 4


def test_config_is_shared_and_names_the_sample():
    class A:
        workload, form, rows = "fzp-d0.25m", "dense", 0
    c = bench._config(A, bench.WORKLOADS["fzp-d0.25m"], 316057)
    assert c["samples_per_step"] == 316057 ** 2 and "rows_timed" not in c
    A.rows = 4096
    c = bench._config(A, bench.WORKLOADS["fzp-d0.25m"], 316057)
    assert c["samples_per_step"] == 4096 * 316057 and "4096" in c["rows_timed"]
    A.workload = "fzp-t5"
    c = bench._config(A, bench.WORKLOADS["fzp-t5"], 15037595)
    assert c["levels"] == 2 and abs(c["dx_m"] - 532e-9 * 25 / 2.5 / 16) < 1e-18


def test_bluestein_flop_model_and_traffic_keying():
    info = {"fft_length": 1 << 19, "fft_inner": 4096}
    assert bench.bluestein_f2_flops(info, 256) == 256 * 128 * (10.0 * 4096 * 12 + 6.0 * 4096)
    assert bench._traffic("fzp-d2m", "dense") is None  # nothing captured for this workload
    for wl in ("fzp-d0.25m", "fzp-d1m"):
        t = bench._traffic(wl, "dense")
        assert t is None or t > 1e9  # reported only while the sources hash to the capture


def test_reference_arm_under_torchrun_prints_on_rank0_only():
    """Launched as N ranks (torchrun's environment), the reference arm runs on
    rank 0 alone; the other ranks exit 0 without work or output."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--workload",
           "fzp-d0.05m", "--steps", "1", "--warmup", "0", "--ref-rows", "2"]
    outs = {}
    for rank in (0, 1):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank))
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
        assert r.returncode == 0, r.stderr[-2000:]
        outs[rank] = [l for l in r.stdout.splitlines() if l.strip()]
    assert outs[1] == []
    assert len(outs[0]) == 1
    d = json.loads(outs[0][0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2


def test_disc_sample_count_of_the_roofline(oracle_mod):
    """The roofline's work count (samples inside the aperture disc over the
    timed rows) from the library's host plan equals the oracle's aperture
    count over all rows, and splits additively over row ranges."""
    import paper_2609_01978_gb300 as fzp
    import __graft_entry__
    __graft_entry__.build()
    for D, f in [(4e-3, 20e-3), (0.05, 0.25)]:
        q = fzp.plan_query(D=D, f=f, lam=632.8e-9, M=64, pitch=0.4e-6)
        g = oracle_mod.Geometry(D=D, f=f, lam=632.8e-9, M=64, p=0.4e-6)
        N, c, sR = q["N"], q["c"], q["s_R"]
        assert N == g.N
        assert bench.disc_samples(N, c, sR, 0, N) == oracle_mod.count_aperture(g)
        mid = N // 3
        assert bench.disc_samples(N, c, sR, 0, mid) + bench.disc_samples(N, c, sR, mid, N) == \
            bench.disc_samples(N, c, sR, 0, N)


def test_reference_arm_saczt_line():
    """The SA-CZT workload's reference arm: the oracle's SA-CZT of the 2 mm
    sample plate, whole, with the sample named."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "saczt-d8mm", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["workload"] == "saczt-d8mm"
    assert d["config"]["sample_N"] == 2529 and "4096^2" in d["cpu_baseline"]["sample"]
    assert d["e2e"]["value"] == d["value"]


def test_partitioned_flop_model():
    """The partitioned row pass's work count: per row one inverse 4096-point
    FFT, per block of S columns that meets the row's chord a forward FFT and
    the spectrum product-sum; the block count checked against a plain loop
    over rows and columns on a small plate, and the rows' counts add up."""
    import math
    import paper_2609_01978_gb300 as fzp
    import __graft_entry__
    __graft_entry__.build()
    q = fzp.plan_query(D=0.01, f=0.05, lam=632.8e-9, M=512, pitch=0.4e-6)
    info = {"N": q["N"], "c": q["c"], "s_R": q["s_R"], "M": 512}
    S = 256 * min(15, (4097 - 512) // 256)
    assert S == 3584
    N, c, sR = info["N"], info["c"], info["s_R"]
    blocks = 0
    for j in range(N):
        rem = sR - (j - c) ** 2
        if rem < 0:
            continue
        b = math.isqrt(rem)
        blocks += len({i // S for i in range(max(c - b, 0), min(c + b, N - 1) + 1)})
    fft = 5.0 * 4096 * 12
    assert bench.partitioned_flops(info, 0, N) == blocks * (fft + 8.0 * 4096) + N * fft
    assert bench.partitioned_flops(info, 0, N // 3) + bench.partitioned_flops(info, N // 3, N) == \
        bench.partitioned_flops(info, 0, N)


def test_plan_reports_the_row_convolution():
    """fzp_plan_query resolves fzp_params.conv: partitioned by default in FP32
    (4096-point inner transforms), single when asked for or in FP64."""
    import paper_2609_01978_gb300 as fzp
    import __graft_entry__
    __graft_entry__.build()
    base = dict(D=4e-3, f=20e-3, lam=632.8e-9, M=256, pitch=0.2e-6, form=fzp.FORM_BLUESTEIN)
    q = fzp.plan_query(precision=fzp.PREC_FP32, **base)
    assert q["conv"] == 2 and q["fft_inner"] == 4096 and q["fft_length"] == 8192
    q = fzp.plan_query(precision=fzp.PREC_FP32, conv=fzp.CONV_SINGLE, **base)
    assert q["conv"] == 1 and q["fft_inner"] == 4096
    q = fzp.plan_query(precision=fzp.PREC_FP64, **base)
    assert q["conv"] == 1
    q = fzp.plan_query(precision=fzp.PREC_SPLIT_BF16, form=fzp.FORM_DENSE,
                       **{k: v for k, v in base.items() if k != "form"})
    assert q["conv"] == 0


def test_membrane_batch_roofline_follows_the_majority_form():
    """The membranes line's roofline: tensor work of the dense instances when
    they are at least half the batch, else the FFT work of the partitioned
    FP32 instances, each over the whole step's time."""
    import paper_2609_01978_gb300 as fzp
    import __graft_entry__
    __graft_entry__.build()
    q = fzp.plan_query(D=0.01, f=0.05, lam=550e-9, M=256, pitch=550e-9 * 5 / 8)
    base = {"N": q["N"], "c": q["c"], "s_R": q["s_R"], "M": 256}
    dense = dict(base, form=fzp.FORM_DENSE, precision=fzp.PREC_SPLIT_BF16, conv=0)
    fp32 = dict(base, form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP32, conv=2)
    ms = 1000.0
    forms, roof = bench.membrane_forms_and_roofline(fzp, [fp32, fp32, dense], 256, 1, ms)
    assert forms == {"bluestein/f32": 2, "dense/split-bf16": 1}
    assert roof["bound"] == "alu"
    assert abs(roof["achieved"] - 2 * bench.partitioned_flops(fp32, 0, base["N"]) / 1e12) < 1e-9
    forms, roof = bench.membrane_forms_and_roofline(fzp, [dense, fp32], 256, 2, ms)
    inside = bench.disc_samples(base["N"], base["c"], base["s_R"], 0, base["N"])
    assert roof["bound"] == "tensor" and abs(roof["achieved"] - 2 * 24.0 * 256 * inside / 1e12) < 1e-9
    assert bench.membrane_forms_and_roofline(fzp, [], 256, 1, ms) == ({}, None)
