#!/usr/bin/env python
"""Benchmark of the stripe-processed CZT Fresnel propagator (one JSON line).

A step is one pass of the whole hot path over the workload: every aperture row
of a procedurally generated binary Fresnel zone plate through the row transform
(mask generation, chirps, row CZT), the column pass with FP64 cross-stripe
accumulation, the output chirp / prefactor epilogue, and the metric extractor
(FWHM, DE, MTF).  The metric is aperture samples (N^2 per step) per second into
a 512^2 ROI.

Workload (default "fzp-d1m", the first plate of the D sweep at f/# = 5):
binary amplitude FZP, D = 1.0 m, lambda = 632.8 nm, f/# = 5 (f = 5 m), 4
samples per outermost zone width (dx = 0.791 um, N = 1,264,223 per side,
1.60e12 samples), ROI 512^2 at lambda f/# / 8 = 0.3955 um, centred on the
focus.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form dense|bluestein]
                  [--conv partitioned|single]
                  [--impl ours|reference] [--workload NAME] [--rows R]
                  [--plain-rows R] [--e2e-steps E] [--no-plain] [--no-cpu-baseline]
                  [--ref-rows R] [--instances I] [--seed S] [--replicas]
                  [--train T] [--test E] [--flat F] [--train-steps S]

Workloads: fzp-d0.05m (small case for profiler captures), fzp-d0.25m,
fzp-d1m ... fzp-d5m (the D sweep at f/# = 5), fzp-t1 ... fzp-t5 (the phase
plates of Tables 1-5 on their own grids), membranes (a batch of the seeded
deformed membranes, autotuned per instance, one CUDA graph per step),
surrogate (training-set generation and the trained network's held-out
error), saczt-d8mm (the SA-CZT form on an exact-radii plate; its roofline is
the zoom product's, and its oracle sample a 2 mm plate of the same method).
--rows R times R central aperture rows per step (a sample, named in the
config); --form bluestein times the plain FP32 form itself, with --conv its
row convolution (partitioned into 4096-point blocks, the default, or the
paper's single L-point convolution).  Beside the dense form the line carries
the plain FP32 form with both convolutions ("plain_fp32": partitioned,
"plain_fp32_single"), each timed on the whole aperture up to D = 0.25 m and
on 16 stripes spread evenly over the aperture above (--plain-rows R rows in
all; the partitioned convolution's cost per row follows the row's disc
chord, so a central sample would understate it); --e2e-steps 0 leaves out
the end-to-end leg; --ref-rows sets the oracle's rows per step in the
reference arm.

The cpu_baseline leg also checks parity: the oracle's FP64 field of its timed
row sample against the GPU forms' fields of the same rows (relative L2 of I,
tolerance 1e-4), outside the timed region.

Under torchrun (N > 1) the aperture is split into contiguous row ranges of
about equal open-sample count, one per rank; each rank propagates its range
and one all_reduce sums the M x M fields (strong scaling: the whole job is
one aperture).  With --replicas every rank propagates the whole aperture
instead (independent problems, weak scaling).  Rank 0 prints the line with
the max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "fzp-d0.05m": dict(D=0.05, lam=632.8e-9, fnum=5.0, M=512),  # small case for profiler captures
    "fzp-d0.25m": dict(D=0.25, lam=632.8e-9, fnum=5.0, M=512),
    "fzp-d1m": dict(D=1.0, lam=632.8e-9, fnum=5.0, M=512),  # the D sweep at f/# = 5 (N up to 6.3e6)
    "fzp-d2m": dict(D=2.0, lam=632.8e-9, fnum=5.0, M=512),
    "fzp-d3m": dict(D=3.0, lam=632.8e-9, fnum=5.0, M=512),
    "fzp-d4m": dict(D=4.0, lam=632.8e-9, fnum=5.0, M=512),
    "fzp-d5m": dict(D=5.0, lam=632.8e-9, fnum=5.0, M=512),
    # the paper's Tables 1-5 (lambda = 532 nm, f/# = 5, dx = Lambda_edge / k with
    # Lambda_edge = lambda f / R): L-level phase plates; Nx = 12,030,077 /
    # 12,030,077 / 9,022,557 / 12,030,077 / 15,037,595
    "fzp-t1": dict(D=1.0, lam=532e-9, fnum=5.0, M=512, levels=16, k=64),
    "fzp-t2": dict(D=2.0, lam=532e-9, fnum=5.0, M=512, levels=8, k=32),
    "fzp-t3": dict(D=3.0, lam=532e-9, fnum=5.0, M=512, levels=4, k=16),
    "fzp-t4": dict(D=4.0, lam=532e-9, fnum=5.0, M=512, levels=4, k=16),
    "fzp-t5": dict(D=5.0, lam=532e-9, fnum=5.0, M=512, levels=2, k=16),
    # batched deformed membranes (D ~ U[0.05, 0.30] m, 450/550/650 nm, ROI 256^2,
    # seed 0): the first --instances of the 256 draws, one CUDA graph per step
    "membranes": dict(D=0.0, lam=0.0, fnum=5.0, M=256),
    # learned surrogate on D = 0.2 m membranes (λ 450-650 nm, ROI 128², seed 11):
    # --train PSFs from the dense membrane passes, --test held out and judged by
    # the plain FP32 CZT
    "surrogate": dict(D=0.2, lam=0.0, fnum=5.0, M=128),
    # one deformed membrane through the main path: the first config-4 draw
    # (seed 0) with its deformation scaled onto a D = 0.05 m plate (N = 72,729),
    # ROI 256^2 (the small case of the membrane-pass profiles)
    "membrane-d0.05m": dict(D=0.05, lam=0.0, fnum=5.0, M=256, membrane=0),
    # the SA-CZT form (Sec. 3.6, Fig. 5): exact-radii plate (Eq. 3), D = 8 mm at
    # f/# = 5 (N = 10,115, padded grid 16,384^2), exact angular-spectrum residual,
    # Fresnel chirp and zoom onto the 512^2 ROI
    "saczt-d8mm": dict(D=8e-3, lam=632.8e-9, fnum=5.0, M=512, saczt=True),
}
# the oracle's bounded sample for the SA-CZT workloads: the same method on a
# D = 2 mm plate (N = 2,529, padded grid 4096^2), whole, repeated
SACZT_SAMPLE_D = 2e-3
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dominant kernel (for the dense form: one row pass, both of its
# launches), from a one-pass ncu capture of this workload; reported only while
# the kernel's sources hash to what was captured (null otherwise).
KERNEL_SOURCES = {
    "dense": ["dense.cu", "tc_ptx.cuh", "fzp_internal.cuh"],
    "bluestein": ["bluestein.cu", "fzp_internal.cuh"],
}
TRAFFIC = {
    # both launches of a row pass (the cluster launch and the single-CTA band
    # on the leftover SMs), captured one after the other
    ("fzp-d0.25m", "dense"): (80.311e9 + 76.917e9 + 1.657e9 + 1.776e9, "3c073e7364fc6793e3ba5531cd0932794ecbf242e89dca2de577b8b85171f0c2"),
    ("fzp-d1m", "dense"): (1796.474e9 + 1216.386e9 + 43.721e9 + 41.508e9, "3c073e7364fc6793e3ba5531cd0932794ecbf242e89dca2de577b8b85171f0c2"),
}
METRIC = "aperture Gsamples/s into 512² ROI, split-BF16 vs FP32 CZT at ≤1e-4 PSF error"
UNIT = "Gsamples/s"
SM_COUNT = 152
SM_MAX_MHZ_NOMINAL = 2070.0


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _traffic(workload, form):
    """Captured per-launch DRAM bytes of the dominant kernel, or None when the
    kernel has changed since the capture."""
    import hashlib
    hit = TRAFFIC.get((workload, form))
    if hit is None:
        return None
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[form]:
        with open(os.path.join(ROOT, "paper_2609_01978_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return hit[0] if h.hexdigest() == hit[1] else None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _print(obj):
    print(json.dumps(obj), flush=True)


def bluestein_f2_flops(info: dict, rows: int) -> float:
    """Algorithmic FP32 flops of the dominant Bluestein pass (forward L2-point FFT,
    product with H, inverse L2-point FFT) for `rows` aperture rows: per row and
    per inner transform 2 x 5 L2 log2 L2 + 6 L2, L1 inner transforms per row."""
    L = info["fft_length"]
    L2 = info["fft_inner"]
    L1 = L // L2
    lg = L2.bit_length() - 1
    return rows * L1 * (10.0 * L2 * lg + 6.0 * L2)


def partitioned_flops(info: dict, j0: int, j1: int) -> float:
    """Algorithmic FP32 flops of the partitioned row pass over rows [j0, j1):
    per block of S columns that meets a row's disc chord, one forward
    4096-point FFT (5 P log2 P) and the spectrum product-sum (8 P); per row one
    inverse 4096-point FFT.  S = 256 min(15, floor((4097 - M) / 256))."""
    import numpy as np
    P, lgP = 4096, 12
    S = 256 * min(15, (4097 - info["M"]) // 256)
    N, c, s_R = info["N"], info["c"], info["s_R"]
    rem = s_R - (np.arange(j0, j1, dtype=np.int64) - c) ** 2
    rem = rem[rem >= 0]
    b = np.floor(np.sqrt(rem.astype(np.float64))).astype(np.int64)  # exact after the corrections
    b -= (b * b > rem).astype(np.int64)
    b += ((b + 1) * (b + 1) <= rem).astype(np.int64)
    lo, hi = np.maximum(c - b, 0), np.minimum(c + b, N - 1)
    blocks = float(np.sum(hi // S - lo // S + 1))
    fft = 5.0 * P * lgP
    return blocks * (fft + 8.0 * P) + (j1 - j0) * fft


def membrane_forms_and_roofline(fzp, infos: list, M: int, steps: int, ms: float):
    """Forms chosen over a batch of membranes and the roofline of the step:
    the tensor work of the dense instances (24 M flops per in-disc sample:
    2 membrane passes x 3 split products x 2 real rows x M x 2 flops) when
    dense instances are at least half the batch, else the FFT work of the
    partitioned FP32 instances; either over the whole step's time, so a lower
    bound for a mixed batch."""
    forms = {}
    dense_flops = fft_flops = 0.0
    n_dense = n_fft = 0
    for inf in infos:
        k = ("dense" if inf["form"] == fzp.FORM_DENSE else "bluestein") + "/" + \
            {0: "f64", 1: "f32", 2: "split-bf16", 3: "bf16"}[inf["precision"]]
        forms[k] = forms.get(k, 0) + 1
        if inf["form"] == fzp.FORM_DENSE:
            dense_flops += 24.0 * M * disc_samples(inf["N"], inf["c"], inf["s_R"], 0, inf["N"])
            n_dense += 1
        elif inf["precision"] == fzp.PREC_FP32 and inf["conv"] == 2:
            fft_flops += partitioned_flops(inf, 0, inf["N"])
            n_fft += 1
    peaks, peak_kind = _peaks()
    whole = "whole step (graph of every instance's passes)"
    if n_dense and n_dense >= n_fft:
        achieved = dense_flops * steps / (ms / 1e3) / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        return forms, {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                       "frac": achieved / peak, "traffic": None,
                       "kernel": whole + ": tensor work of the dense instances over the whole step's time "
                                         "(a lower bound when some chose the FP32 form)",
                       "peak_source": peak_kind + " bf16 sustained",
                       "work": "24 M flops per aperture sample inside the disc (dense instances only)"}
    if n_fft:
        achieved = fft_flops * steps / (ms / 1e3) / 1e12
        peak = SM_COUNT * 128 * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
        return forms, {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                       "frac": achieved / peak, "traffic": None,
                       "kernel": whole + ": FFT work of the partitioned FP32 instances over the whole step's "
                                         "time (a lower bound when some chose the dense form)",
                       "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                       "work": "per block of S columns meeting a row's chord 5 P log2 P + 8 P, per row "
                               "5 P log2 P (P = 4096; partitioned FP32 instances only)"}
    return forms, None


def run_membranes(args, fzp, torch, dev, ws, pg, rank, local):
    """Config 4: a batch of deformed membranes (autotuned form per instance), the
    whole batch replayed as one CUDA graph, metrics of every instance per step."""
    import fzp_inputs
    wl = WORKLOADS["membranes"]
    fnum, M = wl["fnum"], wl["M"]
    mem = fzp_inputs.batch_draws(256, seed=args.seed)[:args.instances]
    probs = [dict(D=m.D, f=fnum * m.D, lam=m.lam, M=M, pitch=m.lam * fnum / 8, precision=fzp.PREC_AUTO_1E4,
                  deform=fzp.make_deform(m.amp, m.period, m.theta, m.taper, m.ridges)) for m in mem]
    stream = torch.cuda.current_stream(dev)
    b = fzp.Batch(probs)  # autotunes every instance (cached per process for the e2e leg)
    infos = [b.info(i) for i in range(len(probs))]
    samples = sum(inf["N"] ** 2 for inf in infos)
    fields = [torch.empty((M, M), dtype=torch.complex128, device=dev) for _ in probs]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        flush.fill_(1.0)
        b.propagate(fields, stream=stream)
        return [b.metrics(i, fields[i], stream=stream) for i in range(len(probs))]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        mets = step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop() if sampler else None
    if pg:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    kernels = b.kernels
    b.close()
    forms, roof = membrane_forms_and_roofline(fzp, infos, M, args.steps, ms)
    # end to end through the public API with host buffers: batch from host
    # parameters (tuned choices cached in-process), propagate, fields to pinned
    # host memory, every instance's metrics, destroy
    e2e = None
    n_e2e = min(args.e2e_steps, 1)  # one end-to-end batch: a step of the full batch takes minutes
    if n_e2e > 0:
        hosts = [torch.empty((M, M), dtype=torch.complex128, pin_memory=True) for _ in probs]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h2d = 0
        for _ in range(n_e2e):
            b2 = fzp.Batch(probs)
            h2d = sum(8 * b2.info(i)["n_thresholds"] for i in range(len(probs)))
            b2.propagate(fields, stream=stream)
            for i in range(len(probs)):
                hosts[i].copy_(fields[i], non_blocking=True)
            for i in range(len(probs)):
                b2.metrics(i, fields[i], stream=stream)
            torch.cuda.synchronize(dev)
            b2.close()
        e2e_s = (time.perf_counter() - t0) / n_e2e
        e2e = {"value": ws * samples / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": len(probs) * (M * M * 16 + 8 * 1024 + 4),
               "note": "fzp_batch_plan (tuning cached) + graph capture and launch + fields to pinned host + "
                       "fzp_batch_metrics per instance + fzp_batch_destroy"}
    return {"metric": METRIC, "value": ws * args.steps * samples / (ms / 1e3) / 1e9, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "mixed (autotuned per instance)",
            "data": "synthetic (seeded deformed membranes)",
            "config": {"workload": "membranes", "instances": len(probs), "of": 256, "seed": args.seed, "roi": M,
                       "f_number": fnum, "samples_per_step": samples, "forms": forms,
                       "l2": "256 MiB buffer written between steps (flush)"},
            "roofline": roof, "e2e": e2e, "gpu_launches": kernels * args.steps, "clocks": clocks,
            "per_instance_ms": ms / args.steps / len(probs),
            "de_lobe_range": [min(m["de_lobe"] for m in mets), max(m["de_lobe"] for m in mets)]}


def run_surrogate(args, fzp, torch, dev):
    """Config 5 at D = 0.2 m: training PSFs generated by the dense membrane
    passes (timed: the value is their aperture Gsamples/s), a held-out set
    judged by the plain FP32 CZT, the trained network's error on it against
    two baselines without a learned part, and the time per instance of the
    surrogate and of both propagation forms."""
    import numpy as np
    import fzp_inputs
    from paper_2609_01978_gb300 import surrogate as SG
    D = WORKLOADS["surrogate"]["D"]
    ntr, nte = args.train, args.test
    mem, X = fzp_inputs.surrogate_draws(ntr + nte, seed=11, D=D)
    samples = sum(fzp.plan_query(D=m.D, f=5.0 * m.D, lam=m.lam, M=128, pitch=m.lam * 5.0 / 8)["N"] ** 2
                  for m in mem[:ntr])
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    Y, psf, _ = SG.generate(mem[:ntr])
    torch.cuda.synchronize(dev)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    Yte, T, ideal = SG.generate(mem[ntr:], form=SG.PLAIN)
    t_plain = (time.perf_counter() - t0) / nte
    _, Tdense, _ = SG.generate(mem[ntr:])
    dense_vs_plain = [float(np.linalg.norm(Tdense[k] - T[k]) / np.linalg.norm(T[k])) for k in range(nte)]
    t0 = time.perf_counter()
    model = SG.train(X[:ntr], Y, D, steps=args.train_steps)
    t_train = time.perf_counter() - t0
    pred = model.predict(X[ntr:])
    P = SG.psf_from_targets(pred, ideal)
    err = np.array([np.linalg.norm(P[k] - T[k]) / np.linalg.norm(T[k]) for k in range(nte)])
    nflat = min(nte, args.flat)
    flat_mem = [fzp_inputs.Membrane(0.0, m.period, m.theta, 0.0, [(a, b, c, 0.0, w) for a, b, c, _, w in m.ridges],
                                    m.lam, m.D) for m in mem[ntr:ntr + nflat]]
    _, flat, _ = SG.generate(flat_mem, form=SG.PLAIN)
    err_flat = np.array([np.linalg.norm(flat[k] - T[k]) / np.linalg.norm(T[k]) for k in range(nflat)])
    mean_psf = psf.mean(0)
    err_mean = np.array([np.linalg.norm(mean_psf - T[k]) / np.linalg.norm(T[k]) for k in range(nte)])
    de_err = np.abs(pred[:, 4097] - Yte[:, 4097])
    fwhm_err = np.abs(pred[:, 4096] / Yte[:, 4096] - 1)
    xb = torch.from_numpy(SG.encode(np.tile(X[ntr:], (max(1, 256 // nte), 1))[:256], D).astype(np.float32)).to(dev)
    yb = torch.empty((xb.shape[0], Y.shape[1]), dtype=torch.float32, device=dev)
    model.net.infer(xb, yb)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(20):
        model.net.infer(xb, yb)
    torch.cuda.synchronize(dev)
    t_inf = (time.perf_counter() - t0) / (20 * xb.shape[0])
    return {"metric": METRIC, "value": samples / t_gen / 1e9, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": 1e3 * t_gen, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x2 (dense membrane passes)", "data": "synthetic (seeded deformed membranes)",
            "config": {"workload": "surrogate", "D_m": D, "roi": 128, "crop": 64, "f_number": 5.0, "seed": 11,
                       "train": ntr, "test": nte, "train_steps": args.train_steps,
                       "samples_per_step": samples, "note": "value: aperture Gsamples/s of the training-set "
                                                             "generation (dense membrane passes, one batch graph "
                                                             "per 128 instances, metrics and intensity included)"},
            "roofline": None, "e2e": None, "gpu_launches": None,
            "surrogate": {"heldout_psf_rel_l2_median": float(np.median(err)), "heldout_psf_rel_l2_mean": float(err.mean()),
                          "baseline_flat_fzp_median": float(np.median(err_flat)), "baseline_flat_n": nflat,
                          "baseline_mean_psf_median": float(np.median(err_mean)),
                          "de_abs_err_median": float(np.median(de_err)), "fwhm_rel_err_median": float(np.median(fwhm_err)),
                          "judge": "plain FP32 Bluestein CZT", "dense_vs_plain_targets_max": max(dense_vs_plain),
                          "s_per_instance_dense": t_gen / ntr, "s_per_instance_plain": t_plain,
                          "s_per_instance_surrogate": t_inf, "train_s": t_train}}


def _config(args, wl, N):
    """The workload description shared by both arms' JSON lines."""
    rows = N if args.rows <= 0 else min(N, args.rows)
    cfg = {"workload": args.workload, "form": args.form, "D_m": wl["D"], "lambda_m": wl["lam"],
           "f_number": wl["fnum"], "N": N, "samples_per_step": rows * N, "roi": wl["M"],
           "roi_pitch_m": wl["lam"] * wl["fnum"] / 8, "l2": "256 MiB buffer written between steps (flush)"}
    if args.form == "bluestein":
        cfg["conv"] = args.conv
    if wl.get("levels"):
        cfg.update(levels=wl["levels"], dx_m=_dx(wl))
    if wl.get("deform"):
        cfg.update(membrane=f"config-4 draw {wl['membrane']} (seed 0) scaled to D", deform=wl["deform"])
    if rows < N:
        cfg["rows_timed"] = f"{rows} central aperture rows of {N} per step (a sample)"
    return cfg


def _dx(wl):
    """Table workloads: dx = Lambda_edge / k, Lambda_edge = lambda f / R."""
    return wl["lam"] * wl["D"] * wl["fnum"] / (wl["D"] / 2) / wl["k"]


def _oracle_geometry(O, wl):
    kw = dict(D=wl["D"], f=wl["D"] * wl["fnum"], lam=wl["lam"], M=wl["M"], p=wl["lam"] * wl["fnum"] / 8)
    if wl.get("levels"):
        kw.update(kind=O.FZP_PHASE, levels=wl["levels"], dx=_dx(wl))
    if wl.get("deform"):
        kw.update(deform=O.Deform(**wl["deform"]))
    return O.Geometry(**kw)


def _resolve(wl):
    """A membrane workload takes its wavelength and deformation from its seeded
    config-4 draw, the deformation's lengths scaled from the draw's D to the
    workload's."""
    if wl.get("membrane") is None:
        return wl
    import fzp_inputs
    m = fzp_inputs.batch_draws(8, seed=0)[wl["membrane"]]
    k = wl["D"] / m.D
    d = dict(amp=m.amp, period=m.period * k, theta=m.theta, taper=m.taper,
             ridges=[(px * k, py * k, al, h, w * k) for (px, py, al, h, w) in m.ridges])
    return dict(wl, lam=m.lam, deform=d)


def run_reference(args, wl):
    """The oracle (CPU FP64 Bluestein CZT, fzp_oracle.c) timed on the host cores on
    a bounded sample of aperture rows of the same workload."""
    import oracle as O
    if wl.get("saczt"):
        return run_reference_saczt(args, wl)
    g = _oracle_geometry(O, wl)
    rows = args.ref_rows
    j0 = g.c - rows // 2
    for _ in range(args.warmup):
        O.field_czt(g, j0, j0 + rows)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.field_czt(g, j0, j0 + rows)
    dt = time.perf_counter() - t0
    value = args.steps * rows * g.N / dt / 1e9
    cores = O.max_threads()
    sample = f"{rows} central aperture rows of {g.N} (x {args.steps} steps), full row and column CZT, FP64"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (procedural zone plate)",
            "config": dict(_config(args, wl, g.N), rows_per_step=rows),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _saczt_sample_geometry(O, wl):
    D = SACZT_SAMPLE_D
    return O.Geometry(D=D, f=D * wl["fnum"], lam=wl["lam"], M=wl["M"], p=wl["lam"] * wl["fnum"] / 8,
                      kind=O.FZP_EXACT)


def run_reference_saczt(args, wl):
    """The oracle's SA-CZT (FP64, numpy transforms and products) on the 2 mm
    sample plate, whole, once per step."""
    import oracle as O
    from oracle import saczt as SA
    g = _saczt_sample_geometry(O, wl)
    for _ in range(args.warmup):
        SA.field_saczt(g)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        SA.field_saczt(g)
    dt = time.perf_counter() - t0
    value = args.steps * g.N * g.N / dt / 1e9
    sample = (f"SA-CZT of a D = {g.D:g} m exact-radii plate (N = {g.N}, padded grid {SA.pad_size(g.N)}^2), "
              f"whole, x {args.steps} steps, FP64; numpy FFTs on one thread, BLAS products on the host cores")
    cfg = {"workload": args.workload, "form": "saczt", "D_m": wl["D"], "lambda_m": wl["lam"],
           "f_number": wl["fnum"], "roi": wl["M"], "sample_D_m": g.D, "sample_N": g.N}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (procedural zone plate, exact radii)", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def cpu_baseline_saczt(wl, budget_s: float = 15.0) -> dict:
    """The oracle's SA-CZT on the 2 mm sample plate, repeated until half the
    budget has passed; returns its field for the parity check (private keys)."""
    import numpy as np
    import oracle as O
    from oracle import saczt as SA
    g = _saczt_sample_geometry(O, wl)
    reps, t0 = 0, time.perf_counter()
    while True:
        U = SA.field_saczt(g)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= 0.5 * budget_s:
            break
    return {"value": reps * g.N * g.N / dt / 1e9, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"SA-CZT (FP64, numpy) of a D = {g.D:g} m exact-radii plate, N = {g.N}, padded grid "
                      f"{SA.pad_size(g.N)}^2, whole, {reps} x, {dt:.1f} s; numpy FFTs on one thread, BLAS "
                      f"products on the host cores",
            "seconds": dt, "_geometry": g, "_I": np.abs(U) ** 2,
            "_airy_fwhm": O.airy_fwhm_factor() * g.lam * g.f / (2 * g.R),
            "_lobe_de": O.airy_encircled(O.AIRY_NULL) * O.binary_fzp_efficiency()}


def cpu_baseline(wl, budget_s: float = 15.0) -> dict:
    """The oracle (O3, FP64, all host cores) on a sample of central rows grown
    until one evaluation takes at least half the budget.  Also returns the
    sample's rows and intensity (private keys, for the parity check) and the
    closed forms the full-aperture metrics are read against."""
    import numpy as np
    import oracle as O
    g = _oracle_geometry(O, wl)
    # grow the sample until one evaluation takes at least half the budget (small
    # samples carry fixed costs, so one extrapolation undershoots)
    rows = 16
    while True:
        j0 = g.c - rows // 2
        t0 = time.perf_counter()
        U = O.field_czt(g, j0, j0 + rows)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * budget_s or rows >= g.N:
            break
        rows = min(g.N, max(2 * rows, int(rows * budget_s / max(dt, 1e-3))))
    return {"value": rows * g.N / dt / 1e9, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
            "sample": f"{rows} central aperture rows of N = {g.N} (row + column CZT, FP64), {dt:.1f} s",
            "seconds": dt, "_rows": (j0, j0 + rows), "_I": np.abs(U) ** 2,
            "_airy_fwhm": O.airy_fwhm_factor() * g.lam * g.f / (2 * g.R),
            "_lobe_de": O.airy_encircled(O.AIRY_NULL) * (O.phase_fzp_efficiency(g.levels) if g.levels
                                                         else O.binary_fzp_efficiency())}


def _rel_l2(a, b):
    import numpy as np
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _rows_intensity(fzp, torch, plan, M, j0, j1, stream, dev):
    U = torch.empty((M, M), dtype=torch.complex128, device=dev)
    plan.propagate_roi(j0, j1, U, stream=stream)
    I = torch.empty((M, M), dtype=torch.float64, device=dev)
    plan.intensity(U, I, stream=stream)
    torch.cuda.synchronize(dev)
    return I.cpu().numpy()


def disc_samples(N: int, c: int, s_R: int, j0: int, j1: int) -> int:
    """Aperture samples inside the disc on rows [j0, j1): per row the chord
    2 floor(sqrt(s_R - dj^2)) + 1 (integer arithmetic; dj = j - c)."""
    import math
    b = math.isqrt(s_R)
    lo, hi = max(j0, c - b), min(j1, c + b + 1)
    return sum(2 * math.isqrt(s_R - (j - c) ** 2) + 1 for j in range(lo, hi))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fzp-d1m", choices=sorted(WORKLOADS))
    ap.add_argument("--form", default="dense", choices=["dense", "bluestein", "saczt"])
    ap.add_argument("--conv", default="partitioned", choices=["partitioned", "single"],
                    help="--form bluestein: the row convolution (fzp_params.conv)")
    ap.add_argument("--ref-rows", type=int, default=48)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain FP32 Bluestein form")
    ap.add_argument("--plain-rows", type=int, default=-1,
                    help="rows of the plain form's timed sample (0: all; -1: all up to N = 316,057, else 16,384)")
    ap.add_argument("--replicas", action="store_true",
                    help="N > 1: every rank propagates the whole aperture (weak scaling) instead of its rows")
    ap.add_argument("--instances", type=int, default=256, help="membranes workload: instances per batch")
    ap.add_argument("--seed", type=int, default=0, help="membranes workload: seed of the 256 draws (0: config 4's)")
    ap.add_argument("--train", type=int, default=768, help="surrogate workload: training PSFs")
    ap.add_argument("--test", type=int, default=64, help="surrogate workload: held-out PSFs (judged by the plain CZT)")
    ap.add_argument("--flat", type=int, default=32, help="surrogate workload: held-out PSFs of the flat baseline")
    ap.add_argument("--train-steps", type=int, default=3000, help="surrogate workload: AdamW steps")
    ap.add_argument("--rows", type=int, default=0,
                    help="time only this many central aperture rows per step (a sample; 0: all N)")
    args = ap.parse_args()
    wl = _resolve(WORKLOADS[args.workload])
    ws, rank, local = _dist()

    if args.impl == "reference":
        if rank == 0:
            _print(run_reference(args, wl))
        return

    import torch
    import __graft_entry__
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    import paper_2609_01978_gb300 as fzp

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
        if rank != 0:
            __graft_entry__.build()  # already built by rank 0; loads the library
        dist.barrier()
    if args.workload == "surrogate":
        if rank == 0:
            _print(run_surrogate(args, fzp, torch, dev))
        if pg:
            pg.destroy_process_group()
        return
    if args.workload == "membranes":
        out = run_membranes(args, fzp, torch, dev, ws, pg, rank, local)
        if rank == 0:
            _print(out)
        if pg:
            pg.destroy_process_group()
        return
    D, lam, fnum, M = wl["D"], wl["lam"], wl["fnum"], wl["M"]
    if wl.get("saczt"):
        args.form, args.no_plain = "saczt", True
    if args.form == "saczt":
        if not wl.get("saczt"):
            raise SystemExit("--form saczt needs an SA-CZT workload (saczt-d8mm)")
        form, prec = fzp.FORM_SACZT, fzp.PREC_FP32
        dtype = "f32 transforms + bf16x2 zoom" if M % 128 == 0 else "f32"
    elif args.form == "dense":
        form, prec, dtype = fzp.FORM_DENSE, fzp.PREC_SPLIT_BF16, "bf16x2"
    else:
        form, prec, dtype = fzp.FORM_BLUESTEIN, fzp.PREC_FP32, "f32"
    params = dict(D=D, f=D * fnum, lam=lam, M=M, pitch=lam * fnum / 8, form=form, precision=prec)
    if args.form == "bluestein":
        params.update(conv=fzp.CONV_SINGLE if args.conv == "single" else fzp.CONV_PARTITIONED)
    if args.form == "saczt":
        params.update(exact_radii=1)
        if ws > 1 and not args.replicas:
            raise SystemExit("the SA-CZT form transforms the whole padded grid: run it with --replicas")
    if wl.get("levels"):
        params.update(levels=wl["levels"], dx=_dx(wl))
    if wl.get("deform"):
        params.update(deform=fzp.make_deform(**wl["deform"]))
    plan = fzp.Plan(**params)
    info = plan.info
    N = info["N"]
    rows = N if args.rows <= 0 else min(N, args.rows)  # timed rows per step (all ranks together)
    r0 = (N - rows) // 2
    sharded = ws > 1 and not args.replicas
    j0, j1 = r0, r0 + rows  # this rank's rows
    if sharded:
        from paper_2609_01978_gb300 import shard
        w = shard.chord_weights(N, info["c"], info["s_R"])[r0:r0 + rows]
        a, b = shard.row_ranges(rows, ws, w)[rank]
        j0, j1 = r0 + a, r0 + b
    stream = torch.cuda.current_stream(dev)
    U = torch.empty((M, M), dtype=torch.complex128, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MiB > L2 (129 MB)

    def step():
        flush.fill_(1.0)  # evict L2 between steps
        plan.propagate_roi(j0, j1, U, stream=stream)
        if sharded:
            pg.all_reduce(U)  # the one exchange: sum of the ranks' partial fields
        return plan.metrics(U, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    plan.profile(True)
    plan.profile_read()  # reset counters
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        m = step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    ms = ev0.elapsed_time(ev1)
    prof = plan.profile_read()
    plan.profile(False)
    clocks = sampler.stop() if sampler else None
    if pg:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    value = (1 if sharded else ws) * args.steps * rows * N / (ms / 1e3) / 1e9

    # roofline of the dominant kernel, from CUDA events on its own stream
    peaks, peak_kind = _peaks()
    avg_ms = prof["dominant_ms"] / max(1, prof["dominant_launches"])
    if args.form == "dense":
        # algorithmic work of the contraction: 2 real rows (Re, Im) x M outputs x
        # 2 flops x 2 split terms per aperture sample inside the disc = 8 M
        # flops per such sample and mask pass (a phase plate with L >= 4 takes
        # L/2 passes); samples outside the disc carry no work and are skipped
        launches = max(1, prof["dominant_launches"])
        inside = disc_samples(N, info["c"], info["s_R"], j0, j1)
        per = 12.0 if wl.get("deform") else 8.0  # a membrane pass takes 3 split products, not 2
        flops_launch = per * M * inside * info["passes"] * args.steps / launches
        achieved = flops_launch / (avg_ms / 1e3) / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": _traffic(args.workload, "dense"), "kernel": prof["dominant_name"],
                "peak_source": peak_kind + " bf16 sustained",
                "work": f"{per:g} M flops per aperture sample inside the disc and mask pass",
                "disc_samples_per_launch": inside * args.steps / launches}
    elif args.form == "saczt":
        # k_sa_rows<1>: one pass of the padded grid through HBM (P^2 complex64
        # read and written) with two transforms and the residual phase between
        Pg = info["fft_length"]
        bytes_launch = 2.0 * 8.0 * Pg * Pg
        achieved = bytes_launch / (avg_ms / 1e3) / 1e9
        peak = peaks["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": prof["dominant_name"], "peak_source": peak_kind + " HBM copy",
                "work": "16 P^2 bytes per launch (P = padded grid side)"}
    else:
        launches = max(1, prof["dominant_launches"])
        if info["conv"] == 2:
            flops_launch = partitioned_flops(info, j0, j1) * args.steps / launches
            work = ("per block of S columns meeting a row's chord 5 P log2 P + 8 P, per row 5 P log2 P "
                    "(P = 4096)")
        else:
            flops_launch = bluestein_f2_flops(info, rows * args.steps / launches)
            work = "per row L1 (10 L2 log2 L2 + 6 L2)"
        achieved = flops_launch / (avg_ms / 1e3) / 1e12
        peak = SM_COUNT * 128 * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12  # FP32 FMA lanes x clock
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": _traffic(args.workload, "bluestein") if info["conv"] == 1 else None,
                "kernel": prof["dominant_name"], "work": work,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}

    # end to end through the public API with host buffers: plan from host
    # parameters (zone-threshold table uploaded), propagate, copy the ROI field
    # to pinned host memory, metrics to host, destroy.
    e2e = None
    if args.e2e_steps > 0:
        host = torch.empty((M, M), dtype=torch.complex128, pin_memory=True)
        torch.cuda.synchronize(dev)
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        h2d = 0
        for _ in range(args.e2e_steps):
            with fzp.Plan(**params) as p2:
                h2d = 8 * p2.info["n_thresholds"]  # the zone-threshold table, the plan's one upload
                p2.propagate_roi(j0, j1, U, stream=stream)
                if sharded:
                    pg.all_reduce(U)
                host.copy_(U, non_blocking=True)
                p2.metrics(U, stream=stream)
                torch.cuda.synchronize(dev)
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        if pg:
            t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            e2e_s = float(t.item())
        # read back: the complex128 field, the metric extractor's 1024-double
        # result block and its 4-byte error word
        e2e = {"value": (1 if sharded else ws) * rows * N / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": M * M * 16 + 8 * 1024 + 4,
               "note": "fzp_plan + fzp_propagate_roi + field to pinned host + fzp_metrics + fzp_plan_destroy"}

    # the oracle on the host cores (cpu_baseline), and parity: the oracle's
    # FP64 field of its timed rows against this form's field of the same rows
    cb, parity = None, None
    if ws == 1 and not args.no_cpu_baseline and args.form == "saczt":
        cb = cpu_baseline_saczt(wl)
        gs = cb.pop("_geometry")
        Iref = cb.pop("_I")
        with fzp.Plan(D=gs.D, f=gs.f, lam=gs.lam, M=gs.M, pitch=gs.p, form=form, precision=prec,
                      exact_radii=1) as ps:
            Is = _rows_intensity(fzp, torch, ps, M, 0, ps.info["N"], stream, dev)
        parity = {"oracle": "oracle SA-CZT (FP64) of the cpu_baseline sample plate, whole", "tolerance": 1e-4,
                  "sample_D_m": gs.D, "rel_l2_I_saczt": _rel_l2(Is, Iref)}
        cb.pop("_airy_fwhm")
        lobe = cb.pop("_lobe_de")
        import oracle as O
        gw = O.Geometry(D=D, f=D * fnum, lam=lam, M=M, p=lam * fnum / 8, kind=O.FZP_EXACT)
        airy = O.airy_fwhm_factor() * gw.lam * gw.f / (2 * gw.R)
        parity["full_aperture_vs_closed_forms"] = {
            "fwhm_x_over_airy_minus_1": m["fwhm_x"] / airy - 1,
            "de_lobe_over_ee_efficiency_minus_1": m["de_lobe"] / lobe - 1}
    elif ws == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(wl)
        pa, pb_ = cb.pop("_rows")
        Iref = cb.pop("_I")
        parity = {"rows": [pa, pb_], "oracle": "O3 (Bluestein CZT rows then columns, FP64) on the cpu_baseline sample",
                  "tolerance": 1e-4,
                  f"rel_l2_I_{args.form}": _rel_l2(_rows_intensity(fzp, torch, plan, M, pa, pb_, stream, dev), Iref)}
        airy, lobe = cb.pop("_airy_fwhm"), cb.pop("_lobe_de")
        if rows == N and not wl.get("deform"):  # the closed forms are the flat plate's
            parity["full_aperture_vs_closed_forms"] = {
                "fwhm_x_over_airy_minus_1": m["fwhm_x"] / airy - 1,
                "de_lobe_over_ee_efficiency_minus_1": m["de_lobe"] / lobe - 1}
    plan.close()

    # the plain FP32 Bluestein form on the same workload (the metric compares
    # the split-BF16 dense form with it), both of its row convolutions:
    # partitioned (the library's FP32 default) and single (one L-point
    # convolution per row, the paper's structure); one warm and one timed
    # step each, on the whole aperture or on 16 stripes spread evenly over it
    plain = {}
    if args.form == "dense" and not args.no_plain:
        prow = args.plain_rows if args.plain_rows >= 0 else (0 if N <= 316057 else 16384)
        rows = N if prow <= 0 else min(N, prow)
        if rows == N:
            ranges = [(0, N)]
        else:
            ns, h = 16, max(1, rows // 16)
            ranges = [(max(0, int((k + 0.5) * N / ns) - h // 2), max(0, int((k + 0.5) * N / ns) - h // 2) + h)
                      for k in range(ns)]
            rows = ns * h
        for conv, key in ((fzp.CONV_PARTITIONED, "partitioned"), (fzp.CONV_SINGLE, "single")):
            with fzp.Plan(**dict(params, form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP32, conv=conv)) as pb:
                def run_rows():
                    for k, (a, b) in enumerate(ranges):
                        pb.propagate_roi(a, b, U, accumulate=k > 0, stream=stream)
                run_rows()
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                run_rows()
                mb = pb.metrics(U, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                pms = e0.elapsed_time(e1)
                if parity is not None:
                    pa, pb_ = parity["rows"]
                    parity[f"rel_l2_I_bluestein_fp32_{key}"] = _rel_l2(
                        _rows_intensity(fzp, torch, pb, M, pa, pb_, stream, dev), Iref)
            rec = {"form": "bluestein", "conv": key, "dtype": "f32", "value": rows * N / (pms / 1e3) / 1e9,
                   "unit": UNIT, "ms_per_step": pms, "rows": rows,
                   "row_sample": "whole aperture" if rows == N else f"16 stripes of {rows // 16} rows spread over N"}
            if rows == N:
                rec.update(fwhm_x=mb["fwhm_x"], de_lobe=mb["de_lobe"])
            plain[key] = rec

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "strong" if sharded else "weak",
           "vs_baseline": None, "dtype": dtype,
           "data": "synthetic (procedural zone plate" + (", seeded membrane deformation)" if wl.get("deform") else ")"),
           "config": _config(args, wl, N),
           "roofline": roof, "e2e": e2e, "gpu_launches": prof["kernel_launches"], "clocks": clocks,
           "metrics_last_step": {k: m[k] for k in ("fwhm_x", "de_lobe", "mtf_half_cut")}}
    if args.form == "saczt":
        out["config"].update(exact_radii=True, padded_grid=info["fft_length"])
    if sharded:
        out["config"]["parallelism"] = f"rows split over {ws} ranks by open-sample count, one all_reduce per step"
    if plain:
        out["plain_fp32"] = plain["partitioned"]
        out["speedup_vs_plain_fp32"] = value / plain["partitioned"]["value"]
        out["plain_fp32_single"] = plain["single"]
        out["speedup_vs_plain_fp32_single"] = value / plain["single"]["value"]
    if cb is not None:
        out["cpu_baseline"] = cb
        out["parity"] = parity
    _print(out)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
