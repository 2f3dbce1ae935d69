"""Learned surrogate of the propagation: data, training and evaluation.

Training data are PSFs that this library's propagation computes for deformed
membranes (a ``Batch`` per chunk, one CUDA graph: by default the dense
tensor-core form's membrane passes; the plain FP32 Bluestein CZT judges the
held-out set), with the metric extractor's FWHM, diffraction efficiency and
16 MTF samples.  The intensity and the Strehl denominator come from the
library (fzp_batch_intensity; peak / Strehl).  The
network (``SurrogateNet``: hand-written BF16 tensor-core training kernels) maps
the 8-vector (A/lambda, log10 period, theta, taper, three ridge heights /
lambda, lambda) to 4114 outputs: log10(I / I_ideal + 1e-6) on the central 64^2
of a 128^2 ROI at pitch lambda f/# / 8 (I_ideal = (pi R^2/(lambda f))^2, the
Strehl denominator of Fig. 18), then FWHM, DE and the MTF samples.  The
propagation stays the reference: held-out predictions are compared with what it
computes.
"""
from __future__ import annotations

import math

import numpy as np

from . import FORM_BLUESTEIN, FORM_DENSE, PREC_FP32, PREC_SPLIT_BF16, Batch, SurrogateNet, make_deform

ROI = 128
CROP = 64
EPS = 1e-6


def _problem(m, fnum: float, form: int, precision: int, cluster: int):
    f = fnum * m.D
    return dict(D=m.D, f=f, lam=m.lam, M=ROI, pitch=m.lam * fnum / 8, form=form, precision=precision,
                cluster=cluster, deform=make_deform(m.amp, m.period, m.theta, m.taper, m.ridges))


PLAIN = dict(form=FORM_BLUESTEIN, precision=PREC_FP32, cluster=0)  # the plain CZT: judge of the error
DENSE = dict(form=FORM_DENSE, precision=PREC_SPLIT_BF16, cluster=1)  # fastest at ROI 128^2 (measured)


def generate(membranes, fnum: float = 5.0, chunk: int = 128, torch=None, form: dict = DENSE):
    """Propagate every membrane; returns (Y[n, 4114] raw targets, psf[n, 64, 64],
    ideal[n]: each instance's Strehl denominator)."""
    import torch as _t
    torch = torch or _t
    dev = torch.device("cuda")
    Y = np.zeros((len(membranes), CROP * CROP + 18), dtype=np.float64)
    psf = np.zeros((len(membranes), CROP, CROP))
    ideals = np.zeros(len(membranes))
    lo = (ROI - CROP) // 2
    for s in range(0, len(membranes), chunk):
        ms = membranes[s:s + chunk]
        b = Batch([_problem(m, fnum, **form) for m in ms])
        fields = [torch.empty((ROI, ROI), dtype=torch.complex128, device=dev) for _ in ms]
        inten = torch.empty((ROI, ROI), dtype=torch.float64, device=dev)
        b.propagate(fields)
        torch.cuda.synchronize()
        for k, (m, U) in enumerate(zip(ms, fields)):
            met = b.metrics(k, U)
            b.intensity(k, U, inten)
            torch.cuda.synchronize()
            I = inten[lo:lo + CROP, lo:lo + CROP].cpu().numpy()
            ideal = met["peak"] / met["strehl"]  # (pi R^2 / (lambda f))^2, the Strehl denominator
            psf[s + k] = I
            Y[s + k, :CROP * CROP] = np.log10(I / ideal + EPS).ravel()
            Y[s + k, CROP * CROP] = met["fwhm_x"] / (m.lam * fnum)  # in units of lambda f/#
            Y[s + k, CROP * CROP + 1] = met["de_lobe"]
            Y[s + k, CROP * CROP + 2:] = met["mtf16"]
            ideals[s + k] = ideal
        b.close()
    return Y, psf, ideals


def encode(X: np.ndarray, D: float) -> np.ndarray:
    """Raw 8-vector -> network input in [-1, 1] (ranges of fzp_inputs.surrogate_draws)."""
    scale = D / 0.2
    lo, hi = math.log10(1e-3 * scale), math.log10(20e-3 * scale)
    Z = np.empty_like(X, dtype=np.float64)
    Z[:, 0] = X[:, 0] * 8 - 1
    Z[:, 1] = (X[:, 1] - (lo + hi) / 2) / ((hi - lo) / 2)
    Z[:, 2] = X[:, 2] / math.pi * 2 - 1
    Z[:, 3] = X[:, 3] * 2 - 1
    Z[:, 4:7] = X[:, 4:7] * 16 - 1
    Z[:, 7] = (X[:, 7] - 550e-9) / 100e-9
    return Z


class Trained:
    """A trained network with its output standardisation."""

    def __init__(self, net: SurrogateNet, mean: np.ndarray, std: np.ndarray, D: float):
        self.net, self.mean, self.std, self.D = net, mean, std, D

    def predict(self, X: np.ndarray, torch=None) -> np.ndarray:
        import torch as _t
        torch = torch or _t
        dev = torch.device("cuda")
        out = np.zeros((X.shape[0], self.net.n_out))
        for s in range(0, X.shape[0], self.net.max_batch):
            x = torch.from_numpy(encode(X[s:s + self.net.max_batch], self.D).astype(np.float32)).to(dev)
            y = torch.empty((x.shape[0], self.net.n_out), dtype=torch.float32, device=dev)
            self.net.infer(x, y)
            torch.cuda.synchronize()
            out[s:s + x.shape[0]] = y.cpu().numpy()
        return out * self.std + self.mean


def train(X: np.ndarray, Y: np.ndarray, D: float, steps: int = 2000, batch: int = 256, lr: float = 1e-3,
          weight_decay: float = 1e-4, seed: int = 0, hidden: int = 512, layers: int = 3, torch=None, log=None):
    import torch as _t
    torch = torch or _t
    dev = torch.device("cuda")
    mean, std = Y.mean(0), Y.std(0) + 1e-6
    xs = torch.from_numpy(encode(X, D).astype(np.float32)).to(dev)
    ys = torch.from_numpy(((Y - mean) / std).astype(np.float32)).to(dev)
    net = SurrogateNet(n_in=X.shape[1], hidden=hidden, layers=layers, n_out=Y.shape[1], max_batch=batch, seed=seed)
    rng = np.random.default_rng(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    n = X.shape[0]
    for t in range(steps):
        idx = torch.from_numpy(rng.choice(n, size=batch, replace=n < batch)).to(dev)
        cur = lr * 0.5 * (1 + math.cos(math.pi * t / steps))
        net.train_step(xs[idx].contiguous(), ys[idx].contiguous(), cur, weight_decay, loss_out=loss)
        if log is not None and (t % 200 == 0 or t == steps - 1):
            torch.cuda.synchronize()
            log.append((t, float(loss.item())))
    torch.cuda.synchronize()
    return Trained(net, mean, std, D)


def psf_from_targets(Y: np.ndarray, ideal: np.ndarray) -> np.ndarray:
    """PSFs from predicted targets; ideal[k] is instance k's Strehl denominator
    (the ``ideal`` returned by ``generate``)."""
    out = np.zeros((Y.shape[0], CROP, CROP))
    for k in range(Y.shape[0]):
        out[k] = (10.0 ** Y[k, :CROP * CROP].reshape(CROP, CROP) - EPS) * ideal[k]
    return out
