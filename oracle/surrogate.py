"""FP64 reference for the learned surrogate (test infrastructure only).

The surrogate is a multilayer perceptron: hidden layers z_l = W_l h_{l-1} + b_l,
h_l = SiLU(z_l) = z_l sigma(z_l); linear output layer; loss = mean squared
error over the batch and all outputs.  This module computes the forward pass,
the exact gradients by back-propagation, and one AdamW step, in float64.

With ``bf16=True`` every operand of every matrix product is first rounded to
bfloat16 (round to nearest even), at the same points where the GPU kernels
round: layer inputs and weights in the forward pass, the back-propagated error
and the layer inputs / weights in the backward pass.  Sums stay in float64,
so the GPU (float32 accumulation of the same bfloat16 operands) must agree to
accumulation rounding.  With ``bf16=False`` it is the plain float64 network,
which the tests pin by central finite differences.
"""
from __future__ import annotations

import numpy as np


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def _sig(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * _sig(z)


def silu_grad(z):
    s = _sig(z)
    return s * (1.0 + z * (1.0 - s))


def forward(params, X, rnd: bool = False):
    """params: list of (W [out x in], b [out]).  Returns (Z list, H list) where
    H[0] = X and Z[-1] is the network output."""
    r = bf16 if rnd else (lambda a: a)
    H = [np.asarray(X, dtype=np.float64)]
    Z = []
    for l, (W, b) in enumerate(params):
        z = r(H[-1]) @ r(W).T + b
        Z.append(z)
        if l < len(params) - 1:
            H.append(silu(z))
    return Z, H


def loss_and_grads(params, X, Y, rnd: bool = False):
    """MSE loss mean((yhat - y)^2) and its gradients [(dW, db), ...]."""
    r = bf16 if rnd else (lambda a: a)
    Z, H = forward(params, X, rnd)
    yhat = Z[-1]
    B, n_out = yhat.shape
    loss = float(np.mean((yhat - Y) ** 2))
    G = 2.0 * (yhat - Y) / (B * n_out)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        grads[l] = (r(G).T @ r(H[l]), G.sum(axis=0))
        if l > 0:
            G = (r(G) @ r(W)) * silu_grad(Z[l - 1])
    return loss, grads


def adamw_step(params, grads, state, lr, wd, t, b1=0.9, b2=0.999, eps=1e-8):
    """Decoupled weight decay on the weights (not the biases)."""
    new = []
    for l, ((W, b), (dW, db)) in enumerate(zip(params, grads)):
        mW, vW, mb, vb = state[l]
        mW = b1 * mW + (1 - b1) * dW
        vW = b2 * vW + (1 - b2) * dW ** 2
        mb = b1 * mb + (1 - b1) * db
        vb = b2 * vb + (1 - b2) * db ** 2
        c1, c2 = 1 - b1 ** t, 1 - b2 ** t
        W = W - lr * ((mW / c1) / (np.sqrt(vW / c2) + eps) + wd * W)
        b = b - lr * (mb / c1) / (np.sqrt(vb / c2) + eps)
        state[l] = (mW, vW, mb, vb)
        new.append((W, b))
    return new


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten(vec, sizes):
    out, k = [], 0
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        W = vec[k:k + n_in * n_out].reshape(n_out, n_in)
        k += n_in * n_out
        b = vec[k:k + n_out]
        k += n_out
        out.append((np.array(W, dtype=np.float64), np.array(b, dtype=np.float64)))
    return out
