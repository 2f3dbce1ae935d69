"""Pins of the FP64 surrogate reference (oracle/surrogate.py)."""
import numpy as np
import pytest

from oracle import surrogate as S


def _tiny(seed=0, sizes=(3, 5, 4, 2)):
    rng = np.random.default_rng(seed)
    params = [(rng.normal(0, 0.7, (o, i)), rng.normal(0, 0.2, o)) for i, o in zip(sizes[:-1], sizes[1:])]
    X = rng.normal(size=(4, sizes[0]))
    Y = rng.normal(size=(4, sizes[-1]))
    return list(sizes), params, X, Y


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-8, 8, 20000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.bf16(x), ref)


def test_gradients_match_central_differences():
    sizes, params, X, Y = _tiny()
    _, grads = S.loss_and_grads(params, X, Y)
    g = S.flatten(grads)
    v = S.flatten(params)
    h = 1e-6
    fd = np.zeros_like(v)
    for k in range(len(v)):
        vp, vm = v.copy(), v.copy()
        vp[k] += h
        vm[k] -= h
        fd[k] = (S.loss_and_grads(S.unflatten(vp, sizes), X, Y)[0] - S.loss_and_grads(S.unflatten(vm, sizes), X, Y)[0]) / (2 * h)
    assert np.max(np.abs(g - fd)) / np.max(np.abs(fd)) < 1e-6


def test_silu_and_its_derivative():
    z = np.linspace(-8, 8, 1001)
    assert np.allclose(S.silu(z), z / (1 + np.exp(-z)), rtol=0, atol=1e-15)
    h = 1e-6
    assert np.max(np.abs(S.silu_grad(z) - (S.silu(z + h) - S.silu(z - h)) / (2 * h))) < 1e-8


def test_adamw_matches_torch():
    torch = pytest.importorskip("torch")
    sizes, params, X, Y = _tiny(seed=3)
    tp = [torch.nn.Parameter(torch.tensor(a)) for W, b in params for a in (W, b)]
    opt = torch.optim.AdamW([{"params": tp[0::2], "weight_decay": 0.01}, {"params": tp[1::2], "weight_decay": 0.0}],
                            lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    state = [tuple(np.zeros_like(a) for a in (W, W, b, b)) for W, b in params]
    p = params
    for t in range(1, 4):
        _, grads = S.loss_and_grads(p, X, Y)
        for k, (dW, db) in enumerate(grads):
            tp[2 * k].grad = torch.tensor(dW)
            tp[2 * k + 1].grad = torch.tensor(db)
        opt.step()
        p = S.adamw_step(p, grads, state, lr=1e-2, wd=0.01, t=t)
    for k, (W, b) in enumerate(p):
        assert np.allclose(W, tp[2 * k].detach().numpy(), rtol=1e-12, atol=1e-14)
        assert np.allclose(b, tp[2 * k + 1].detach().numpy(), rtol=1e-12, atol=1e-14)
