"""Learned surrogate: GPU training kernels against the FP64 oracle, and a
trained network checked against the plain CZT on held-out membranes."""
import math
import time

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
    import paper_2609_01978_gb300 as fzp
    from oracle import surrogate as S
    return fzp, torch, S


@pytest.mark.parametrize("sizes,B", [((8, 64, 64, 64, 40), 32), ((8, 512, 512, 512, 4114), 256)])
def test_gradients_match_oracle(env, sizes, B):
    fzp, torch, S = env
    net = fzp.SurrogateNet(n_in=sizes[0], hidden=sizes[1], layers=len(sizes) - 2, n_out=sizes[-1], max_batch=B, seed=7)
    rng = np.random.default_rng(1)
    X = rng.normal(size=(B, sizes[0])).astype(np.float32)
    Y = rng.normal(size=(B, sizes[-1])).astype(np.float32)
    dev = torch.device("cuda:0")
    g = torch.empty(net.param_count, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    net.grad(torch.from_numpy(X).to(dev), torch.from_numpy(Y).to(dev), g, loss)
    torch.cuda.synchronize()
    params = S.unflatten(net.get_params().astype(np.float64), list(sizes))
    lref, gref = S.loss_and_grads(params, X.astype(np.float64), Y.astype(np.float64), rnd=True)
    assert abs(loss.item() / lref - 1) < 1e-5
    gv = g.cpu().numpy().astype(np.float64)
    k = 0
    for (dW, db) in gref:
        for ref in (dW.ravel(), db):
            got = gv[k:k + ref.size]
            k += ref.size
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-3
    # one AdamW step: the optimiser arithmetic against the oracle's, applied to
    # the GPU's own (deterministic) gradient of the same batch
    p0 = net.get_params().astype(np.float64)
    net.train_step(torch.from_numpy(X).to(dev), torch.from_numpy(Y).to(dev), 1e-3, 1e-2)
    torch.cuda.synchronize()
    p1 = net.get_params().astype(np.float64)
    ggpu = S.unflatten(gv, list(sizes))
    state = [tuple(np.zeros_like(a) for a in (W, W, b, b)) for W, b in params]
    pref = S.flatten(S.adamw_step(params, ggpu, state, lr=1e-3, wd=1e-2, t=1))
    assert np.max(np.abs(p1 - pref)) < 1e-6
    net.close()


def test_trained_surrogate_judged_by_czt(env):
    """Train on 1536 membranes propagated by the library's dense membrane passes
    (D = 2 mm, f/# = 5, lambda 450-650 nm, 128^2 ROI), evaluate 128 held-out
    membranes against the plain CZT (FP32 Bluestein form, the judge), and
    compare with the method without a learned part: the undeformed zone
    plate's PSF at the same wavelength, and the mean training PSF.  The dense
    targets of the held-out set equal the plain CZT's (PSF rel L2 <= 1e-4)."""
    fzp, torch, S = env
    import fzp_inputs
    from paper_2609_01978_gb300 import surrogate as SG
    D = 2e-3
    ntr = 1536
    mem, X = fzp_inputs.surrogate_draws(ntr + 128, seed=11, D=D)
    t0 = time.perf_counter()
    Y, psf, _ = SG.generate(mem[:ntr])
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    Yte, T, ideal = SG.generate(mem[ntr:], form=SG.PLAIN)
    t_plain = (time.perf_counter() - t0) / 128
    _, Tdense, _ = SG.generate(mem[ntr:])
    dense_vs_plain = np.array([np.linalg.norm(Tdense[k] - T[k]) / np.linalg.norm(T[k]) for k in range(len(T))])
    Xtr, Ytr, Xte = X[:ntr], Y, X[ntr:]
    model = SG.train(Xtr, Ytr, D, steps=1500, log=[])
    pred = model.predict(Xte)
    P = SG.psf_from_targets(pred, ideal)
    err = np.array([np.linalg.norm(P[k] - T[k]) / np.linalg.norm(T[k]) for k in range(len(T))])
    flat_mem = [fzp_inputs.Membrane(0.0, m.period, m.theta, 0.0, [(a, b, c, 0.0, w) for a, b, c, _, w in m.ridges],
                                    m.lam, m.D) for m in mem[ntr:]]
    _, flat, _ = SG.generate(flat_mem, form=SG.PLAIN)
    err_flat = np.array([np.linalg.norm(flat[k] - T[k]) / np.linalg.norm(T[k]) for k in range(len(T))])
    mean_psf = psf.mean(0)
    err_mean = np.array([np.linalg.norm(mean_psf - T[k]) / np.linalg.norm(T[k]) for k in range(len(T))])
    de_err = np.abs(pred[:, 4097] - Yte[:, 4097])
    # throughput: surrogate inference vs the propagation it replaces
    dev = torch.device("cuda:0")
    xb = torch.from_numpy(SG.encode(np.repeat(Xte, 2, 0), D).astype(np.float32)).to(dev)
    yb = torch.empty((xb.shape[0], Y.shape[1]), dtype=torch.float32, device=dev)
    model.net.infer(xb, yb)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(10):
        model.net.infer(xb, yb)
    torch.cuda.synchronize()
    per_inst_sur = (time.perf_counter() - t1) / (10 * xb.shape[0])
    per_inst_dense = t_gen / ntr
    print(f"held-out PSF rel L2 (judge: plain CZT): surrogate median {np.median(err):.3f} mean {err.mean():.3f}; "
          f"flat-FZP baseline {np.median(err_flat):.3f}; mean-PSF baseline {np.median(err_mean):.3f}; "
          f"DE abs err median {np.median(de_err):.2e}; dense vs plain targets max {dense_vs_plain.max():.2e}; "
          f"per instance: surrogate {per_inst_sur * 1e6:.1f} us, dense {per_inst_dense * 1e3:.2f} ms, "
          f"plain CZT {t_plain * 1e3:.2f} ms")
    assert dense_vs_plain.max() <= 1e-4
    assert np.median(err) < 0.5 * np.median(err_flat)
    assert np.median(err) < 0.5 * np.median(err_mean)
    assert per_inst_dense / per_inst_sur > 10
