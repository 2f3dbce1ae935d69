"""Failure detection without a GPU fault: a bounded device wait that runs out
is reported to the host as FZP_E_TIMEOUT, and the context keeps working; an
out-of-memory error on the row intermediate (injected on the host) halves the
chunk until it fits, or ends in FZP_E_OOM below 256 rows."""
import numpy as np
import pytest

from gpu_util import rel_l2, run_plan

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


def test_expired_wait_is_reported_and_context_survives(env):
    fzp, torch, O = env
    import time
    t0 = time.perf_counter()
    with pytest.raises(fzp.FzpError) as e:
        fzp.selftest_wait_timeout(50000)  # 50 ms, a barrier nothing completes
    dt = time.perf_counter() - t0
    assert e.value.status == fzp.FZP_E_TIMEOUT
    assert 0.04 < dt < 5.0
    with pytest.raises(fzp.FzpError) as e2:
        fzp.selftest_wait_timeout(0)
    assert e2.value.status == fzp.FZP_E_INVALID
    # the context still runs the propagation correctly
    g = O.Geometry(D=1e-3, f=5e-3, lam=632.8e-9, M=128, p=0.4e-6)
    for form, prec in [(fzp.FORM_DENSE, fzp.PREC_SPLIT_BF16), (fzp.FORM_BLUESTEIN, fzp.PREC_FP32)]:
        with fzp.Plan(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, dx=g.dx, N=g.N, form=form, precision=prec) as plan:
            _, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
            assert rel_l2(I, np.abs(O.field_czt(g)) ** 2) <= 1e-4
            U = torch.empty((g.M, g.M), dtype=torch.complex128, device="cuda")
            plan.propagate_roi(0, g.N, U)
            plan.metrics(U)  # reads the plan's error word: clean


def test_workspace_halves_on_allocation_failure(env, monkeypatch):
    """Config 1 (N = 5057, ROI 256^2): the row intermediate of one chunk is
    512 x 5120 x 4 B = 10.5 MB; with requests above 3 MB failing, the plan
    halves the chunk twice (1280 rows, four chunks) and the field still
    matches the oracle in both forms.  Below one 256-row chunk the plan fails
    with FZP_E_OOM and leaves the context usable."""
    fzp, torch, O = env
    g = O.Geometry(D=4e-3, f=20e-3, lam=632.8e-9, M=256, p=0.2e-6)
    Iref = np.abs(O.field_czt(g)) ** 2
    kw = dict(D=g.D, f=g.f, lam=g.lam, M=g.M, pitch=g.p, dx=g.dx, N=g.N)
    with fzp.Plan(form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP32, **kw) as plan:
        assert plan.info["chunk_rows"] == 5120
    monkeypatch.setenv("FZP_FAULT_ALLOC_LIMIT", str(3_000_000))
    for form, prec in [(fzp.FORM_BLUESTEIN, fzp.PREC_FP32), (fzp.FORM_DENSE, fzp.PREC_SPLIT_BF16)]:
        with fzp.Plan(form=form, precision=prec, **kw) as plan:
            assert plan.info["chunk_rows"] == 1280, plan.info["chunk_rows"]
            _, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
            assert rel_l2(I, Iref) <= 1e-4, (form, rel_l2(I, Iref))
    monkeypatch.setenv("FZP_FAULT_ALLOC_LIMIT", str(100_000))
    with pytest.raises(fzp.FzpError) as e:
        fzp.Plan(form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP32, **kw)
    assert e.value.status == fzp.FZP_E_OOM
    monkeypatch.delenv("FZP_FAULT_ALLOC_LIMIT")
    with fzp.Plan(form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_FP32, **kw) as plan:
        _, I = run_plan(fzp, torch, plan, g.M, 0, g.N)
        assert rel_l2(I, Iref) <= 1e-4
