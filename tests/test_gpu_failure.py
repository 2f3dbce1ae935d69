"""Failure detection without a GPU fault: a bounded device wait that runs out
is reported to the host as FZP_E_TIMEOUT, and the context keeps working."""
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
