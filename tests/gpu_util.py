"""Helpers shared by the GPU tests (no method arithmetic here)."""
import numpy as np


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def run_plan(fzp, torch, plan, M, j0, j1, accumulate_into=None):
    """Propagate rows [j0, j1) through the C ABI; returns (U, I) as numpy."""
    dev = torch.device("cuda:0")
    U = accumulate_into if accumulate_into is not None else torch.empty((M, M), dtype=torch.complex128, device=dev)
    plan.propagate_roi(j0, j1, U, accumulate=accumulate_into is not None)
    I = torch.empty((M, M), dtype=torch.float64, device=dev)
    plan.intensity(U, I)
    torch.cuda.synchronize()
    return U.cpu().numpy(), I.cpu().numpy()
