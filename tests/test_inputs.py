"""The seeded input generators (fzp_inputs): the draws follow the ranges of
the batched-membrane and surrogate configurations and are reproducible."""
import math

import numpy as np

import fzp_inputs as FI


def test_batch_draws_ranges_and_reproducibility():
    a = FI.batch_draws(256, seed=0)
    b = FI.batch_draws(256, seed=0)
    c = FI.batch_draws(256, seed=1)
    assert len(a) == 256
    assert all(x == y for x, y in zip(a, b))
    assert any(x != y for x, y in zip(a, c))
    counts = np.bincount([len(m.ridges) for m in a], minlength=4)
    assert len(counts) == 4 and np.all(counts > 0)  # 0 to 3 ridges, each present
    for m in a:
        assert 0.05 <= m.D <= 0.30
        assert m.lam in (450e-9, 550e-9, 650e-9)
        assert 0 <= m.amp <= m.lam / 4
        assert 1e-3 <= m.period <= 20e-3
        assert 0 <= m.theta < math.pi and 0 <= m.taper <= 1
        for (px, py, alpha, h, w) in m.ridges:
            assert math.hypot(px, py) <= m.D / 2  # crease line through a point of the disc
            assert 0 <= alpha < math.pi and 0 <= h <= m.lam / 8 and 0.5e-3 <= w <= 5e-3
    # wavelengths drawn from all three lines; diameters spread over the range
    assert {m.lam for m in a} == {450e-9, 550e-9, 650e-9}
    Ds = np.array([m.D for m in a])
    assert Ds.min() < 0.07 and Ds.max() > 0.28


def test_surrogate_draws_vector_matches_membranes():
    D = 2e-3
    mem, X = FI.surrogate_draws(200, seed=11, D=D)
    assert X.shape == (200, 8)
    mem2, X2 = FI.surrogate_draws(200, seed=11, D=D)
    assert np.array_equal(X, X2)
    scale = D / 0.2
    for m, x in zip(mem, X):
        assert math.isclose(x[0], m.amp / m.lam, rel_tol=1e-12) and 0 <= x[0] <= 0.25
        assert math.isclose(10 ** x[1], m.period, rel_tol=1e-12)
        assert 1e-3 * scale <= m.period <= 20e-3 * scale
        assert x[2] == m.theta and x[3] == m.taper and x[7] == m.lam
        assert 450e-9 <= m.lam <= 650e-9
        assert len(m.ridges) == 3
        for q, (px, py, alpha, h, w) in enumerate(m.ridges):
            assert math.isclose(x[4 + q], h / m.lam, rel_tol=1e-12) and 0 <= x[4 + q] <= 0.125
            # only the heights vary across the set; the geometry is fixed
            assert (px, py, alpha, w) == mem[0].ridges[q][:3] + (mem[0].ridges[q][4],)
