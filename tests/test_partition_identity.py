"""CPU checks of the arithmetic identities the partitioned Bluestein row pass
relies on (no GPU, no library call): numpy FFTs stand in for the kernel's.

1. The row convolution (y * h)[m], m < M (Sec. 2.6), equals the inverse
   4096-point transform of sum_s FFT(y_s) FFT(g_s), y_s the s-th block of S
   columns and g_s[q] = h_{q - i_s} (q < M), h_{q - 4096 - i_s} (q > 4096 - S),
   when S + M - 1 <= 4096; with one block more than that bound allows, lags
   alias and the identity fails.
2. The block size rule of fzp_params.conv, S = 256 min(15, floor((4097 - M)/256)),
   meets the bound for every allowed M and is a multiple of 256.
3. The three-pass distribution of the 4096-point transform (thread t holding
   elements t + 256 r; 16-point DFTs over r, over b with t = a + 16 b, over a;
   twiddles e^{-2 pi i t k0/4096} and e^{-2 pi i a c/256}; transposes through
   the padded shared-memory layouts) is the DFT, with its output at t + 256 d.
"""
import numpy as np
import pytest

P = 4096


def block_size(M):
    return 256 * min(15, (4097 - M) // 256)


def partitioned(y, h, M, S):
    N = len(y)
    acc = np.zeros(P, complex)
    q = np.arange(P)
    for s in range((N + S - 1) // S):
        i_s = s * S
        u = np.zeros(P, complex)
        blk = y[i_s:i_s + S]
        u[:len(blk)] = blk
        g = np.zeros(P, complex)
        lo = q < M
        g[lo] = h(q[lo] - i_s)
        hi = q > P - S
        g[hi] = h(q[hi] - P - i_s)
        acc += np.fft.fft(u) * np.fft.fft(g)
    return np.fft.ifft(acc)[:M]


@pytest.mark.parametrize("M", [64, 128, 256, 512, 1024])
def test_block_size_rule(M):
    S = block_size(M)
    assert S % 256 == 0 and S + M - 1 <= P and S >= 3072


@pytest.mark.parametrize("M,N", [(512, 10001), (1024, 7000), (64, 4000), (256, 3000)])
def test_partitioned_convolution_identity(M, N):
    rng = np.random.default_rng(M + N)
    delta = 0.37 / N
    y = (rng.random(N) < 0.5) * np.exp(2j * np.pi * rng.random(N))

    def h(k):
        return np.exp(1j * np.pi * delta * np.asarray(k, float) ** 2)

    i = np.arange(N)
    ref = np.array([np.sum(y * h(m - i)) for m in range(M)])
    out = partitioned(y, h, M, block_size(M))
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref)) * N ** 0.5
    if block_size(M) < 15 * 256:  # one block more than the bound allows
        bad = partitioned(y, h, M, block_size(M) + 256)
        assert np.max(np.abs(bad - ref)) > 1e-3 * np.max(np.abs(ref))


def three_pass(x):
    """The kernel's distribution, written with index arrays."""
    t = np.arange(256)
    v = x.reshape(16, 256).T                      # v[t, r] = x[t + 256 r]
    A = np.fft.fft(v, axis=1)                     # over r -> k0
    A *= np.exp(-2j * np.pi * np.outer(t, np.arange(16)) / P)
    b0 = np.zeros(256 * 17, complex)
    b0[(t[:, None] * 17 + np.arange(16)[None, :]).ravel()] = A.ravel()
    a, k0 = t & 15, t >> 4                        # pass B thread (a, k0)
    B = b0[(a[:, None] + 16 * np.arange(16)[None, :]) * 17 + k0[:, None]]
    B = np.fft.fft(B, axis=1)                     # over b -> c
    B *= np.exp(-2j * np.pi * np.outer(a, np.arange(16)) / 256)
    b1 = np.zeros(16 * 273, complex)
    b1[(k0[:, None] * 273 + np.arange(16)[None, :] * 17 + a[:, None]).ravel()] = B.ravel()
    k0c, c = t & 15, t >> 4                       # pass C thread (k0, c)
    Cc = b1[k0c[:, None] * 273 + c[:, None] * 17 + np.arange(16)[None, :]]
    return np.fft.fft(Cc, axis=1)                 # [t, d] = X[t + 256 d]


def test_three_pass_distribution_is_the_dft():
    rng = np.random.default_rng(7)
    x = rng.standard_normal(P) + 1j * rng.standard_normal(P)
    X = three_pass(x)
    ref = np.fft.fft(x)
    assert np.max(np.abs(X.T.ravel() - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_shared_memory_layouts_are_conflict_free():
    """64-bit accesses of a half-warp (16 threads) touch 16 distinct bank pairs
    in every transpose store and load (bank of 8-byte word w: 2 w mod 32)."""
    for k in range(16):                           # pass A store: thread t, word t*17 + k
        w = np.arange(16) * 17 + k
        assert len(set((2 * w) % 32)) == 16
    for half in range(16):
        a = np.arange(16)
        for b in range(16):                       # pass B load: (a + 16 b) * 17 + k0
            assert len(set((2 * ((a + 16 * b) * 17 + half)) % 32)) == 16
        for c in range(16):                       # pass B store: k0 * 273 + c * 17 + a
            assert len(set((2 * (half * 273 + c * 17 + a)) % 32)) == 16
        k0 = np.arange(16)
        for aa in range(16):                      # pass C load: k0 * 273 + c * 17 + a
            assert len(set((2 * (k0 * 273 + half * 17 + aa)) % 32)) == 16
