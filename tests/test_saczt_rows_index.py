"""The SA-CZT row transforms' index scheme (k_sa_rows in saczt.cu), emulated
on the CPU: radix-2 stages fused four at a time, decimation in frequency
forward (natural order in, bit-reversed out) and decimation in time inverse
(bit-reversed in, natural out), with the twiddle table e^{-2 pi i t / P},
t < P/2, and the kernel's group and twiddle indices; the three row kernels
and two transposes then equal numpy's 2-D transform, phase and inverse
applied in natural order.  No GPU: this checks the index arithmetic."""
import numpy as np
import pytest


def brev(v, bits):
    v = np.asarray(v, dtype=np.int64)
    r = np.zeros_like(v)
    for b in range(bits):
        r |= ((v >> b) & 1) << (bits - 1 - b)
    return r


def fwd(x, tw):
    """row_fft_fwd: dif_pass<R> over passes of up to four stages."""
    x = x.copy()
    P = x.size
    logP = P.bit_length() - 1
    done = 0
    while done < logP:
        R = min(4, logP - done)
        lgH = logP - 1 - done
        lsig = lgH - (R - 1)
        sig = 1 << lsig
        g = np.arange(P >> R)
        k0 = g & (sig - 1)
        base = ((g >> lsig) << (lgH + 1)) + k0
        v = [x[base + j * sig].copy() for j in range(1 << R)]
        for t in range(R):
            span = 1 << (R - 1 - t)
            tsh = logP - 1 - (lsig + R - 1 - t)
            for j in range(1 << R):
                if j & span:
                    continue
                u, w = v[j], v[j + span]
                w2 = tw[(k0 + (j & (span - 1)) * sig) << tsh]
                v[j], v[j + span] = u + w, (u - w) * w2
        for j in range(1 << R):
            x[base + j * sig] = v[j]
        done += R
    return x


def inv(x, tw):
    """row_fft_inv: dit_inv_pass<R>, conjugate twiddles, no 1/P."""
    x = x.copy()
    P = x.size
    logP = P.bit_length() - 1
    done = 0
    while done < logP:
        R = min(4, logP - done)
        lsig = done
        sig = 1 << lsig
        g = np.arange(P >> R)
        k0 = g & (sig - 1)
        base = ((g >> lsig) << (lsig + R)) + k0
        v = [x[base + j * sig].copy() for j in range(1 << R)]
        for t in range(R):
            span = 1 << t
            tsh = logP - 1 - (lsig + t)
            for j in range(1 << R):
                if j & span:
                    continue
                w2 = np.conj(tw[(k0 + (j & (span - 1)) * sig) << tsh])
                u, b = v[j], v[j + span] * w2
                v[j], v[j + span] = u + b, u - b
        for j in range(1 << R):
            x[base + j * sig] = v[j]
        done += R
    return x


def table(P):
    return np.exp(-2j * np.pi * np.arange(P // 2) / P)


@pytest.mark.parametrize("logP", [1, 2, 5, 6, 7, 9, 10, 13])
def test_forward_is_bit_reversed_fft(logP):
    P = 1 << logP
    rng = np.random.default_rng(logP)
    x = rng.standard_normal(P) + 1j * rng.standard_normal(P)
    y = fwd(x, table(P))
    X = np.fft.fft(x)
    assert np.allclose(y, X[brev(np.arange(P), logP)], atol=1e-9 * np.abs(X).max())
    z = inv(y, table(P))
    assert np.allclose(z, P * x, atol=1e-9 * P * np.abs(x).max())


def test_three_row_kernels_and_transposes():
    """MODE 0 rows, transpose, MODE 1 rows (forward, phase at the bit-reversed
    frequencies of both axes, inverse), transpose, MODE 2 rows == ifft2(fft2(T)
    H) for a phase H(fa, fb) that tells the axes apart."""
    logP = 6
    P = 1 << logP
    tw = table(P)
    rng = np.random.default_rng(3)
    T = (rng.uniform(size=(P, P)) < 0.3).astype(complex)
    f = np.fft.fftfreq(P, 1.0 / P).astype(np.int64)  # signed index of natural position
    H = np.exp(2j * np.pi * (0.013 * f[:, None] ** 2 + 0.007 * f[None, :] ** 2 + 0.001 * f[:, None] * f[None, :]))
    ref = np.fft.ifft2(np.fft.fft2(T) * H) * P * P
    G = np.stack([fwd(T[p], tw) for p in range(P)])          # G[p][b'] along the columns q
    Tt = G.T.copy()                                           # T[b'][p]
    out = np.empty_like(Tt)
    br = brev(np.arange(P), logP)
    sgn = np.where(br < P // 2, br, br - P)                   # signed frequency at a bit-reversed position
    for r in range(P):
        y = fwd(Tt[r], tw)                                    # along p: positions a'
        fb = sgn[r]
        fa = sgn
        y = y * np.exp(2j * np.pi * (0.013 * fa ** 2 + 0.007 * fb ** 2 + 0.001 * fa * fb))
        out[r] = inv(y, tw)                                   # natural p
    G2 = out.T.copy()                                         # G[p][b']
    U = np.stack([inv(G2[p], tw) for p in range(P)])          # natural q
    assert np.allclose(U, ref, atol=1e-9 * np.abs(ref).max())
