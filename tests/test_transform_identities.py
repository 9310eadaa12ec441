"""CPU checks of the two transform identities the CUDA path is built on (no GPU needed).

1. DST-I of n = M - 1 points from one real DFT of length M: with x_0 = x_M = 0 and
   y_j = sin(pi j / M) (x_j + x_{M-j}) + (x_j - x_{M-j}) / 2, Y = DFT(y) = R + i I,
   S_{2k} = -I_k, S_{2k+1} = S_{2k-1} + R_k, S_1 = R_0 / 2; two real lines packed into one
   complex DFT (the spatial H_k solves, exact form of eq. 4.4).
2. Stockham radix-8/4/2 passes: butterfly i of a pass after total radix p reads i + m M/R,
   twiddles by exp(-2 pi i m (i mod p) / (p R)) and writes (i - i mod p) R + i mod p + m p;
   natural order in and out.

Both are compared with scipy.fft, whose DST-I is (2x) the definition sum_j x_j sin(pi j k / M).
"""
import numpy as np
import pytest
import scipy.fft as sf


def stockham_fft(z):
    M = len(z)
    logM = M.bit_length() - 1
    tw = np.exp(-2j * np.pi * np.arange(M) / M)
    a = np.array(z, dtype=complex)
    s = 0
    while s < logM:
        rem = logM - s
        lr = 3 if (rem >= 5 or rem == 3) else (2 if rem in (2, 4) else 1)
        R, nb, p = 1 << lr, M >> lr, 1 << s
        out = np.empty_like(a)
        for i in range(nb):
            k = i & (p - 1)
            u = np.array([a[i + m * nb] for m in range(R)])
            u = u * tw[((np.arange(R) * k) << (logM - s - lr))]
            u = np.fft.fft(u)  # the radix-R butterfly is a DFT of length R
            j = ((i - k) << lr) + k
            out[j + np.arange(R) * p] = u
        a = out
        s += lr
    return a


def dsti_pair(va, vb):
    n = len(va)
    M = n + 1
    x = np.zeros((2, M + 1))
    x[0, 1:M] = va
    x[1, 1:M] = vb
    j = np.arange(M)
    s = np.sin(np.pi * j / M)
    y = s * (x[:, j] + x[:, M - j]) + 0.5 * (x[:, j] - x[:, M - j])
    Z = stockham_fft(y[0] + 1j * y[1])
    Zm = np.conj(Z[(-np.arange(M)) % M])
    Ya, Yb = (Z + Zm) / 2, (Z - Zm) / 2j
    out = []
    for Y in (Ya, Yb):
        R, I = Y.real[: M // 2], Y.imag[: M // 2]
        S = np.zeros(M)
        S[1::2] = np.cumsum(np.concatenate(([R[0] / 2], R[1:])))  # S_1, S_3, ...
        S[2::2] = -I[1:]                                          # S_2, S_4, ...
        out.append(S[1:])
    return out


@pytest.mark.parametrize("M", [2, 4, 8, 16, 32, 128, 256, 1024])
def test_stockham_passes_are_the_dft(M):
    z = np.random.default_rng(M).standard_normal(M) + 1j * np.random.default_rng(M + 1).standard_normal(M)
    ref = sf.fft(z)
    assert np.abs(stockham_fft(z) - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("n", [1, 3, 7, 15, 63, 255, 1023])
def test_half_length_dst1_pair(n):
    rng = np.random.default_rng(n)
    va, vb = rng.standard_normal(n), rng.standard_normal(n)
    Sa, Sb = dsti_pair(va, vb)
    for v, S in ((va, Sa), (vb, Sb)):
        ref = sf.dst(v, type=1) / 2
        assert np.abs(S - ref).max() <= 1e-13 * np.abs(ref).max() * max(1.0, np.log2(n + 1))
    if n <= 63:  # the definition itself
        k = np.arange(1, n + 1)
        Smat = np.sin(np.pi * np.outer(k, k) / (n + 1))
        assert np.abs(Sa - Smat @ va).max() <= 1e-12
