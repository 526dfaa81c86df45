"""The tensor-core channel node's formulation, checked in FP64 on the CPU.

The GPU variant computes the channel node (kernel (a)) as a correlation in the
frequency domain of the symbol-sum alphabet.  This test runs the same recipe in
FP64 numpy, step by step as the kernel takes it, and compares it with the
oracle's trellis (an exact sum-product over the symbol sums):
  * DFT length L = the first multiple of 16 >= K(q-1)+1, so the circular
    correlation equals the linear one on a = 0..q-1;
  * spectra folded onto frequencies 0..L/2 (real inputs): pair 0 holds the real DC
    and Nyquist terms, pair p >= 1 the real and imaginary parts of frequency p;
  * the Gaussian score transformed over a window of W = min(L, 128) sums that
    starts at u_lo, and rotated back by e^{-2 pi i p u_lo / L};
  * every spectrum scaled to DC 1, leave-one-out X_k = G^ conj(prod_{j != k} mu^_j),
    inverse over the folded spectrum (weights 1, (-1)^a, 2 cos, -2 sin).
In exact arithmetic this is the trellis; in FP64 the two agree to rounding
(the window drops only sums far below the message floor at these noise levels).
"""
import math

import numpy as np
import pytest

from paper_2605_26580_gb300 import inputs as I


def _forward(n, x, L):
    p = n // 2
    if p == 0:
        return np.where(n % 2 == 1, np.where(x % 2 == 1, -1.0, 1.0), 1.0)
    th = 2.0 * np.pi * ((p * x) % L) / L
    return np.where(n % 2 == 1, -np.sin(th), np.cos(th))


def _inverse(n, a, L):
    p = n // 2
    if p == 0:
        return np.where(n % 2 == 1, np.where(a % 2 == 1, -1.0, 1.0), 1.0)
    th = 2.0 * np.pi * ((p * a) % L) / L
    return np.where(n % 2 == 1, -2.0 * np.sin(th), 2.0 * np.cos(th))


def dft_channel(K, q, sigma2, y, mu):
    """ch2v [K, q] (max 1) of one channel use from the users' messages mu [K, q]."""
    U = K * (q - 1) + 1
    L = (U + 15) // 16 * 16
    W = min(L, 128)
    KD = K * (q - 1)
    ss = int(min(max(np.rint((y + KD) * 0.5), 0), KD))
    r = y - (2 * ss - KD)
    u_lo = min(max(ss - W // 2, 0), max(U - W, 0))
    u = u_lo + np.arange(W)
    d = ss - u
    g = np.where(u < U, np.exp(-2.0 * d * (r + d) / sigma2), 0.0)
    Fm = np.array([[_forward(n, x, L) for x in range(max(q, W))] for n in range(L)], dtype=np.float64)
    spec = np.stack([Fm[:, :q] @ mu[j] for j in range(K)] + [Fm[:, :W] @ g])   # [K+1, L]
    spec /= spec[:, :1]                                                            # DC 1
    P = L // 2
    X = np.zeros((K, L))
    # pair 0: DC (1 after scaling) and Nyquist, both real; the window's Nyquist term turns by (-1)^u_lo
    nyq_g = spec[K, 1] * (-1.0 if u_lo % 2 else 1.0)
    for k in range(K):
        X[k, 0] = 1.0
        X[k, 1] = nyq_g * np.prod([spec[j, 1] for j in range(K) if j != k])
    for p in range(1, P):
        mhat = spec[:K, 2 * p] + 1j * spec[:K, 2 * p + 1]
        th = 2.0 * np.pi * ((p * u_lo) % L) / L
        ghat = (spec[K, 2 * p] + 1j * spec[K, 2 * p + 1]) * (np.cos(th) - 1j * np.sin(th))
        for k in range(K):
            e = np.prod([mhat[j] for j in range(K) if j != k])
            x = ghat * np.conj(e)
            X[k, 2 * p], X[k, 2 * p + 1] = x.real, x.imag
    Binv = np.array([[_inverse(n, a, L) for n in range(L)] for a in range(q)])
    out = X @ Binv.T                                                               # [K, q]
    out /= out.max(axis=1, keepdims=True)
    return np.maximum(out, 1e-12)


@pytest.mark.parametrize("K,q,snr", [(2, 16, 8.0), (3, 16, 14.0), (4, 16, 10.0), (2, 64, 12.0), (4, 64, 14.0),
                                     (8, 16, 12.0), (5, 32, 16.0), (3, 32, 6.0)])
def test_dft_formulation_equals_the_trellis(oracle, K, q, snr):
    O = oracle
    m = int(math.log2(q))
    Es = (q * q - 1) / 3.0
    sigma2 = Es * 10 ** (-snr / 10)
    rng = np.random.default_rng(K * 100 + q)
    worst = 0.0
    for trial in range(6):
        logmu = I.random_log_messages(rng, (K,), q, spread=2.5)
        mu = np.exp(logmu)
        sym = rng.integers(0, q, K)
        y = float((2 * sym - (q - 1)).sum() + rng.normal() * math.sqrt(sigma2))
        ref = np.exp(O.channel_node(K, m, sigma2, y, logmu))
        got = dft_channel(K, q, sigma2, y, mu)
        ref = ref / ref.max(axis=1, keepdims=True)
        worst = max(worst, float(np.abs(got - ref).max()))
    print("K=%d q=%d %.0f dB: max |DFT - trellis| = %.2e" % (K, q, snr, worst))
    assert worst <= 1e-9


def test_dft_formulation_window_offset_and_nyquist(oracle):
    """Observations at both ends of the sum range put the window at its first and
    last offsets (u_lo = 0 and U - W) and give odd offsets, which exercises the
    rotation and the Nyquist sign."""
    O = oracle
    K, q = 4, 64
    sigma2 = 1365.0 * 10 ** (-1.2)
    rng = np.random.default_rng(11)
    for y in (-250.0, -180.5, 0.3, 181.7, 249.0):
        logmu = I.random_log_messages(rng, (K,), q, spread=2.0)
        ref = np.exp(O.channel_node(K, 6, sigma2, y, logmu))
        ref = ref / ref.max(axis=1, keepdims=True)
        got = dft_channel(K, q, sigma2, y, np.exp(logmu))
        assert np.abs(got - ref).max() <= 1e-9, y
