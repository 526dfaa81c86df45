"""The register-resident channel node's formulation, checked on the CPU.

For K <= 4 and q <= 16 the GPU computes each user's extrinsic channel message
without division by splitting the users into two halves (reading R11):
  * K = 2: ch2v_0(a) = sum_b mu_1(b) G(a + b), and the mirror for user 1;
  * K = 3: the prefix F_2 = mu_0 (*) mu_1 scores user 2 directly, and the
    suffix B_2(v) = sum_b mu_2(b) G(v + b) is correlated with mu_0 (user 1) and
    mu_1 (user 0);
  * K = 4: P_23 = mu_2 (*) mu_3, H_23(v) = sum_s P_23(s) G(v + s), users 0 and 1
    correlate mu_1 and mu_0 with H_23; users 2 and 3 use P_01 and H_01.
G(u) is the Gaussian score of the sum value u, computed relative to the nearest
symbol sum s* (reading R10): exp(-2 d (r + d) / sigma2) = 2^(d (k2 d + k2 r)) with
d = s* - u, r = y - (2 s* - K(q-1)) and k2 = -2 log2(e) / sigma2, which differs from exp(-(y - (2u - K(q-1)))^2 / (2 sigma2))
only by the factor exp(-r^2 / (2 sigma2)) common to every u.
Run in FP64 this must equal the oracle's trellis to rounding; run in FP32 (the
GPU's arithmetic, sums in the kernel's order) it must meet the parity bar of
1e-4 in log on every entry above 1e-4 of the maximum.  The team shape (any K,
q up to 64) uses the full prefix/suffix chain instead; its formulation is pinned
the same way in FP64, for K up to 16.
"""
import math
import os
import sys

import numpy as np
import pytest

from paper_2605_26580_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def gauss(K, q, sigma2, y, dt):
    """G(u) as the kernels form it: 2^(d (k2 d + k2 r)) with k2 = -2 log2(e) / sigma2,
    the inner sum one fused multiply-add (emulated: the FP32 product is exact in FP64)."""
    KD = K * (q - 1)
    ss = int(min(max(np.rint((y + KD) * 0.5), 0), KD))
    r = dt(y - (2 * ss - KD))
    d = (ss - np.arange(KD + 1)).astype(dt)
    k2 = dt(dt(-2.0 * math.log2(math.e)) * dt(1.0 / sigma2))
    k2r = dt(k2 * r)
    t = (k2.astype(np.float64) * d.astype(np.float64) + np.float64(k2r)).astype(dt)
    return np.exp2((d * t).astype(dt)).astype(dt)


def corr(P, X, nh, dt):
    """H(v) = sum_s P(s) X(v + s), v = 0..nh-1, accumulated over s in order."""
    H = np.zeros(nh, dtype=dt)
    for s in range(P.shape[0]):
        H = (H + P[s] * X[s:s + nh]).astype(dt)
    return H


def conv(A, B, dt):
    C = np.zeros(A.shape[0] + B.shape[0] - 1, dtype=dt)
    for i in range(A.shape[0]):
        C[i:i + B.shape[0]] = (C[i:i + B.shape[0]] + A[i] * B).astype(dt)
    return C


def split_node(K, q, sigma2, y, mu, dt):
    mu = mu.astype(dt)
    G = gauss(K, q, sigma2, y, dt)
    D = q - 1
    out = [None] * K
    if K == 1:
        out[0] = G[:q]
    elif K == 2:
        out[0] = corr(mu[1], G, q, dt)
        out[1] = corr(mu[0], G, q, dt)
    elif K == 3:
        F2 = conv(mu[0], mu[1], dt)
        out[2] = corr(F2, G, q, dt)
        B2 = corr(mu[2], G, 2 * D + 1, dt)
        out[1] = corr(mu[0], B2, q, dt)
        out[0] = corr(mu[1], B2, q, dt)
    else:
        H23 = corr(conv(mu[2], mu[3], dt), G, 2 * D + 1, dt)
        out[0] = corr(mu[1], H23, q, dt)
        out[1] = corr(mu[0], H23, q, dt)
        H01 = corr(conv(mu[0], mu[1], dt), G, 2 * D + 1, dt)
        out[2] = corr(mu[3], H01, q, dt)
        out[3] = corr(mu[2], H01, q, dt)
    o = np.stack(out).astype(np.float64)
    return np.maximum(o / o.max(axis=1, keepdims=True), 1e-12)


CASES = [(1, 16, 6.0), (2, 4, 10.0), (2, 16, 8.0), (3, 8, 12.0), (3, 16, 14.0), (4, 4, 10.0), (4, 16, 16.0),
         (4, 16, 6.0)]


@pytest.mark.parametrize("K,q,snr", CASES)
def test_split_formulation_equals_the_trellis(oracle, K, q, snr):
    m = int(math.log2(q))
    sigma2 = (q * q - 1) / 3.0 * 10 ** (-snr / 10)
    rng = np.random.default_rng(K * 31 + q)
    for _ in range(8):
        logmu = I.random_log_messages(rng, (K,), q, spread=2.5)
        sym = rng.integers(0, q, K)
        y = float((2 * sym - (q - 1)).sum() + rng.normal() * math.sqrt(sigma2))
        ref = np.exp(oracle.channel_node(K, m, sigma2, y, logmu))
        got = split_node(K, q, sigma2, y, np.exp(logmu), np.float64)
        assert np.abs(np.log(got) - np.log(ref)).max() <= 1e-9


@pytest.mark.parametrize("K,q,snr", CASES)
def test_split_in_fp32_meets_the_parity_bar(oracle, K, q, snr):
    m = int(math.log2(q))
    sigma2 = (q * q - 1) / 3.0 * 10 ** (-snr / 10)
    rng = np.random.default_rng(K * 37 + q)
    worst, underflow = 0.0, 0
    for _ in range(16):
        lc = I.random_log_messages(rng, (2, K), q, spread=3.0)
        logmu = lc.sum(axis=0)
        logmu -= logmu.max(axis=-1, keepdims=True)
        mu = np.exp(logmu).astype(np.float32)
        sym = rng.integers(0, q, K)
        y = float(np.float32((2 * sym - (q - 1)).sum() + rng.normal() * math.sqrt(sigma2)))
        ref = oracle.channel_node(K, m, sigma2, y, np.log(mu.astype(np.float64)))
        with np.errstate(invalid="ignore", divide="ignore"):
            got = np.log(split_node(K, q, sigma2, y, mu, np.float32))
        if not np.isfinite(got).all():   # all scores underflowed: the kernel's log-space fallback takes it
            underflow += 1
            continue
        mask = ref >= math.log(1e-4)
        worst = max(worst, float(np.abs(got - ref)[mask].max()))
    print("K=%d q=%d %.0f dB: FP32 split, max log err above 1e-4: %.2e (%d underflows)" % (K, q, snr, worst, underflow))
    assert underflow <= 2
    assert worst <= 1e-4


def chain_node(K, q, sigma2, y, mu):
    """Team shape (any K): prefixes F_0 = delta_0, F_{j+1} = F_j (*) mu_j; scored
    suffixes B_K = G, B_j(v) = sum_b mu_j(b) B_{j+1}(v + b); messages
    ch2v_k(a) ~ sum_s F_k(s) B_{k+1}(s + a).  Every prefix and suffix is
    rescaled to max 1, as the kernel does (a constant per array)."""
    dt = np.float64
    D = q - 1
    G = gauss(K, q, sigma2, y, dt)
    F = [np.ones(1)]
    for j in range(K - 1):
        f = conv(F[-1], mu[j].astype(dt), dt)
        F.append(f / f.max())
    B = [None] * (K + 1)
    B[K] = G / G.max()
    for j in range(K - 1, 0, -1):
        b = corr(mu[j].astype(dt), B[j + 1], j * D + 1, dt)
        B[j] = b / b.max()
    out = np.stack([corr(F[k], B[k + 1], q, dt) for k in range(K)])
    return np.maximum(out / out.max(axis=1, keepdims=True), 1e-12)


@pytest.mark.parametrize("K,q,snr", [(2, 32, 10.0), (5, 16, 12.0), (8, 4, 10.0), (4, 64, 14.0), (6, 32, 16.0),
                                     (8, 64, 14.0), (16, 4, 12.0), (1, 64, 8.0)])
def test_prefix_suffix_chain_equals_the_trellis(oracle, K, q, snr):
    m = int(math.log2(q))
    sigma2 = (q * q - 1) / 3.0 * 10 ** (-snr / 10)
    rng = np.random.default_rng(K * 41 + q)
    for _ in range(4):
        logmu = I.random_log_messages(rng, (K,), q, spread=2.5)
        sym = rng.integers(0, q, K)
        y = float((2 * sym - (q - 1)).sum() + rng.normal() * math.sqrt(sigma2))
        ref = np.exp(oracle.channel_node(K, m, sigma2, y, logmu))
        got = chain_node(K, q, sigma2, y, np.exp(logmu))
        assert np.abs(np.log(got) - np.log(ref)).max() <= 1e-9


def test_roofline_mac_count_matches_the_formulations(monkeypatch):
    """The benchmark's channel-node work per channel use (its roofline FLOP count)
    equals the multiply-adds the formulations above perform, counted as they run
    (products with the unit prefix F_0 = delta_0 are free and not counted)."""
    sys.path.insert(0, ROOT)
    import bench
    count = [0]
    mod = sys.modules[__name__]
    real_corr, real_conv = mod.corr, mod.conv

    def corr_n(P, X, nh, dt):
        if P.shape[0] > 1:
            count[0] += P.shape[0] * nh
        return real_corr(P, X, nh, dt)

    def conv_n(A, B, dt):
        if A.shape[0] > 1:
            count[0] += A.shape[0] * B.shape[0]
        return real_conv(A, B, dt)

    monkeypatch.setattr(mod, "corr", corr_n)
    monkeypatch.setattr(mod, "conv", conv_n)
    rng = np.random.default_rng(1)
    for K, q in [(2, 4), (2, 16), (3, 8), (3, 16), (4, 4), (4, 16), (5, 16), (4, 32), (8, 64), (6, 8)]:
        mu = np.exp(I.random_log_messages(rng, (K,), q, spread=1.0))
        count[0] = 0
        if K <= 4 and q <= 16:
            split_node(K, q, 10.0, 0.5, mu, np.float64)
        else:
            chain_node(K, q, 10.0, 0.5, mu)
        assert count[0] == bench.channel_macs_per_use(K, q), (K, q, count[0])
