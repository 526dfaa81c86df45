"""The tensor-core channel node's rounding, modelled on the CPU.

`test_dft_channel_math.py` shows that the DFT formulation equals the trellis in
FP64.  This test runs the same recipe with the arithmetic of the GPU kernel:
  * mu_j (FP32, max 1) and the Gaussian window (FP32, as 2^(d (k2 d + k2 r))) rounded to one FP16
    term each;
  * the forward and inverse DFT matrices as the library's own FP16 hi + lo tables
    (`jbp_dft_tables`);
  * forward products A B_hi + A B_lo and inverse products X_hi B_hi + X_lo B_hi +
    X_hi B_lo, each product of two FP16 values exact, the sums rounded to FP32
    (tensor-core accumulation; its own rounding, about 2^-24 of the sum, is far
    below the FP16 terms and is not modelled order by order);
  * DC scaling, window rotation by FP32 twiddles and the leave-one-out products in
    FP32; X_k split into FP16 hi + lo;
  * a row whose accumulated peak is below 2^-12 L goes to the trellis (not
    compared here).
The modelled error against the FP64 oracle must stay inside the bound the
library states for the DFT node, (K+2) 2^-9 + K 2^-12 of each message's maximum,
and is of the size measured on the GPU (a few 1e-4): the error is the designed
FP16 quantisation, nothing else.
"""
import math

import numpy as np
import pytest

from paper_2605_26580_gb300 import inputs as I

K_MIN_PEAK = 2.0 ** -12


def _f16(x):
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float64)


def _tables(jbp, K, q):
    """The library's tables, decoded (core-matrix tile order) into dense matrices."""
    S, t = jbp.dft_tables(K, q)
    L, KB, Nc = S["L"], S["KB"], S["Nc"]

    def tile(buf, rows, D):
        h = np.frombuffer(buf, dtype=np.float16, count=rows * D).astype(np.float64)
        m = np.arange(rows)[:, None]
        k = np.arange(D)[None, :]
        return h[((m // 8) * (D // 8) * 128 + (k // 8) * 128 + (m % 8) * 16 + (k % 8) * 2) // 2]

    Fh, Fl, Bh, Bl = (np.zeros((L, KB)), np.zeros((L, KB)), np.zeros((q, L)), np.zeros((q, L)))
    off, b1, b3 = 0, Nc * KB * 2, q * Nc * 2
    for c in range(S["chunks"]):
        sl = slice(c * Nc, (c + 1) * Nc)
        Fh[sl] = tile(t[off:off + b1].tobytes(), Nc, KB); off += b1
        Fl[sl] = tile(t[off:off + b1].tobytes(), Nc, KB); off += b1
        Bh[:, sl] = tile(t[off:off + b3].tobytes(), q, Nc); off += b3
        Bl[:, sl] = tile(t[off:off + b3].tobytes(), q, Nc); off += b3
    tw = np.frombuffer(t[off:].tobytes(), dtype=np.float32).reshape(L, 2)
    return S, Fh, Fl, Bh, Bl, tw


def _loo(m, g):
    """X_k = g conj(prod_{j != k} m_j) by prefix and suffix products (complex64)."""
    R, K, P = m.shape
    one = np.ones((R, P), dtype=np.complex64)
    pre = [one]
    for k in range(1, K):
        pre.append((pre[-1] * m[:, k - 1]).astype(np.complex64))
    X = np.empty_like(m)
    suf = one
    for k in range(K - 1, -1, -1):
        X[:, k] = (g * np.conj(pre[k] * suf)).astype(np.complex64)
        suf = (suf * m[:, k]).astype(np.complex64)
    return X


def dft_node_fp16(tabs, K, q, sigma2, y, mu, round16=_f16):
    """Modelled kernel output [R, K, q] (max 1, floored) and the resolved-row mask;
    round16 is the rounding of the single-term and split operands."""
    S, Fh, Fl, Bh, Bl, tw = tabs
    L, W = S["L"], S["W"]
    R = y.shape[0]
    U, KD = K * (q - 1) + 1, K * (q - 1)
    # Gaussian window in FP32 around the nearest symbol sum
    y32 = y.astype(np.float32)
    ss = np.clip(np.rint((y32 + np.float32(KD)) * np.float32(0.5)), 0, KD).astype(np.int64)
    r = (y32 - (2 * ss - KD).astype(np.float32)).astype(np.float32)
    inv_s2 = np.float32(1.0 / sigma2)
    u_lo = np.minimum(np.maximum(ss - W // 2, 0), max(U - W, 0))
    u = u_lo[:, None] + np.arange(W)[None, :]
    d = (ss[:, None] - u).astype(np.float32)
    k2 = np.float32(np.float32(-2.0 * math.log2(math.e)) * inv_s2)
    k2r = (k2 * r).astype(np.float32)
    t = (np.float64(k2) * d.astype(np.float64) + k2r[:, None].astype(np.float64)).astype(np.float32)
    e = np.exp2((d * t).astype(np.float32))
    g16 = round16(np.where(u < U, e, 0.0))
    mu16 = round16(mu)
    # forward products, FP32 sums of exact FP16 products
    spec = np.concatenate([mu16 @ Fh[:, :q].T + mu16 @ Fl[:, :q].T,
                           (g16 @ Fh[:, :W].T + g16 @ Fl[:, :W].T)[:, None, :]], axis=1).astype(np.float32)
    spec = (spec * (np.float32(1.0) / spec[:, :, :1])).astype(np.float32)      # DC 1
    P = L // 2
    mh = (spec[:, :K, 2::2] + 1j * spec[:, :K, 3::2]).astype(np.complex64)        # f = 1..P-1
    gw = (spec[:, K, 2::2] + 1j * spec[:, K, 3::2]).astype(np.complex64)
    w = tw[(np.arange(1, P)[None, :] * u_lo[:, None]) % L]
    gh = (gw * (w[..., 0] - 1j * w[..., 1]).astype(np.complex64)).astype(np.complex64)
    X = _loo(mh, gh)
    # pair 0: DC (1) and Nyquist, real
    nyq_m = spec[:, :K, 1]
    nyq_g = spec[:, K, 1] * np.where(u_lo % 2 == 1, -1.0, 1.0).astype(np.float32)
    Xn = np.empty((R, K), dtype=np.float32)
    for k in range(K):
        Xn[:, k] = nyq_g * np.prod(np.delete(nyq_m, k, axis=1), axis=1, dtype=np.float32)
    Xc = np.empty((R, K, L), dtype=np.float32)
    Xc[:, :, 0] = 1.0
    Xc[:, :, 1] = Xn
    Xc[:, :, 2::2] = X.real
    Xc[:, :, 3::2] = X.imag
    Xh = round16(Xc)
    Xl = round16(Xc - Xh)
    out = (Xh @ Bh.T + Xl @ Bh.T + Xh @ Bl.T).astype(np.float32)
    mx = out.max(axis=2, keepdims=True)
    resolved = (mx[:, :, 0] >= np.float32(K_MIN_PEAK * L)).all(axis=1)
    return np.maximum(out / mx, 1e-12), resolved


@pytest.mark.parametrize("K,q,snr", [(2, 16, 8.0), (4, 16, 10.0), (8, 16, 12.0), (3, 32, 6.0), (5, 32, 16.0),
                                     (2, 64, 12.0), (4, 64, 14.0), (8, 64, 14.0)])
def test_fp16_model_of_the_dft_node_is_inside_the_stated_bound(jbp_lib, oracle, K, q, snr):
    m = int(math.log2(q))
    sigma2 = (q * q - 1) / 3.0 * 10 ** (-snr / 10)
    rng = np.random.default_rng(1000 * K + q)
    R = 96
    # the node's inputs as in the GPU parity tests: mu = product of two random c2v, max 1
    lc = I.random_log_messages(rng, (R, 2, K), q, spread=3.0)
    logmu = lc.sum(axis=1)
    logmu -= logmu.max(axis=-1, keepdims=True)
    mu = np.exp(logmu).astype(np.float32)
    sym = rng.integers(0, q, (R, K))
    y = ((2 * sym - (q - 1)).sum(axis=1) + rng.normal(size=R) * math.sqrt(sigma2)).astype(np.float32)
    got, ok = dft_node_fp16(_tables(jbp_lib, K, q), K, q, sigma2, y.astype(np.float64), mu)
    assert ok.mean() >= 0.5
    worst = 0.0
    for i in np.flatnonzero(ok):
        ref = np.exp(oracle.channel_node(K, m, sigma2, float(y[i]), logmu[i]))
        ref = ref / ref.max(axis=1, keepdims=True)
        worst = max(worst, float(np.abs(got[i] - ref).max()))
    bound = (K + 2) * 2.0 ** -9 + K * 2.0 ** -12
    print("K=%d q=%d %.0f dB: %d of %d rows resolved, max |FP16 model - oracle| = %.2e (bound %.2e)"
          % (K, q, snr, ok.sum(), R, worst, bound))
    assert worst <= bound
    assert worst <= 2e-3          # the size measured on the GPU, not just inside the bound


def test_fp64_arithmetic_closes_the_gap(jbp_lib, oracle):
    """With the same tables and FP32 arithmetic but no FP16 rounding of mu, the
    window or X, the error falls below 1e-5 (the FP32 sums and the tables' hi + lo
    precision): the FP16 operand terms are the error budget of the model above."""
    K, q, snr = 4, 64, 14.0
    sigma2 = (q * q - 1) / 3.0 * 10 ** (-snr / 10)
    rng = np.random.default_rng(3)
    R = 32
    logmu = I.random_log_messages(rng, (R, K), q, spread=3.0)
    mu = np.exp(logmu)
    sym = rng.integers(0, q, (R, K))
    y = (2 * sym - (q - 1)).sum(axis=1) + rng.normal(size=R) * math.sqrt(sigma2)
    S, Fh, Fl, Bh, Bl, tw = _tables(jbp_lib, K, q)
    exact = (S, Fh + Fl, np.zeros_like(Fl), Bh + Bl, np.zeros_like(Bl), tw)
    got, ok = dft_node_fp16(exact, K, q, sigma2, y, mu, round16=lambda x: np.asarray(x, dtype=np.float64))
    worst = 0.0
    for i in np.flatnonzero(ok):
        ref = np.exp(oracle.channel_node(K, 6, sigma2, float(y[i]), logmu[i]))
        ref = ref / ref.max(axis=1, keepdims=True)
        worst = max(worst, float(np.abs(got[i] - ref).max()))
    print("no FP16 operand rounding: max err %.2e" % worst)
    assert worst <= 1e-5, worst
