"""The DFT channel node's constant operand tables, read back through the C ABI on
the CPU (jbp_dft_tables builds them on the host, as jbp_create does).

The tables are decoded here from the layout the header documents (per chunk:
forward hi/lo tiles [Nc x KB], inverse hi/lo tiles [q x Nc] in 8x8 core-matrix
order; then L twiddle pairs) and checked against the mathematics they encode:
  * every FP16 hi + lo pair is the value within the two-term split bound, and
    hi alone is its FP16 rounding;
  * the folded inverse undoes the folded forward: B F = L I on the q columns the
    messages use, and F's first q columns carry the DFT of a real vector, so
    transforming a random vector and inverting it returns L times the vector;
  * the window columns x >= q continue the same transform (the Gaussian score
    uses x = 0..W-1);
  * the twiddles are (cos, sin)(2 pi m / L) in FP32.
A transposed tile, a wrong sign on the sine rows, a swapped DC/Nyquist pair or a
wrong factor 2 on the folded pairs fails one of these.
"""
import numpy as np
import pytest

from paper_2605_26580_gb300 import jbp


def _tile(buf, rows, D):
    """(rows x D) FP16 tile in core-matrix order -> dense float64 matrix."""
    h = np.frombuffer(buf, dtype=np.float16, count=rows * D).astype(np.float64)
    m = np.arange(rows)[:, None]
    k = np.arange(D)[None, :]
    byte = (m // 8) * (D // 8) * 128 + (k // 8) * 128 + (m % 8) * 16 + (k % 8) * 2
    return h[byte // 2]


def _decode(K, q):
    S, t = jbp.dft_tables(K, q)
    L, KB, Nc, chunks = S["L"], S["KB"], S["Nc"], S["chunks"]
    b1, b3 = Nc * KB * 2, q * Nc * 2
    Fhi = np.zeros((L, KB)); Flo = np.zeros((L, KB))
    Bhi = np.zeros((q, L)); Blo = np.zeros((q, L))
    off = 0
    for c in range(chunks):
        rows = slice(c * Nc, (c + 1) * Nc)
        Fhi[rows] = _tile(t[off:off + b1].tobytes(), Nc, KB); off += b1
        Flo[rows] = _tile(t[off:off + b1].tobytes(), Nc, KB); off += b1
        Bhi[:, rows] = _tile(t[off:off + b3].tobytes(), q, Nc); off += b3
        Blo[:, rows] = _tile(t[off:off + b3].tobytes(), q, Nc); off += b3
    tw = np.frombuffer(t[off:].tobytes(), dtype=np.float32).reshape(L, 2).astype(np.float64)
    assert off + 8 * L == t.size
    return S, Fhi, Flo, Bhi, Blo, tw


def _expected(L, KB, q):
    """Folded real DFT of length L (rows n: pair p = n // 2) and its inverse."""
    n = np.arange(L)[:, None]
    p = n // 2
    x = np.arange(KB)[None, :]
    th = 2 * np.pi * ((p * x) % L) / L
    F = np.where(n % 2 == 1, -np.sin(th), np.cos(th))
    F[1] = np.where(np.arange(KB) % 2 == 1, -1.0, 1.0)       # Nyquist term of pair 0
    a = np.arange(q)[:, None]
    nn = np.arange(L)[None, :]
    pp = nn // 2
    th = 2 * np.pi * ((pp * a) % L) / L
    B = np.where(nn % 2 == 1, -2 * np.sin(th), 2 * np.cos(th))
    B[:, 0] = 1.0
    B[:, 1] = np.where(np.arange(q) % 2 == 1, -1.0, 1.0)
    return F, B


SHAPES = [(2, 16), (3, 16), (4, 16), (8, 16), (2, 32), (5, 32), (8, 32), (2, 64), (4, 64), (6, 64), (8, 64)]


@pytest.mark.parametrize("K,q", SHAPES)
def test_tables_hold_the_folded_transform_pair(jbp_lib, K, q):
    S, Fhi, Flo, Bhi, Blo, tw = _decode(K, q)
    L, W, KB = S["L"], S["W"], S["KB"]
    assert L % 16 == 0 and L >= K * (q - 1) + 1 > L - 16
    assert W == min(L, 128) and KB == max(q, W)
    assert L % S["Nc"] == 0 and S["chunks"] == L // S["Nc"]
    F, B = _expected(L, KB, q)
    # hi is the FP16 rounding; hi + lo is the value to the two-term split bound
    assert np.array_equal(Fhi, F.astype(np.float16).astype(np.float64))
    assert np.array_equal(Bhi, B.astype(np.float16).astype(np.float64))
    assert np.abs(Fhi + Flo - F).max() <= 2.0 ** -21
    assert np.abs(Bhi + Blo - B).max() <= 2.0 ** -20
    # the inverse undoes the forward on the message columns: B F = L I
    Fs, Bs = Fhi + Flo, Bhi + Blo
    assert np.abs(Bs @ Fs[:, :q] - L * np.eye(q)).max() <= L * 2.0 ** -19
    rng = np.random.default_rng(K * 64 + q)
    v = rng.random(q)
    assert np.abs(Bs @ (Fs[:, :q] @ v) / L - v).max() <= q * 2.0 ** -19
    # the window columns are the same transform: the DFT of a real window g
    g = rng.random(W)
    spec = np.fft.fft(g, L)
    P = L // 2
    got = Fs[:, :W] @ g
    assert abs(got[0] - spec[0].real) <= 1e-4 and abs(got[1] - spec[P].real) <= 1e-4
    assert np.abs(got[2::2] - spec[1:P].real).max() <= 1e-4
    assert np.abs(got[3::2] - spec[1:P].imag).max() <= 1e-4
    # twiddles
    m = np.arange(L)
    assert np.abs(tw[:, 0] - np.cos(2 * np.pi * m / L)).max() <= 2.0 ** -24
    assert np.abs(tw[:, 1] - np.sin(2 * np.pi * m / L)).max() <= 2.0 ** -24


@pytest.mark.parametrize("K,q", [(1, 16), (9, 16), (2, 8), (2, 128), (4, 2), (0, 32)])
def test_shapes_without_a_dft_form_are_refused(jbp_lib, K, q):
    with pytest.raises(jbp.JBPError) as e:
        jbp.dft_tables(K, q)
    assert e.value.code == jbp.EINVAL


def test_null_size_is_refused(jbp_lib):
    assert jbp.lib().jbp_dft_tables(4, 64, None, None, None) == jbp.EINVAL
