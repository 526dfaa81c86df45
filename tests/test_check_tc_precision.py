"""The tensor-core check node's rounding, modelled on the CPU.

The GPU variants run both Walsh-Hadamard transforms of the check node as products
with the +-1 Sylvester matrix on the tensor cores: every FP32 operand is split
into 1, 2 or 3 BF16 terms (BF16, BF16X2, BF16X3), each product of a term with
+-1 is exact, and the sums accumulate in FP32.  This test runs that arithmetic
in numpy (BF16 rounding to nearest even from the format's definition; the FP32
sums as one rounding of the exact sum) over checks of degree 4 and compares it
with the FP64 oracle's check node.  The error must stay inside the bound the
GPU tests assert, 2 B_q + 4 q u with u the split's unit (2^-9, 2^-17, 2^-25) and
B_q = q (4 log2 q + 2) 2^-24, and the BF16 and BF16X2 errors (where the split,
not the FP32 sums, dominates) come out at the size the GPU measures.
"""
import math

import numpy as np
import pytest

from paper_2605_26580_gb300 import inputs as I


def bf16(x):
    """Round FP32 values to BF16 (nearest, ties to even), returned as FP32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def split(x, n):
    """n BF16 terms of FP32 x: hi, then the rounded remainders."""
    x = np.asarray(x, dtype=np.float32)
    terms, r = [], x
    for _ in range(n):
        t = bf16(r)
        terms.append(t.astype(np.float64))
        r = (r - t).astype(np.float32)
    return terms


def sylvester(q):
    k = np.arange(q)
    pc = np.vectorize(lambda v: bin(v).count("1"))(k[:, None] & k[None, :])
    return np.where(pc % 2 == 1, -1.0, 1.0)


def check_tc_model(gdiv, coef, v2c, nsplit):
    """c2v [C, 4, q] of C degree-4 checks from v2c [C, 4, q] (FP32, max 1)."""
    C, dc, q = v2c.shape
    H = sylvester(q)
    z = np.arange(q)
    # permuted messages p~_e(z) = v2c_e(z / h_e)
    P = np.take_along_axis(v2c, gdiv[z[None, None, :], coef[:, :, None]], axis=2).astype(np.float32)

    def transform(A):
        return sum(t @ H for t in split(A, nsplit)).astype(np.float32)

    T = transform(P)
    e = np.arange(dc)
    V = (T[:, e ^ 1] * (T[:, e ^ 2] * T[:, e ^ 3])).astype(np.float32)
    O = transform(V)
    mx = O.max(axis=2, keepdims=True)
    O = (np.maximum(O, np.float32(1e-12) * mx) * (np.float32(1.0) / mx)).astype(np.float32)
    out = np.empty_like(O)
    # c2v_e(z / h_e) = O_e(z)
    np.put_along_axis(out, gdiv[z[None, None, :], coef[:, :, None]], O, axis=2)
    return out


@pytest.mark.parametrize("q,nsplit,lo,hi", [(16, 1, 5e-4, 3e-2), (16, 2, 1e-7, 1e-4), (16, 3, 0.0, 1e-5),
                                            (64, 1, 5e-4, 3e-2), (64, 2, 1e-7, 1e-4), (64, 3, 0.0, 1e-5)])
def test_bf16_split_model_of_the_check_node(oracle, q, nsplit, lo, hi):
    m = int(math.log2(q))
    mul = np.array([[oracle.gf_mul(m, a, b) for b in range(q)] for a in range(q)])
    gdiv = np.zeros((q, q), dtype=np.int64)            # gdiv[z, h] = z / h
    for h in range(1, q):
        gdiv[mul[:, h], h] = np.arange(q)
    rng = np.random.default_rng(7 * q + nsplit)
    C = 256
    coef = rng.integers(1, q, (C, 4))
    logv = I.random_log_messages(rng, (C, 4), q, spread=3.0)
    v2c = np.exp(logv).astype(np.float32)
    got = check_tc_model(gdiv, coef, v2c, nsplit)
    ref = np.stack([oracle.check_node(m, coef[c], np.log(v2c[c].astype(np.float64))) for c in range(C)])
    rho = np.exp(ref)
    lin = float(np.abs(got - rho).max())
    log_hi = float(np.abs(np.log(got) - ref)[rho >= 0.5].max())
    Bq = q * (4 * m + 2) * 2.0 ** -24
    u = {1: 2.0 ** -9, 2: 2.0 ** -17, 3: 2.0 ** -25}[nsplit]
    print("q=%d %d-term BF16: linear err %.2e (bound %.2e), log err at rho >= 0.5 %.2e"
          % (q, nsplit, lin, 2 * Bq + 4 * q * u, log_hi))
    assert lin <= 2 * Bq + 4 * q * u
    assert lo <= log_hi <= hi
