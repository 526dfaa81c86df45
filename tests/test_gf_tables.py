"""The decoder's setup tables of GF(q) (step a0), read back through the C ABI on
the CPU: jbp_gf_tables returns the multiply and divide tables jbp_create uploads.
They must equal the textbook tables (tests/golden), the oracle's independent
field arithmetic bit for bit, and divide exactly."""
import os

import numpy as np
import pytest

from paper_2605_26580_gb300 import jbp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return np.array([[int(v) for v in ln.split()] for ln in f if ln.strip() and not ln.startswith("#")])


def test_gf4_and_gf16_match_the_textbook_tables(jbp_lib):
    mul4, _ = jbp.gf_tables(4)
    assert np.array_equal(mul4, _golden("gf4_mul.txt"))
    mul16, _ = jbp.gf_tables(16)
    x = 1
    for i, expect in _golden("gf16_powers.txt"):          # powers of alpha = x
        assert x == expect, (i, x, expect)
        x = int(mul16[x, 2])


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6])
def test_tables_equal_the_oracle_and_divide_exactly(jbp_lib, oracle, m):
    q = 1 << m
    mul, div = jbp.gf_tables(q)
    ref = np.array([[oracle.gf_mul(m, a, b) for b in range(q)] for a in range(q)])
    assert np.array_equal(mul, ref)
    assert (div[0] == 0).all()
    x = np.arange(q)
    for h in range(1, q):
        assert np.array_equal(mul[h, div[h]], x)           # h (x / h) = x
        assert np.array_equal(div[h, mul[h]], x)           # (h x) / h = x


@pytest.mark.parametrize("q", [0, 1, 3, 12, 128, 256])
def test_other_field_sizes_are_refused(jbp_lib, q):
    with pytest.raises(jbp.JBPError) as e:
        jbp.gf_tables(q) if q > 0 else jbp.check(jbp.lib().jbp_gf_tables(q, None, None))
    assert e.value.code == jbp.EINVAL


@pytest.mark.parametrize("m", [2, 4, 5, 6])
def test_division_by_a_coefficient_is_linear_over_gf2(jbp_lib, m):
    """The staged check kernel permutes by XOR of basis images: x / h is the XOR
    of (2^i) / h over the set bits i of x, for every nonzero h."""
    q = 1 << m
    _, div = jbp.gf_tables(q)
    for h in range(1, q):
        basis = [int(div[h, 1 << i]) for i in range(m)]
        for x in range(q):
            acc = 0
            for i in range(m):
                if (x >> i) & 1:
                    acc ^= basis[i]
            assert acc == div[h, x], (h, x)
