"""Seeded input generator: code structure, encoder, interleavers, channel output."""
import math

import numpy as np
import pytest

from paper_2605_26580_gb300 import inputs as I


@pytest.mark.parametrize("n,q", [(64, 4), (256, 16), (512, 64), (128, 2)])
def test_regular_code_structure(n, q):
    code = I.make_code(n, q)
    P, dc = code["P"], code["dc"]
    assert P == n // 2 and code["chk_var"].size == P * dc
    counts = np.bincount(code["chk_var"], minlength=n)
    assert (counts == 2).all()                              # dv = 2 regular
    rows = code["chk_var"].reshape(P, dc)
    assert all(len(set(r)) == dc for r in rows.tolist())    # no double edges
    pairs = set()
    for i in range(n):                                      # no 4-cycles: no two vars share two checks
        cs = tuple(sorted(set(np.nonzero((rows == i).any(1))[0].tolist())))
        assert cs not in pairs
        pairs.add(cs)
    assert ((code["chk_coef"] >= 1) & (code["chk_coef"] < q)).all()
    assert code["k"] == n - code["rank"] and code["k"] >= n // 2


def test_code_is_reproducible():
    a, b = I.make_code(128, 16), I.make_code(128, 16)
    assert (a["chk_var"] == b["chk_var"]).all() and (a["chk_coef"] == b["chk_coef"]).all()
    c = I.make_code(128, 16, seed=1)
    assert not (a["chk_var"] == c["chk_var"]).all()


def test_encoder_is_systematic_and_linear():
    code = I.make_code(64, 16)
    rng = np.random.default_rng(0)
    info = rng.integers(0, 16, size=(10, code["k"]))
    c = I.encode(code, info)
    assert (c[:, code["info_pos"]] == info).all()
    # linearity over GF(2^m): c(u) xor c(v) = c(u xor v)
    u, v = info[:5], info[5:]
    assert (I.encode(code, u) ^ I.encode(code, v) == I.encode(code, u ^ v)).all()


def test_interleavers():
    pi = I.make_interleavers(100, 4, seed=3)
    assert (pi[0] == np.arange(100)).all()
    for k in range(4):
        assert sorted(pi[k].tolist()) == list(range(100))
    assert (I.make_interleavers(100, 4, seed=3, interleave=False) == np.arange(100)).all()


def test_channel_output_noiseless_and_noise_variance():
    code = I.make_code(64, 4)
    fr = I.make_frames(code, 3, 10.0, 50, seed=1, noiseless=True)
    pi = fr["perm"]
    y = np.zeros((50, 64))
    for k in range(3):
        for i in range(64):
            y[:, pi[k, i]] += 2.0 * fr["c"][:, k, i].astype(np.float64) - 3
    assert np.array_equal(fr["y"], y.astype(np.float32))
    noisy = I.make_frames(code, 3, 10.0, 2000, seed=1)
    clean = np.zeros((2000, 64))
    for k in range(3):
        clean[:, pi[k]] += 2.0 * noisy["c"][:, k] - 3
    w = noisy["y"] - clean
    assert abs(w.var() / noisy["sigma2"] - 1) < 0.05
    assert math.isclose(noisy["sigma2"], 5.0 * 10 ** -1.0)   # E_s = (q^2-1)/3 = 5 at q = 4


def test_random_messages_are_max_normalised():
    rng = np.random.default_rng(0)
    m = I.random_log_messages(rng, (7, 3), 16)
    assert m.shape == (7, 3, 16)
    assert np.allclose(m.max(-1), 0.0) and m.min() >= math.log(1e-12)


def test_ura_frames_follow_the_slot_model():
    """Noiseless y equals sqrt(P_sym) * FFT of the activity vector at the slot's
    rows, / sqrt(ns); rows are distinct per slot; (2,3) codes have rate 1/3."""
    import math
    code = I.make_code(12, 64, dv=2, dc=3)
    assert code["P"] == 8 and code["k"] == 4
    fr = I.make_ura_frames(code, 2, 10.0, 3, seed=1, noiseless=True)
    assert fr["psym"] == pytest.approx(6 * 4 * 10.0 / 12)
    for l in range(12):
        assert len(set(fr["rows"][l].tolist())) == 24
    for f in range(3):
        for l in range(12):
            u = np.zeros(64)
            for k in range(2):
                u[fr["X"][f, k, l]] += 1
            want = np.fft.fft(u)[fr["rows"][l]] / math.sqrt(24) * math.sqrt(fr["psym"])
            got = fr["y"][f, l, :, 0] + 1j * fr["y"][f, l, :, 1]
            assert np.abs(got - want).max() < 1e-4


def test_ura_noise_is_unit_complex_gaussian():
    code = I.make_code(12, 64, dv=2, dc=3)
    a = I.make_ura_frames(code, 2, 10.0, 400, seed=2)
    b = I.make_ura_frames(code, 2, 10.0, 400, seed=2, noiseless=True)
    w = (a["y"] - b["y"]).reshape(-1, 2).astype(np.float64)
    assert abs(w.var(axis=0).mean() - 0.5) < 0.01


def test_girth_of_known_graphs():
    # two variables on the same two checks: a 4-cycle
    four = I.code_from_edges(4, 4, 2, [0, 1, 0, 1, 2, 3], [1, 1, 1, 1, 1, 1])
    assert I.girth(four) == 4
    # two checks of degree 3 sharing one variable: no cycle
    tree = I.code_from_edges(5, 4, 3, [0, 1, 2, 2, 3, 4], [1, 2, 3, 2, 1, 3])
    assert I.girth(tree) == 0
    # a 6-cycle: v0-c0-v1-c1-v2-c2-v0
    six = I.code_from_edges(3, 4, 2, [0, 1, 1, 2, 2, 0], [1, 1, 1, 1, 1, 1])
    assert I.girth(six) == 6


@pytest.mark.parametrize("L", [12, 24, 48])
def test_peg_codes_are_regular_with_larger_girth(L):
    c = I.make_peg_code(L, 64)
    assert c["P"] == 2 * L // 3 and c["k"] == L // 3
    assert set(np.bincount(c["chk_var"], minlength=L).tolist()) == {2}
    for j in range(c["P"]):
        assert len(set(c["chk_var"][3 * j:3 * j + 3].tolist())) == 3
    assert I.girth(c) > I.girth(I.make_code(L, 64, dv=2, dc=3))
    again = I.make_peg_code(L, 64)
    assert np.array_equal(c["chk_var"], again["chk_var"]) and np.array_equal(c["chk_coef"], again["chk_coef"])


def test_irregular_code_follows_its_profile(oracle):
    """make_irregular_code: the variable degrees follow the profile (rounded, the
    edge count made a multiple of dc), every check has dc distinct variables, no
    two variables share two checks, and generated codewords satisfy H c = 0."""
    import itertools
    code = I.make_irregular_code(128, 16, {2: 0.5, 3: 0.3, 4: 0.2}, 4)
    deg = np.bincount(code["chk_var"], minlength=128)
    assert code["dv"] == deg.max() == 4
    assert sum(deg) == code["P"] * 4
    assert abs((deg == 2).sum() - 64) <= 1 and abs((deg == 3).sum() - 38) <= 3 and abs((deg == 4).sum() - 26) <= 3
    rows = code["chk_var"].reshape(code["P"], 4)
    assert all(len(set(r)) == 4 for r in rows)
    pairs = set()
    for r in rows:
        for a, b in itertools.combinations(sorted(r), 2):
            assert (a, b) not in pairs
            pairs.add((a, b))
    assert I.girth(code) >= 6
    rng = np.random.default_rng(3)
    c = I.encode(code, rng.integers(0, 16, size=(5, code["k"])))
    assert (oracle.syndrome_ok(code, 5, c[None].astype(np.uint8)) == 1).all()   # the oracle's field, not the generator's
