"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against a closed form, a textbook special case,
brute-force enumeration or an invariant, chosen so that a dropped term, a sign
error, a transposed index or a wrong permutation direction in the oracle fails
at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

from paper_2605_26580_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LOG_FLOOR = math.log(1e-12)


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(v) for v in line.split()])
    return np.array(rows)


# --------------------------------------------------------------------------- field

def test_gf4_table_matches_definition(oracle):
    tab = _golden("gf4_mul.txt")
    got = np.array([[oracle.gf_mul(2, a, b) for b in range(4)] for a in range(4)])
    assert (got == tab).all()


def test_gf16_powers_match_textbook_table(oracle):
    tab = _golden("gf16_powers.txt")
    x = 1
    for i, expect in tab:
        assert x == expect, (i, x, expect)
        x = oracle.gf_mul(4, x, 2)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6])
def test_gf_field_axioms(oracle, m):
    q = 1 << m
    mul = np.array([[oracle.gf_mul(m, a, b) for b in range(q)] for a in range(q)])
    assert (mul == mul.T).all()                                       # commutative
    assert (mul[1] == np.arange(q)).all() and (mul[0] == 0).all()     # identity, zero
    for a in range(1, q):                                             # every nonzero is invertible
        assert (mul[a] == 1).sum() == 1
        assert sorted(mul[a].tolist()) == list(range(q))              # multiplication permutes F_q
    rng = np.random.default_rng(m)
    for a, b, c in rng.integers(0, q, size=(200, 3)):
        assert mul[mul[a, b], c] == mul[a, mul[b, c]]                 # associative
        assert mul[a, b ^ c] == mul[a, b] ^ mul[a, c]                 # distributes over XOR (char 2)
    # x generates the multiplicative group: the polynomial is primitive
    x, seen = 1, set()
    for _ in range(q - 1):
        seen.add(x)
        x = mul[x, 2 % q] if q > 2 else 1
    assert len(seen) == q - 1


# --------------------------------------------------------------------------- channel node

@pytest.mark.parametrize("K,m", [(1, 1), (1, 3), (2, 1), (2, 2), (2, 3), (3, 2), (3, 3), (4, 2), (2, 4), (5, 1)])
def test_channel_trellis_equals_enumeration(oracle, K, m):
    q = 1 << m
    rng = np.random.default_rng(100 * K + m)
    for _ in range(4):
        lm = I.random_log_messages(rng, (K,), q, spread=4.0)
        y = rng.normal() * 2 * K * (q - 1) / 3
        s2 = rng.uniform(0.3, 6.0)
        a = oracle.channel_node(K, m, s2, y, lm)
        b = oracle.channel_node(K, m, s2, y, lm, brute=True)
        assert np.abs(a - b).max() < 1e-11


@pytest.mark.parametrize("K,m,y,s2", [(3, 2, 0.7, 2.0), (3, 2, 40.0, 0.05), (2, 3, -60.0, 0.1), (4, 1, 9.5, 0.01)])
def test_channel_node_equals_python_enumeration_in_log_space(oracle, K, m, y, s2):
    """The channel factor written out in plain Python, in log space so that far
    observations (beyond the largest symbol sum, tiny noise) do not underflow:
    msg_k(a) = log sum over the other users' symbols of prod_j mu_j(x_j) times
    N(y; level(a) + sum_j level(x_j), s2), max-normalised and floored."""
    q = 1 << m
    rng = np.random.default_rng(K * 13 + m)
    lm = I.random_log_messages(rng, (K,), q, spread=3.0)
    lev = 2.0 * np.arange(q) - (q - 1)
    ref = np.full((K, q), -np.inf)
    for k in range(K):
        others = [j for j in range(K) if j != k]
        for a in range(q):
            terms = []
            for xs in itertools.product(range(q), repeat=K - 1):
                mean = lev[a] + sum(lev[x] for x in xs)
                terms.append(sum(lm[j, x] for j, x in zip(others, xs)) - (y - mean) ** 2 / (2 * s2))
            t = np.array(terms)
            ref[k, a] = t.max() + math.log(np.exp(t - t.max()).sum())
    ref = np.maximum(ref - ref.max(axis=1, keepdims=True), LOG_FLOOR)
    got = oracle.channel_node(K, m, s2, y, lm)
    assert np.abs(got - ref).max() < 1e-9


@pytest.mark.parametrize("m", [1, 2, 4, 6])
def test_channel_single_user_is_gaussian_likelihood(oracle, m):
    """K = 1: the channel message is log N(y; 2a - (q-1), sigma2), max-normalised."""
    q = 1 << m
    rng = np.random.default_rng(7 + m)
    for _ in range(5):
        y, s2 = rng.normal() * q, rng.uniform(0.5, 4.0) * q
        got = oracle.channel_node(1, m, s2, y, np.zeros((1, q)))[0]
        lev = 2.0 * np.arange(q) - (q - 1)
        ll = -(y - lev) ** 2 / (2 * s2)
        assert np.allclose(got, np.maximum(ll - ll.max(), LOG_FLOOR), atol=1e-12)


def test_channel_two_users_closed_form(oracle):
    """K = 2: message to user 0 is log sum_b mu_1(b) N(y; level(a) + level(b))."""
    q, m = 4, 2
    rng = np.random.default_rng(3)
    lm = I.random_log_messages(rng, (2,), q, spread=3.0)
    y, s2 = 1.3, 0.8
    lev = 2.0 * np.arange(q) - (q - 1)
    lik = np.exp(-(y - lev[:, None] - lev[None, :]) ** 2 / (2 * s2))       # [a0, a1]
    to0 = np.log(lik @ np.exp(lm[1]))
    to1 = np.log(np.exp(lm[0]) @ lik)
    got = oracle.channel_node(2, m, s2, y, lm)
    assert np.allclose(got[0], np.maximum(to0 - to0.max(), LOG_FLOOR), atol=1e-12)
    assert np.allclose(got[1], np.maximum(to1 - to1.max(), LOG_FLOOR), atol=1e-12)


# --------------------------------------------------------------------------- check node

@pytest.mark.parametrize("m,dc", [(1, 3), (2, 2), (2, 3), (2, 4), (3, 4), (4, 3), (4, 4)])
def test_check_wht_direct_literal_agree(oracle, m, dc):
    q = 1 << m
    rng = np.random.default_rng(10 * m + dc)
    for _ in range(3):
        coef = rng.integers(1, q, dc)
        lv = I.random_log_messages(rng, (dc,), q, spread=5.0)
        lit = oracle.check_node(m, coef, lv, oracle.CHECK_LITERAL, rel_floor=0.0)
        dirc = oracle.check_node(m, coef, lv, oracle.CHECK_DIRECT, rel_floor=0.0)
        wht = oracle.check_node(m, coef, lv, oracle.CHECK_WHT, rel_floor=0.0)
        assert np.abs(np.exp(lit) - np.exp(dirc)).max() < 1e-13
        assert np.abs(np.exp(lit) - np.exp(wht)).max() < 1e-12
        mask = lit > math.log(1e-8)
        assert np.abs(lit - wht)[mask].max() < 1e-6


@pytest.mark.parametrize("m,dc", [(1, 4), (2, 3), (2, 4), (3, 3)])
def test_check_node_equals_enumeration_of_the_parity_equation(oracle, m, dc):
    """Eq. app_ldpc_c2v by enumeration in plain Python: c2v_d(a) is proportional to
    the sum, over the other symbols x_e with h_d a + sum_e h_e x_e = 0 in GF(q), of
    the product of their v2c_e(x_e).  Field products come from the golden-pinned
    multiplication (x is the generator, tables checked above)."""
    q = 1 << m
    mul = [[oracle.gf_mul(m, a, b) for b in range(q)] for a in range(q)]
    rng = np.random.default_rng(100 + 10 * m + dc)
    coef = [int(h) for h in rng.integers(1, q, dc)]
    lv = I.random_log_messages(rng, (dc,), q, spread=2.0)
    v = np.exp(lv)
    ref = np.zeros((dc, q))
    for d in range(dc):
        others = [e for e in range(dc) if e != d]
        for xs in itertools.product(range(q), repeat=dc - 1):
            syn = 0
            w = 1.0
            for e, x in zip(others, xs):
                syn ^= mul[coef[e]][x]
                w *= v[e, x]
            for a in range(q):
                if mul[coef[d]][a] == syn:       # h_d a + syn = 0 (characteristic 2)
                    ref[d, a] += w
    ref /= ref.max(axis=1, keepdims=True)
    for method in (oracle.CHECK_LITERAL, oracle.CHECK_DIRECT, oracle.CHECK_WHT):
        got = np.exp(oracle.check_node(m, coef, lv, method, rel_floor=0.0))
        assert np.abs(got - ref).max() < 1e-12, method


@pytest.mark.parametrize("m", [2, 4, 6])
def test_check_degree_two_is_a_permutation(oracle, m):
    """dc = 2: h0 a0 + h1 a1 = 0 forces a0 = h0^-1 h1 a1, so c2v_0(a) = v2c_1(h1^-1 h0 a)."""
    q = 1 << m
    rng = np.random.default_rng(m)
    mul = np.array([[oracle.gf_mul(m, a, b) for b in range(q)] for a in range(q)])
    inv = np.array([0] + [int(np.nonzero(mul[a] == 1)[0][0]) for a in range(1, q)])
    for method in (oracle.CHECK_WHT, oracle.CHECK_DIRECT, oracle.CHECK_LITERAL):
        h0, h1 = rng.integers(1, q, 2)
        lv = I.random_log_messages(rng, (2,), q, spread=2.0)
        got = oracle.check_node(m, [h0, h1], lv, method, rel_floor=0.0)
        for a in range(q):
            b = mul[inv[h1], mul[h0, a]]
            assert abs(got[0, a] - lv[1, b]) < 1e-9


def test_check_floor(oracle):
    """r <- max(r, 1e-12 max r): every c2v entry is >= ln(1e-12) and the max is 0."""
    rng = np.random.default_rng(5)
    lv = I.random_log_messages(rng, (4,), 16, spread=30.0)
    out = oracle.check_node(4, [3, 7, 9, 1], lv, oracle.CHECK_WHT)
    assert out.min() >= LOG_FLOOR - 1e-12
    assert np.allclose(out.max(axis=1), 0.0)


# --------------------------------------------------------------------------- whole decoder

def _brute_vs_bp(oracle, code, K, perm, y, sigma2, iters):
    exact, size = oracle.brute_marginals(code, K, sigma2, perm, y)
    out = oracle.decode(code, K, sigma2, perm, y[None, :], iters, early_stop=False,
                        check_method=oracle.CHECK_DIRECT, rel_floor=0.0, log_floor=-math.inf, want_post=True)
    pe = np.exp(exact)
    pe /= pe.sum(-1, keepdims=True)
    pb = np.exp(out["post"][0])
    pb /= pb.sum(-1, keepdims=True)
    return pe, pb, size, out


@pytest.mark.parametrize("q,n,checks", [(2, 8, [0, 1, 2, 3, 4, 5, 6, 7]), (4, 5, [0, 1, 2, 4])])
def test_brute_marginals_equal_python_enumeration(oracle, q, n, checks):
    """The oracle's exact joint marginals (the reference of the tree pins) against
    plain enumeration: every pair of codewords (c_0, c_1) with H c_k = 0 weighted
    by prod_t N(y_t; sum_k (2 c_k(pi_k^-1(t)) - (q-1)), sigma2), then summed per
    user, position and symbol."""
    m = int(math.log2(q))
    rng = np.random.default_rng(q * 7 + n)
    dc = 4
    coef = rng.integers(1, q, len(checks))
    code = I.code_from_edges(n, q, dc, checks, coef)
    mul = [[oracle.gf_mul(m, a, b) for b in range(q)] for a in range(q)]
    words = []
    for x in itertools.product(range(q), repeat=n):
        ok = True
        for j in range(len(checks) // dc):
            syn = 0
            for d in range(dc):
                e = j * dc + d
                syn ^= mul[int(coef[e])][x[checks[e]]]
            ok = ok and syn == 0
        if ok:
            words.append(x)
    W = np.array(words)                                   # [C, n]
    perm = np.stack([np.arange(n), rng.permutation(n)]).astype(np.int32)
    sigma2 = 1.7
    y = (rng.normal(size=n) * 2.0).astype(np.float32)
    lev = [np.zeros((len(W), n)), np.zeros((len(W), n))]
    for k in range(2):
        lev[k][:, perm[k]] = 2.0 * W - (q - 1)           # level on channel use pi_k(i)
    r = y.astype(np.float64)[None, None, :] - lev[0][:, None, :] - lev[1][None, :, :]
    ll = -(r * r).sum(-1) / (2 * sigma2)                  # [C, C]
    w = np.exp(ll - ll.max())
    ref = np.zeros((2, n, q))
    for i in range(n):
        for a in range(q):
            sel = W[:, i] == a
            ref[0, i, a] = w[sel, :].sum()
            ref[1, i, a] = w[:, sel].sum()
    ref /= ref.sum(-1, keepdims=True)
    exact, size = oracle.brute_marginals(code, 2, sigma2, perm, y)
    pe = np.exp(exact)
    pe /= pe.sum(-1, keepdims=True)
    assert size == len(W)
    assert np.abs(pe - ref).max() < 1e-12


@pytest.mark.parametrize("q,n,shift", [(2, 8, 4), (4, 7, 4)])
def test_bp_is_exact_on_cycle_free_joint_graph(oracle, q, n, shift):
    """Two users, one dc = 4 check each on positions 0..3; user 1's interleaver
    places its checked symbols on channel uses that meet at most one checked
    symbol of user 0, so the joint factor graph is a forest and BP marginals
    after enough iterations equal the exact marginals (enumeration)."""
    rng = np.random.default_rng(q * 100 + n)
    code = I.code_from_edges(n, q, 4, [0, 1, 2, 3], rng.integers(1, q, 4))
    perm = np.stack([np.arange(n), (np.arange(n) + shift) % n]).astype(np.int32)
    fr_c = I.encode(code, rng.integers(0, q, size=(2, code["k"])))
    sigma2 = I.sigma2_from_snr(q, 4.0)
    lev = 2.0 * fr_c - (q - 1)
    y = np.zeros(n)
    for k in range(2):
        y[perm[k]] += lev[k]
    y = (y + rng.normal(size=n) * math.sqrt(sigma2)).astype(np.float32)
    pe, pb, size, _ = _brute_vs_bp(oracle, code, 2, perm, y, sigma2, iters=12)
    assert size == q ** (n - 1)
    assert np.abs(pe - pb).max() < 1e-10


def test_bp_is_exact_on_single_user_tree_code(oracle):
    """K = 1, two checks sharing one variable: a tree; BP is exact."""
    q, n = 4, 7
    rng = np.random.default_rng(21)
    code = I.code_from_edges(n, q, 4, [0, 1, 2, 3, 3, 4, 5, 6], rng.integers(1, q, 8))
    c = I.encode(code, rng.integers(0, q, size=(1, code["k"])))[0]
    sigma2 = I.sigma2_from_snr(q, 3.0)
    y = (2.0 * c - (q - 1) + rng.normal(size=n) * math.sqrt(sigma2)).astype(np.float32)
    pe, pb, size, _ = _brute_vs_bp(oracle, code, 1, None, y, sigma2, iters=8)
    assert size == q ** 5
    assert np.abs(pe - pb).max() < 1e-10


def test_loopy_bp_differs_from_exact(oracle):
    """Sanity of the exactness pin: on a loopy joint graph (both users' checks on
    the same channel uses) BP marginals are not exact."""
    q, n = 2, 8
    rng = np.random.default_rng(4)
    code = I.code_from_edges(n, q, 4, [0, 1, 2, 3], [1, 1, 1, 1])
    perm = np.stack([np.arange(n), np.array([1, 0, 3, 2, 4, 5, 6, 7])]).astype(np.int32)
    y = (rng.normal(size=n) * 2).astype(np.float32)
    pe, pb, _, _ = _brute_vs_bp(oracle, code, 2, perm, y, 1.0, iters=12)
    assert np.abs(pe - pb).max() > 1e-4


def _single_user_qspa(code, y, sigma2, iters):
    """Textbook single-user GF(q) sum-product decoder (flooding), written
    independently of the oracle: local belief lambda(a) = N(y; 2a-(q-1), sigma2),
    v2c = lambda * other c2v, c2v by XOR convolution of coefficient-permuted
    messages, marginal = lambda * all c2v.  Same floors as the decoder."""
    q, m, n, dc = code["q"], code["m"], code["n"], code["dc"]
    poly = I.PRIM_POLY[m]

    def gmul(a, b):
        r = 0
        for i in range(m):
            if (b >> i) & 1:
                r ^= a << i
        for i in range(2 * m - 2, m - 1, -1):
            if (r >> i) & 1:
                r ^= poly << (i - m)
        return r

    mul = np.array([[gmul(a, b) for b in range(q)] for a in range(q)])
    E = code["P"] * dc
    var = code["chk_var"].astype(int)
    coef = code["chk_coef"].astype(int)
    lev = 2.0 * np.arange(q) - (q - 1)
    lam = -(y.astype(np.float64)[:, None] - lev[None, :]) ** 2 / (2 * sigma2)
    lam = np.maximum(lam - lam.max(1, keepdims=True), LOG_FLOOR)
    c2v = np.zeros((E, q))
    post = None
    for _ in range(iters):
        tot = lam.copy()
        np.add.at(tot, var, c2v)
        v2c = tot[var] - c2v
        v2c -= v2c.max(1, keepdims=True)
        p = np.exp(v2c)
        new = np.empty_like(c2v)
        for j in range(code["P"]):
            es = range(j * dc, (j + 1) * dc)
            pt = {e: np.zeros(q) for e in es}
            for e in es:
                pt[e][mul[coef[e]]] = p[e]
            for e in es:
                conv = np.zeros(q)
                conv[0] = 1.0
                for e2 in es:
                    if e2 == e:
                        continue
                    nxt = np.zeros(q)
                    for x1 in range(q):
                        nxt[np.arange(q) ^ x1] += conv[x1] * pt[e2]
                    conv = nxt
                r = conv[mul[coef[e]]]
                r = np.maximum(r, 1e-12 * r.max())
                new[e] = np.log(r) - np.log(r.max())
        c2v = new
        post = lam.copy()
        np.add.at(post, var, c2v)
    return post - post.max(1, keepdims=True)


def test_single_user_reduces_to_textbook_qspa(oracle):
    code = I.make_code(32, 4)
    fr = I.make_frames(code, 1, 6.0, 3, seed=9)
    out = oracle.decode(code, 1, fr["sigma2"], fr["perm"], fr["y"], 4, early_stop=False,
                        check_method=oracle.CHECK_DIRECT, want_post=True)
    for f in range(3):
        ref = _single_user_qspa(code, fr["y"][f], fr["sigma2"], 4)
        assert np.abs(out["post"][f, 0] - ref).max() < 1e-9
        assert (out["hat"][f, 0] == ref.argmax(1)).all()


def test_noiseless_single_user_decodes(oracle):
    """K = 1 without noise: every frame decodes to the transmitted codeword and stops early."""
    code = I.make_code(64, 16)
    fr = I.make_frames(code, 1, 10.0, 20, seed=5, noiseless=True)
    out = oracle.decode(code, 1, fr["sigma2"], fr["perm"], fr["y"], 20)
    assert (out["hat"] == fr["c"]).all()
    assert (out["iters"] < 20).all() and out["ok"].all()


def test_noiseless_two_users_cycle_free(oracle):
    """Noiseless two-user frames on the cycle-free graph: the exact posterior and BP
    both put their maximum on the transmitted symbols where the exact maximum is unique."""
    q, n = 2, 8
    rng = np.random.default_rng(8)
    code = I.code_from_edges(n, q, 4, [0, 1, 2, 3], [1, 1, 1, 1])
    perm = np.stack([np.arange(n), (np.arange(n) + 4) % n]).astype(np.int32)
    sigma2 = I.sigma2_from_snr(q, 10.0)
    for _ in range(5):
        c = I.encode(code, rng.integers(0, q, size=(2, code["k"])))
        y = np.zeros(n)
        for k in range(2):
            y[perm[k]] += 2.0 * c[k] - (q - 1)
        y = y.astype(np.float32)
        pe, pb, _, out = _brute_vs_bp(oracle, code, 2, perm, y, sigma2, iters=12)
        unique = np.sort(pe, -1)[..., -1] - np.sort(pe, -1)[..., -2] > 1e-6
        assert (pe.argmax(-1)[unique] == c[unique]).all()
        assert (out["hat"][0][unique] == c[unique]).all()


def test_user_permutation_equivariance(oracle):
    code = I.make_code(64, 4)
    K = 3
    fr = I.make_frames(code, K, 12.0, 6, seed=13)
    rng = np.random.default_rng(1)
    perm = np.stack([rng.permutation(64) for _ in range(K)]).astype(np.int32)
    # re-synthesise y for these interleavers (all users interleaved)
    y = np.zeros((6, 64))
    for k in range(K):
        y[:, perm[k]] += 2.0 * fr["c"][:, k] - 3
    y = (y + rng.normal(size=y.shape) * math.sqrt(fr["sigma2"])).astype(np.float32)
    sig = [2, 0, 1]
    a = oracle.decode(code, K, fr["sigma2"], perm, y, 8, early_stop=False, want_post=True)
    b = oracle.decode(code, K, fr["sigma2"], perm[sig], y, 8, early_stop=False, want_post=True)
    assert (b["hat"] == a["hat"][:, sig]).all()
    assert np.abs(b["post"] - a["post"][:, sig]).max() < 1e-9


def test_early_stop_frames_have_zero_syndrome(oracle):
    code = I.make_code(64, 4)
    fr = I.make_frames(code, 2, 14.0, 60, seed=17)
    out = oracle.decode(code, 2, fr["sigma2"], fr["perm"], fr["y"], 20, early_stop=True)
    stopped = out["iters"] < 20
    assert stopped.any()
    assert out["ok"][stopped].all()
    ok = oracle.syndrome_ok(code, 2, out["hat"])
    assert (ok[stopped] == 1).all()
    full = oracle.decode(code, 2, fr["sigma2"], fr["perm"], fr["y"], 20, early_stop=False)
    assert (full["iters"] == 20).all()


def test_generated_codewords_satisfy_parity(oracle):
    """The generator's encoder (its own GF arithmetic) and the oracle's syndrome
    (shift-and-add GF arithmetic) agree: every codeword has H c = 0."""
    for n, q in [(64, 4), (256, 16), (128, 64)]:
        code = I.make_code(n, q)
        fr = I.make_frames(code, 2, 10.0, 20, seed=n + q)
        assert oracle.syndrome_ok(code, 2, fr["c"]).all()
        bad = fr["c"].copy()
        bad[:, 0, 0] ^= 1
        assert not oracle.syndrome_ok(code, 2, bad)[:, 0].any()


def test_single_steps_compose_to_the_decoder(oracle):
    """The oracle's single-step functions (the references of the GPU step tests)
    run in the flooding schedule (reading R2: channel from c2v^{t-1}, checks from
    v2c = ch2v^t x c2v^{t-1} of the other edge, posterior from ch2v^t and c2v^t,
    c2v^0 uniform) reproduce the whole decoder's messages, posterior, decisions and
    syndrome flags; and v2c then the check update equals the fused check step."""
    K, q, n, T = 3, 8, 24, 4
    code = I.make_code(n, q)
    fr = I.make_frames(code, K, 12.0, 3, seed=29)
    E = code["P"] * code["dc"]
    c2v = np.zeros((3, K, E, q))
    for _ in range(T):
        ch2v = oracle.step_channel(code, K, fr["sigma2"], fr["perm"], fr["y"], c2v)
        v2c = oracle.step_v2c(code, K, ch2v, c2v)
        new = oracle.step_check(code, K, ch2v, c2v)
        assert np.abs(oracle.step_check_v2c(code, K, v2c) - new).max() < 1e-12
        c2v = new
    post, hat = oracle.step_var(code, K, ch2v, c2v)
    full = oracle.decode(code, K, fr["sigma2"], fr["perm"], fr["y"], T, early_stop=False, want_post=True,
                         want_msgs=True)
    assert np.abs(full["ch2v"] - ch2v).max() < 1e-12
    assert np.abs(full["c2v"] - c2v).max() < 1e-12
    assert np.abs(full["post"] - post).max() < 1e-12
    assert np.array_equal(full["hat"], hat)
    assert np.array_equal(full["ok"], oracle.syndrome_ok(code, K, hat))


@pytest.mark.parametrize("q,dc,edges,n", [
    # dc = 3: a chain of three checks; variables 2 and 4 of degree 2, the rest of degree 1
    (4, 3, [0, 1, 2, 2, 3, 4, 4, 5, 6], 7),
    # dc = 6: two checks sharing variable 5 (degree 2); variable 11 has no edge
    (2, 6, [0, 1, 2, 3, 4, 5, 5, 6, 7, 8, 9, 10], 12),
])
def test_bp_is_exact_on_trees_of_other_degrees(oracle, q, dc, edges, n):
    """Check degrees 3 and 6 with irregular variable degrees (0, 1 and 2) on a
    cycle-free single-user graph: BP marginals equal the exact marginals
    (codebook enumeration) -- the oracle's edge walk and check node for
    degrees other than 4 and variable degrees other than 2."""
    rng = np.random.default_rng(q * 31 + dc)
    code = I.code_from_edges(n, q, dc, edges, rng.integers(1, q, len(edges)))
    c = I.encode(code, rng.integers(0, q, size=(1, code["k"])))[0]
    sigma2 = I.sigma2_from_snr(q, 3.0)
    y = (2.0 * c - (q - 1) + rng.normal(size=n) * math.sqrt(sigma2)).astype(np.float32)
    pe, pb, size, _ = _brute_vs_bp(oracle, code, 1, None, y, sigma2, iters=10)
    assert size == q ** (n - len(edges) // dc)
    assert np.abs(pe - pb).max() < 1e-10


def test_bp_is_exact_on_cycle_free_joint_graph_dc3(oracle):
    """Two users, one dc = 3 check each on positions 0..2, interleaved so that the
    joint factor graph is a forest: BP = exact joint marginals."""
    q, n = 4, 6
    rng = np.random.default_rng(77)
    code = I.code_from_edges(n, q, 3, [0, 1, 2], rng.integers(1, q, 3))
    perm = np.stack([np.arange(n), (np.arange(n) + 3) % n]).astype(np.int32)
    fr_c = I.encode(code, rng.integers(0, q, size=(2, code["k"])))
    sigma2 = I.sigma2_from_snr(q, 4.0)
    y = np.zeros(n)
    for k in range(2):
        y[perm[k]] += 2.0 * fr_c[k] - (q - 1)
    y = (y + rng.normal(size=n) * math.sqrt(sigma2)).astype(np.float32)
    pe, pb, size, _ = _brute_vs_bp(oracle, code, 2, perm, y, sigma2, iters=12)
    assert size == q ** (n - 1)
    assert np.abs(pe - pb).max() < 1e-10
