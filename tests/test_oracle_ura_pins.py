"""Pins of the evidence-interface oracle (AMP detector, single-row FFT-BP with a
prior, SIC over K rows) against quantities fixed independently of it:
quadrature of Bayes' rule, finite differences, the FFT, unitary special cases,
AMP state evolution, the already pinned joint decoder at K = 1, and brute-force
marginals on a cycle-free code."""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_26580_gb300 import inputs as I


def _bg_quadrature(r, nu, rho, su2, half=12.0, h=0.02):
    """Activity posterior and posterior mean of U given R = r by integrating
    the Bernoulli-Gaussian prior against the complex Gaussian likelihood on a
    grid (Bayes' rule, no closed form)."""
    g = np.arange(-half, half + h / 2, h)
    ur, ui = np.meshgrid(g + r.real * su2 / (nu + su2), g + r.imag * su2 / (nu + su2), indexing="ij")
    u = ur + 1j * ui
    like = np.exp(-np.abs(r - u) ** 2 / nu) / (math.pi * nu)
    prior = np.exp(-np.abs(u) ** 2 / su2) / (math.pi * su2)
    w = like * prior * h * h
    p_active = rho * w.sum()
    p_zero = (1 - rho) * math.exp(-abs(r) ** 2 / nu) / (math.pi * nu)
    post = p_active / (p_active + p_zero)
    mean = rho * (u * w).sum() / (p_active + p_zero)
    return post, mean


@pytest.mark.parametrize("r,nu,rho,su2", [(0.3 + 0.2j, 1.0, 0.1, 4.0), (2.5 - 1.0j, 0.7, 0.03, 6.0),
                                         (-1.2 + 3.1j, 1.5, 0.3, 2.0), (0.0 + 0.0j, 1.0, 0.05, 3.0)])
def test_bg_denoiser_equals_bayes_quadrature(r, nu, rho, su2):
    post, mean = _bg_quadrature(r, nu, rho, su2)
    s = abs(r) ** 2
    assert abs(math.exp(O.bg_log_activity(s, nu, rho, su2)) - post) < 1e-7
    eta = O.bg_gain(s, nu, rho, su2) * r
    assert abs(eta - mean) < 1e-6 * max(1.0, abs(mean))


@pytest.mark.parametrize("r,nu,rho,su2", [(0.7 + 0.4j, 1.0, 0.1, 4.0), (3.0 - 2.0j, 0.5, 0.03, 20.0),
                                         (1.1 + 0.1j, 2.0, 0.5, 1.0)])
def test_bg_sensitivity_is_half_divergence(r, nu, rho, su2):
    def eta(z):
        return O.bg_gain(abs(z) ** 2, nu, rho, su2) * z
    d = 1e-5
    dre = (eta(r + d).real - eta(r - d).real) / (2 * d)
    dim = (eta(r + 1j * d).imag - eta(r - 1j * d).imag) / (2 * d)
    assert abs(O.bg_deriv(abs(r) ** 2, nu, rho, su2) - 0.5 * (dre + dim)) < 1e-6


def test_bg_activity_log_is_finite_far_out():
    # |r|^2 / nu = 2000: the densities underflow, their ratio does not
    v = O.bg_log_activity(2000.0, 1.0, 0.03, 20.0)
    assert math.isfinite(v) and v <= 0.0 and v > -1e-6
    w = O.bg_log_activity(0.0, 1.0, 0.03, 20.0)
    assert math.isfinite(w) and w < math.log(0.03) + 1e-12


def test_amp_first_pseudo_observation_is_adjoint_fft():
    """With no iteration, R = A^H y; A = F_{rows,:}/sqrt(ns) with F_{k,a} =
    exp(-2 pi i k a / Q) gives A^H y = Q * ifft(z) / sqrt(ns), z[rows] = y."""
    rng = np.random.default_rng(3)
    Q, ns = 64, 24
    rows = rng.choice(Q, ns, replace=False)
    y = rng.standard_normal((ns, 2)).astype(np.float32)
    _, R, nu = O.amp_slot(Q, rows, y, 0, 0.05, 4.0)
    z = np.zeros(Q, dtype=np.complex128)
    z[rows] = y[:, 0].astype(np.float64) + 1j * y[:, 1].astype(np.float64)
    want = Q * np.fft.ifft(z) / math.sqrt(ns)
    assert np.abs(R - want).max() < 1e-12
    assert abs(nu - float((y.astype(np.float64) ** 2).sum()) / ns) < 1e-12


def test_amp_unitary_dictionary_recovers_noiseless_signal():
    """ns = Q (all rows): A is unitary, so A^H A u = u for a noiseless y."""
    Q = 64
    rows = np.arange(Q)
    u = np.zeros(Q, dtype=np.complex128)
    u[[5, 17, 40]] = [3.0, 3.0 + 1.0j, 6.0]
    y = np.fft.fft(u) / math.sqrt(Q)
    yv = np.stack([y.real, y.imag], -1).astype(np.float32)
    _, R, _ = O.amp_slot(Q, rows, yv, 0, 0.05, 9.0)
    yv64 = yv.astype(np.float64)
    want = Q * np.fft.ifft(yv64[:, 0] + 1j * yv64[:, 1]) / math.sqrt(Q)
    assert np.abs(R - want).max() < 1e-12
    assert np.abs(R - u).max() < 1e-5       # float32 rounding of y only


def test_amp_tracks_state_evolution():
    """AMP on a large i.i.d. complex Gaussian dictionary (entries CN(0, 1/ns)),
    signal drawn from the Bernoulli-Gaussian prior: the residual variance
    nu^(t) follows the state-evolution recursion tau_{t+1} = sigma2 +
    (Q/ns) mmse(tau_t) from tau_0 = nu^(0), with the scalar denoiser's mmse
    estimated by Monte Carlo.  At this size the two agree within 5 %; an
    Onsager term dropped, halved or doubled misses by 18-100 %."""
    rng = np.random.default_rng(11)
    Q, ns, rho, su2, sigma2 = 4096, 2048, 0.08, 1.0, 0.01
    A = (rng.standard_normal((ns, Q)) + 1j * rng.standard_normal((ns, Q))) * math.sqrt(0.5 / ns)
    act = rng.random(Q) < rho
    u = np.where(act, (rng.standard_normal(Q) + 1j * rng.standard_normal(Q)) * math.sqrt(su2 / 2), 0)
    noise = (rng.standard_normal(ns) + 1j * rng.standard_normal(ns)) * math.sqrt(sigma2 / 2)
    y = A @ u + noise
    yv = np.stack([y.real, y.imag], -1).astype(np.float32)
    M = 20000
    mrng = np.random.default_rng(12)
    U = np.where(mrng.random(M) < rho,
                 (mrng.standard_normal(M) + 1j * mrng.standard_normal(M)) * math.sqrt(su2 / 2), 0)
    Z = (mrng.standard_normal(M) + 1j * mrng.standard_normal(M)) * math.sqrt(0.5)

    def mmse(tau):
        Rs = U + math.sqrt(tau) * Z
        g = np.array([O.bg_gain(s, tau, rho, su2) for s in np.abs(Rs) ** 2])
        return float(np.mean(np.abs(g * Rs - U) ** 2))

    _, _, tau = O.amp_dict(A, yv, 0, rho, su2)
    for t in range(1, 7):
        tau = sigma2 + (Q / ns) * mmse(tau)
        _, _, nu = O.amp_dict(A, yv, t, rho, su2)
        assert abs(nu - tau) < 0.08 * tau, (t, nu, tau)


def test_amp_slot_is_amp_on_the_partial_dft():
    """or_amp_slot = or_amp_dict with A = F_{rows,:}/sqrt(ns) built here from
    numpy's DFT matrix."""
    rng = np.random.default_rng(13)
    Q, ns = 64, 24
    rows = rng.choice(Q, ns, replace=False)
    A = np.fft.fft(np.eye(Q))[rows] / math.sqrt(ns)
    y = (rng.standard_normal((ns, 2)) * 3).astype(np.float32)
    a = O.amp_slot(Q, rows, y, 20, 2 / 64, 20.0)
    b = O.amp_dict(A, y, 20, 2 / 64, 20.0)
    assert np.abs(a[0] - b[0]).max() < 1e-9
    assert np.abs(a[1] - b[1]).max() < 1e-9


def test_evidence_is_the_activity_log_of_the_final_pseudo_observation():
    """Evidence interface: S_a = log p^(|R_a|^2; nu) of the last AMP iterate (eq.
    bg_activity_prob at the detector's output), and the batched evidence
    [F, L, Q] is the per-slot detector run on each frame's slot with that slot's
    rows (layout of y: [F, L, ns, 2])."""
    rng = np.random.default_rng(21)
    Q, ns, L, F = 64, 24, 3, 2
    rho, su2 = 2 / 64, 30.0
    rows = np.stack([rng.choice(Q, ns, replace=False) for _ in range(L)]).astype(np.int32)
    y = (rng.standard_normal((F, L, ns, 2)) * 3).astype(np.float32)
    S_all = O.amp_evidence(Q, rows, y, 20, rho, su2, threads=2)
    for f in range(F):
        for l in range(L):
            S, R, nu = O.amp_slot(Q, rows[l], y[f, l], 20, rho, su2)
            ref = np.array([O.bg_log_activity(abs(R[a]) ** 2, nu, rho, su2) for a in range(Q)])
            assert np.abs(S - ref).max() < 1e-12
            assert np.array_equal(S_all[f, l], S)


def _gf4_code_tree():
    # two checks of degree 3 sharing variable 2: a tree (no cycle)
    chk_var = np.array([0, 1, 2, 2, 3, 4], dtype=np.int32)
    chk_coef = np.array([1, 2, 3, 2, 1, 3], dtype=np.int32)
    return I.code_from_edges(5, 4, 3, chk_var, chk_coef)


def test_bp_prior_on_tree_equals_enumeration():
    code = _gf4_code_tree()
    rng = np.random.default_rng(5)
    S = rng.standard_normal((1, 5, 4)) * 2.0
    out = O.bp_prior(code, S, 6, early_stop=False, want_post=True)
    m = 2
    words = []
    for w in itertools.product(range(4), repeat=5):
        ok = True
        for j in range(2):
            s = 0
            for d in range(3):
                e = 3 * j + d
                s ^= O.gf_mul(m, int(code["chk_coef"][e]), w[int(code["chk_var"][e])])
            ok &= (s == 0)
        if ok:
            words.append(w)
    lam = S[0] - S[0].max(axis=1, keepdims=True)
    marg = np.zeros((5, 4))
    for w in words:
        p = math.exp(sum(lam[i, w[i]] for i in range(5)))
        for i in range(5):
            marg[i, w[i]] += p
    want = np.log(marg) - np.log(marg).max(axis=1, keepdims=True)
    assert np.abs(out["post"][0] - want).max() < 1e-10


def test_bp_prior_equals_joint_decoder_at_one_user():
    """K = 1 joint BP feeds the Gaussian likelihood as the local belief; the
    same belief given as evidence must give the same decode."""
    q, n = 16, 24
    code = I.make_code(n, q, dv=2, dc=3)
    fr = I.make_frames(code, 1, 4.0, 6, seed=77)
    y = fr["y"].astype(np.float64)
    lev = 2.0 * np.arange(q) - (q - 1)
    S = -(y[:, :, None] - lev[None, None, :]) ** 2 / (2 * fr["sigma2"])
    joint = O.decode(code, 1, fr["sigma2"], fr["perm"], fr["y"], 20, want_post=True)
    mine = O.bp_prior(code, S, 20, want_post=True)
    assert np.array_equal(joint["hat"][:, 0], mine["hat"])
    assert np.array_equal(joint["iters"], mine["iters"])
    assert np.abs(joint["post"][:, 0] - mine["post"]).max() < 1e-9


def test_sic_one_row_equals_bp_prior():
    code = I.make_code(12, 64, dv=2, dc=3)
    S = np.random.default_rng(8).standard_normal((5, 12, 64)) * 3.0
    a = O.sic_decode(code, 1, S, 30, -math.log(64))
    b = O.bp_prior(code, S, 30)
    assert np.array_equal(a["hat"][:, 0], b["hat"])
    assert np.array_equal(a["iters"][:, 0], b["iters"])


def test_sic_cancels_the_decoded_row():
    """Evidence that favours codeword c0 and, less strongly, c1: the first row
    is c0; after cancellation the second is c1 (without it, c0 again)."""
    code = I.make_code(12, 64, dv=2, dc=3)
    info = np.random.default_rng(9).integers(0, 64, size=(2, code["k"]))
    c = I.encode(code, info)
    S = np.full((1, 12, 64), -20.0)
    S[0, np.arange(12), c[1]] = -0.5
    S[0, np.arange(12), c[0]] = 0.0
    out = O.sic_decode(code, 2, S, 30, -math.log(64))
    assert np.array_equal(out["hat"][0, 0], c[0])
    assert np.array_equal(out["hat"][0, 1], c[1])
    same = O.sic_decode(code, 2, S, 30, 0.0)
    assert np.array_equal(same["hat"][0, 1], c[0])


def test_ura_pipeline_decodes_high_snr_frames():
    """At E_b/N_0 = 12 dB every frame decodes to the transmitted rows (after
    row matching).  Noiseless frames are not used: their two rows give exactly
    equal evidence in every slot, so the first row's BP has no reason to pick
    either codeword and does not converge."""
    code = I.make_code(12, 64, dv=2, dc=3)
    fr = I.make_ura_frames(code, 2, 12.0, 40, seed=4)
    S = O.amp_evidence(64, fr["rows"], fr["y"], 20, fr["rho"], fr["su2"])
    out = O.sic_decode(code, 2, S, 50, fr["cancel_log"])
    sym, cw = I.match_rows(out["hat"], fr["X"])
    assert sym.sum() == 0 and cw.sum() == 0
    assert out["ok"].all()


def test_match_rows_counts_errors_after_alignment():
    X = np.array([[[1, 2, 3], [4, 5, 6]]])
    hat = np.array([[[4, 5, 0], [1, 2, 3]]])
    sym, cw = I.match_rows(hat, X)
    assert sym[0] == 1 and cw[0] == 1
