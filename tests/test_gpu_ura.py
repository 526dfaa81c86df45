"""GPU parity of the evidence-interface path (slot-wise AMP detector, SIC row
decoder) against the FP64 oracle, through the C ABI.

Bars:
  * evidence S = log p^ (a log-probability): |gpu - oracle| <= 1e-4 where the
    oracle value is >= ln(1e-4), and <= 1e-4 * |S| below it (FP32 transforms
    and denoiser; the AMP iteration is contracting at these operating points,
    so rounding does not grow across the 20 iterations);
  * SIC rows: decisions bit-exact where the FP64 posterior margin of the row
    exceeds 1e-6; a frame's row k is compared when every earlier row of the
    frame agreed (the cancellation of row k depends on them); iterations and
    syndrome flags of compared rows bit-exact.
"""
import math

import numpy as np
import pytest

from paper_2605_26580_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LOG_MASK = math.log(1e-4)


def _ctx(jbp_lib):
    return jbp_lib.Context(iters=50)


def _evidence_close(S_gpu, S_ref):
    big = S_ref >= LOG_MASK
    err_big = np.abs(S_gpu - S_ref)[big].max() if big.any() else 0.0
    small = ~big
    rel_small = (np.abs(S_gpu - S_ref)[small] / np.abs(S_ref[small])).max() if small.any() else 0.0
    return err_big, rel_small


@pytest.mark.parametrize("L,eb", [(12, 10.0), (48, 10.0), (24, 4.0)])
def test_amp_evidence_matches_oracle(jbp_lib, oracle, L, eb):
    code = I.make_code(L, 64, dv=2, dc=3)
    fr = I.make_ura_frames(code, 2, eb, 64, seed=100 + L)
    ref = oracle.amp_evidence(64, fr["rows"], fr["y"], 20, fr["rho"], fr["su2"])
    ctx = _ctx(jbp_lib)
    dec = jbp_lib.EvidenceDecoder(ctx, code, 2, fr["rows"], fr["rho"], fr["su2"], fr["cancel_log"])
    S = dec.evidence(fr["y"]).astype(np.float64)
    dec.close()
    ctx.close()
    err_big, rel_small = _evidence_close(S, ref)
    print("L=%d Eb=%.0f: max |dS| (S >= ln 1e-4) %.2e, max rel below %.2e" % (L, eb, err_big, rel_small))
    assert err_big <= 1e-4
    assert rel_small <= 1e-4


@pytest.mark.parametrize("q,ns,iters", [(32, 16, 20), (64, 32, 20), (64, 24, 0), (64, 7, 5)])
def test_amp_shapes_match_oracle(jbp_lib, oracle, q, ns, iters):
    code = I.make_code(12, q, dv=2, dc=3)
    fr = I.make_ura_frames(code, 2, 10.0, 16, seed=7, ns=ns)
    ref = oracle.amp_evidence(q, fr["rows"], fr["y"], iters, fr["rho"], fr["su2"])
    ctx = _ctx(jbp_lib)
    dec = jbp_lib.EvidenceDecoder(ctx, code, 2, fr["rows"], fr["rho"], fr["su2"], fr["cancel_log"], amp_iters=iters)
    S = dec.evidence(fr["y"]).astype(np.float64)
    dec.close()
    ctx.close()
    err_big, rel_small = _evidence_close(S, ref)
    assert err_big <= 1e-4 and rel_small <= 1e-4, (err_big, rel_small)


def _compare_sic(got, ref, K):
    """Row-by-row comparison under the margin rule; returns rows compared."""
    F = ref["hat"].shape[0]
    compared = 0
    for f in range(F):
        for k in range(K):
            m = ref["margin"][f, k] > 1e-6
            if not m.all():
                # the row has a near-tie: compare its confident decisions, then stop
                assert np.array_equal(got["hat"][f, k][m], ref["hat"][f, k][m]), (f, k)
                break
            assert np.array_equal(got["hat"][f, k], ref["hat"][f, k]), (f, k)
            assert got["iters"][f, k] == ref["iters"][f, k], (f, k, got["iters"][f, k], ref["iters"][f, k])
            assert got["ok"][f, k] == ref["ok"][f, k], (f, k)
            compared += 1
    return compared


@pytest.mark.parametrize("L,eb,K", [(12, 10.0, 2), (48, 6.0, 2), (24, 4.0, 2), (18, 8.0, 3)])
def test_sic_decode_matches_oracle(jbp_lib, oracle, L, eb, K):
    code = I.make_code(L, 64, dv=2, dc=3)
    fr = I.make_ura_frames(code, K, eb, 96, seed=300 + L)
    S = oracle.amp_evidence(64, fr["rows"], fr["y"], 20, fr["rho"], fr["su2"]).astype(np.float32)
    ref = oracle.sic_decode(code, K, S.astype(np.float64), 50, fr["cancel_log"])
    ctx = _ctx(jbp_lib)
    dec = jbp_lib.EvidenceDecoder(ctx, code, K, fr["rows"], fr["rho"], fr["su2"], fr["cancel_log"])
    got = dec.sic(S)
    dec.close()
    ctx.close()
    n = _compare_sic(got, ref, K)
    print("L=%d Eb=%.0f K=%d: %d of %d rows compared" % (L, eb, K, n, 96 * K))
    assert n >= 0.9 * 96 * K


def test_sic_on_a_peg_code_matches_oracle(jbp_lib, oracle):
    """The progressive-edge-growth code of the paper's PEG-LDPC comparison
    shape (Q=64, L=12, K=2)."""
    code = I.make_peg_code(12, 64)
    fr = I.make_ura_frames(code, 2, 6.0, 96, seed=77)
    S = oracle.amp_evidence(64, fr["rows"], fr["y"], 20, fr["rho"], fr["su2"]).astype(np.float32)
    ref = oracle.sic_decode(code, 2, S.astype(np.float64), 50, fr["cancel_log"])
    ctx = _ctx(jbp_lib)
    dec = jbp_lib.EvidenceDecoder(ctx, code, 2, fr["rows"], fr["rho"], fr["su2"], fr["cancel_log"])
    got = dec.sic(S)
    dec.close()
    ctx.close()
    assert _compare_sic(got, ref, 2) >= 0.9 * 192


def test_sic_other_fields_and_degrees(jbp_lib, oracle):
    """q = 16 with dc = 4 and q = 32 with dc = 3, random evidence, K = 2."""
    for q, dc, n in [(16, 4, 24), (32, 3, 18)]:
        code = I.make_code(n, q, dv=2, dc=dc)
        rng = np.random.default_rng(q)
        S = (rng.standard_normal((40, n, q)) * 3.0).astype(np.float32)
        ref = oracle.sic_decode(code, 2, S.astype(np.float64), 30, -math.log(q))
        ctx = _ctx(jbp_lib)
        dec = jbp_lib.EvidenceDecoder(ctx, code, 2, np.zeros((n, 4), dtype=np.int32) + np.arange(4),
                                      0.1, 1.0, -math.log(q), bp_iters=30)
        got = dec.sic(S)
        dec.close()
        ctx.close()
        assert _compare_sic(got, ref, 2) >= 0.8 * 80


@pytest.mark.parametrize("q,n,bias", [(16, 96, 3.5), (64, 128, 4.5)])
def test_sic_variable_degree_three_matches_oracle(jbp_lib, oracle, q, n, bias):
    """A regular (3, 6) code (rate 1/2): three checks per variable, so each v2c
    leaves one of three incoming messages out and the check node has degree 6."""
    code = I.make_code(n, q, dv=3, dc=6)
    rng = np.random.default_rng(n)
    # evidence that favours one codeword, as a detector would give at moderate SNR
    # (at these strengths most rows converge, some only after many iterations)
    info = rng.integers(0, q, size=(24, code["k"]))
    c = I.encode(code, info)
    S = (rng.standard_normal((24, n, q)) * 1.5).astype(np.float32)
    S[np.arange(24)[:, None], np.arange(n)[None, :], c] += bias
    ref = oracle.sic_decode(code, 1, S.astype(np.float64), 30, -math.log(q))
    ctx = _ctx(jbp_lib)
    dec = jbp_lib.EvidenceDecoder(ctx, code, 1, np.zeros((n, 4), dtype=np.int32) + np.arange(4), 0.1, 1.0,
                                  -math.log(q), bp_iters=30)
    got = dec.sic(S)
    dec.close()
    ctx.close()
    assert _compare_sic(got, ref, 1) >= 0.8 * 24


def test_ura_decode_is_detector_then_decoder_and_matches_oracle_ser(jbp_lib, oracle):
    import torch
    code = I.make_code(24, 64, dv=2, dc=3)
    fr = I.make_ura_frames(code, 2, 6.0, 256, seed=5)
    ctx = _ctx(jbp_lib)
    dec = jbp_lib.EvidenceDecoder(ctx, code, 2, fr["rows"], fr["rho"], fr["su2"], fr["cancel_log"])
    full = dec.decode(fr["y"])
    S = dec.evidence(fr["y"])
    two = dec.sic(S)
    for key in ("hat", "iters", "ok"):
        assert np.array_equal(full[key], two[key])
    # device-pointer path: same results
    dev = torch.device("cuda:0")
    yd = torch.from_numpy(fr["y"]).to(dev)
    hat = torch.empty((256, 2, 24), dtype=torch.uint8, device=dev)
    it = torch.empty((256, 2), dtype=torch.int32, device=dev)
    ok = torch.empty((256, 2), dtype=torch.uint8, device=dev)
    dec.decode_device(yd, hat, it, ok)
    torch.cuda.synchronize()
    assert np.array_equal(hat.cpu().numpy(), full["hat"])
    dec.close()
    ctx.close()
    # matched SER against the transmitted rows equals the oracle pipeline's
    Sref = oracle.amp_evidence(64, fr["rows"], fr["y"], 20, fr["rho"], fr["su2"])
    ref = oracle.sic_decode(code, 2, Sref, 50, fr["cancel_log"])
    sym_g, cw_g = I.match_rows(full["hat"], fr["X"])
    sym_o, cw_o = I.match_rows(ref["hat"], fr["X"])
    print("matched SER gpu %.5f oracle %.5f" % (sym_g.sum() / fr["X"].size, sym_o.sum() / fr["X"].size))
    assert abs(int(sym_g.sum()) - int(sym_o.sum())) <= max(2, 0.01 * fr["X"].size * 0.05)


def test_evidence_path_edge_cases(jbp_lib):
    code = I.make_code(12, 64, dv=2, dc=3)
    fr = I.make_ura_frames(code, 2, 10.0, 4, seed=1)
    ctx = _ctx(jbp_lib)
    dec = jbp_lib.EvidenceDecoder(ctx, code, 2, fr["rows"], fr["rho"], fr["su2"], fr["cancel_log"])
    # F = 0 is a no-op
    assert dec.evidence(fr["y"][:0]).shape == (0, 12, 64)
    assert dec.sic(np.zeros((0, 12, 64), np.float32))["hat"].shape == (0, 2, 12)
    # a single frame, and a ragged batch that is not a multiple of the warps per CTA
    one = dec.decode(fr["y"][:1])
    three = dec.decode(fr["y"][:3])
    assert np.array_equal(one["hat"][0], three["hat"][0])
    dec.close()
    # bad parameters are refused
    bad_rows = fr["rows"].copy()
    bad_rows[0, 1] = bad_rows[0, 0]
    with pytest.raises(jbp_lib.JBPError):
        jbp_lib.EvidenceDecoder(ctx, code, 2, bad_rows, fr["rho"], fr["su2"], fr["cancel_log"])
    with pytest.raises(jbp_lib.JBPError):
        jbp_lib.EvidenceDecoder(ctx, code, 9, fr["rows"], fr["rho"], fr["su2"], fr["cancel_log"])
    with pytest.raises(jbp_lib.JBPError):
        jbp_lib.EvidenceDecoder(ctx, code, 2, fr["rows"], 1.5, fr["su2"], fr["cancel_log"])
    big = I.make_code(512, 64, dv=2, dc=4)
    with pytest.raises(jbp_lib.JBPError):
        jbp_lib.EvidenceDecoder(ctx, big, 2, np.tile(np.arange(24, dtype=np.int32), (512, 1)), 0.03, 20.0,
                                -4.0)
    ctx.close()


@pytest.mark.parametrize("K,n,F", [(1, 12, 40), (2, 12, 64), (3, 1, 64), (5, 300, 20), (8, 24, 6)])
def test_gpu_row_matching_equals_host_alignment(jbp_lib, K, n, F):
    """jbp_match_rows gives the same row-aligned symbol and row errors as the
    host's exhaustive alignment, including its tie rule (a four-letter alphabet
    makes ties common)."""
    rng = np.random.default_rng(K * 1000 + n)
    truth = rng.integers(0, 4, size=(F, K, n)).astype(np.uint8)
    hat = truth[:, rng.permutation(K), :].copy()
    flip = rng.random((F, K, n)) < 0.3
    hat[flip] = rng.integers(0, 4, size=int(flip.sum())).astype(np.uint8)
    ctx = _ctx(jbp_lib)
    try:
        sym, cw = ctx.match_rows(hat, truth)
    finally:
        ctx.close()
    hsym, hcw = I.match_rows(hat, truth)
    assert np.array_equal(sym, hsym) and np.array_equal(cw, hcw)


@pytest.mark.parametrize("L", [12, 48])
def test_evidence_path_many_frames_equal_small_batches(jbp_lib, L):
    """The detector (one warp per slot) and the SIC kernel (one warp per frame) over
    more frames than resident warps, so that warps and their shared memory are
    reused, give bit for bit what the same frames give two at a time (the oracle
    comparisons above use a few frames)."""
    ctx = _ctx(jbp_lib)
    code = I.make_code(L, 64, dv=2, dc=3)
    F = 6000 if L == 12 else 1500
    fr = I.make_ura_frames(code, 2, 10.0, F, seed=800 + L)
    dec = jbp_lib.EvidenceDecoder(ctx, code, 2, fr["rows"], fr["rho"], fr["su2"], fr["cancel_log"])
    try:
        S = dec.evidence(fr["y"])
        rows = dec.sic(S)
        S_small = np.concatenate([dec.evidence(fr["y"][f0:f0 + 2]) for f0 in range(0, F, 2)])
        rows_small = [dec.sic(S[f0:f0 + 2]) for f0 in range(0, F, 2)]
    finally:
        dec.close()
        ctx.close()
    assert np.array_equal(S, S_small)
    for key in ("hat", "iters", "ok"):
        assert np.array_equal(rows[key], np.concatenate([r[key] for r in rows_small])), key
