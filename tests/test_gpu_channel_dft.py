"""Tensor-core channel node (DFT over the symbol-sum alphabet) against the FP64
oracle's trellis.

The transform computes the same extrinsic messages as the trellis (kernel (a))
with two kinds of error.  The user messages mu_j and the window of the Gaussian
score G enter as one FP16 term each: a relative rounding of at most 2^-12 per
value, so each output moves by at most K 2^-12 relative.  The DFT matrices and
the frequency-domain products are hi + lo FP16 terms (about 2^-22) accumulated in
FP32, but the inverse transform cancels terms of the size of the spectrum: with
spectra scaled to DC 1 the accumulated value is L times a probability mass, so
that error is absolute, at most (K + 2) 2^-22 per term over L terms, and rows
whose peak mass is below 2^-12 are handed to the FP32 trellis.  Against the
oracle, max-normalised linear messages therefore differ by at most
(K + 2) 2^-9 + K 2^-12; the tests print the measured value (a few 1e-4).
"""
import math
import time

import numpy as np
import pytest

from paper_2605_26580_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LN_1E4 = math.log(1e-4)


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def env(jbp_lib, oracle):
    return jbp_lib, oracle, _torch()


def _decoder(jbp, code, K, sigma2, perm, iters=20, early_stop=True, channel_node=1):
    ctx = jbp.Context(iters=iters, early_stop=early_stop, channel_node=channel_node)
    return ctx, jbp.Decoder(ctx, code, K, sigma2, perm)


def dft_bound(K):
    return (K + 2) * 2.0 ** -9 + K * 2.0 ** -12


def masked_log_err(gpu, ref, thresh=LN_1E4):
    mask = ref >= thresh
    return float(np.abs(gpu - ref)[mask].max()) if mask.any() else 0.0


def _step_channel(jbp, torch, dec, fr, c2v_lin, K, n, q):
    F = c2v_lin.shape[0]
    y_d = torch.from_numpy(fr["y"]).cuda()
    msg_d = torch.from_numpy(c2v_lin).cuda()
    ch_d = torch.empty((F, K, n, q), dtype=torch.float32, device="cuda")
    dec.step_channel(y_d, msg_d, ch_d)
    torch.cuda.synchronize()
    return ch_d.cpu().numpy().astype(np.float64), msg_d.cpu().numpy().astype(np.float64)


# (K, q, n, F): tiles of 128 channel uses with ragged tails, one and several DFT chunks
DFT_CASES = [
    (2, 16, 64, 7), (4, 16, 256, 5), (3, 32, 64, 9), (4, 64, 120, 3), (7, 32, 32, 11),
    (8, 16, 64, 5), (5, 32, 40, 7), (2, 64, 24, 3), (3, 64, 64, 4),
    (8, 32, 32, 5),                      # K q = 256: the last shape with one pass
    (5, 64, 40, 5), (8, 64, 48, 3),      # K q > 256: users in two passes
]


@pytest.mark.parametrize("K,q,n,F", DFT_CASES)
def test_dft_step_channel_matches_oracle(env, K, q, n, F):
    jbp, O, torch = env
    code = I.make_code(n, q)
    fr = I.make_frames(code, K, 12.0, F, seed=K * 7919 + q * 31 + n)
    rng = np.random.default_rng(n * 13 + q + K)
    E = code["P"] * code["dc"]
    c2v_lin = np.exp(I.random_log_messages(rng, (F, K, E), q, spread=3.0)).astype(np.float32)
    c2v = np.log(c2v_lin.astype(np.float64))
    ctx, dec = _decoder(jbp, code, K, fr["sigma2"], fr["perm"])
    try:
        assert dec.channel_node == jbp.CHAN_DFT
        ch_g, v2c_g = _step_channel(jbp, torch, dec, fr, c2v_lin, K, n, q)
        weak = dec.log_fallbacks()
        assert dec.tc_timeouts() == 0
    finally:
        dec.close()
        ctx.close()
    ch_o = np.exp(O.step_channel(code, K, fr["sigma2"], fr["perm"], fr["y"], c2v))
    lin = float(np.abs(ch_g - ch_o).max())
    # v2c = ch2v * c2v of the other edge, rescaled: the GPU's own ch2v through the oracle's rule
    v2c_o = O.step_v2c(code, K, np.log(ch_g), c2v)
    e_v2c = masked_log_err(np.log(v2c_g), v2c_o)
    print("DFT channel K=%d q=%d n=%d F=%d: linear err %.2e (bound %.2e), rows to trellis %d of %d, v2c err %.2e"
          % (K, q, n, F, lin, dft_bound(K), weak, F * n, e_v2c))
    assert np.isfinite(ch_g).all() and np.isfinite(v2c_g).all()
    assert np.allclose(ch_g.max(-1), 1.0)
    assert lin <= dft_bound(K)
    assert e_v2c <= 1e-4


def test_dft_step_channel_literal_mode(env):
    """interleave = 0 (every user's symbol i on channel use i): the offset table
    comes from identity interleavers; the messages still meet the variant's bar."""
    jbp, O, torch = env
    K, q, n, F = 3, 32, 64, 5
    code = I.make_code(n, q)
    fr = I.make_frames(code, K, 12.0, F, seed=77, interleave=False)
    rng = np.random.default_rng(78)
    E = code["P"] * code["dc"]
    c2v_lin = np.exp(I.random_log_messages(rng, (F, K, E), q, spread=3.0)).astype(np.float32)
    ctx, dec = _decoder(jbp, code, K, fr["sigma2"], None)
    try:
        assert dec.channel_node == jbp.CHAN_DFT
        ch_g, v2c_g = _step_channel(jbp, torch, dec, fr, c2v_lin, K, n, q)
    finally:
        dec.close()
        ctx.close()
    ch_o = np.exp(O.step_channel(code, K, fr["sigma2"], None, fr["y"], np.log(c2v_lin.astype(np.float64))))
    lin = float(np.abs(ch_g - ch_o).max())
    print("DFT channel, literal mode: linear err %.2e (bound %.2e)" % (lin, dft_bound(K)))
    assert lin <= dft_bound(K)


def test_dft_unresolved_rows_go_to_the_trellis(env):
    """Confident messages that make the observed sum (nearly) impossible: the
    transform cannot resolve the peak, so every row is handed to the FP32
    trellis and the messages equal the oracle's in the log domain."""
    jbp, O, torch = env
    K, q, n, F = 4, 64, 64, 3
    code = I.make_code(n, q)
    fr = I.make_frames(code, K, 14.0, F, seed=5)
    E = code["P"] * code["dc"]
    c2v_lin = np.full((F, K, E, q), 1e-12, dtype=np.float32)
    c2v_lin[..., 0] = 1.0                                 # every user believes symbol 0 ...
    fr = dict(fr)
    fr["y"] = np.full((F, n), float(K * (q - 1)), dtype=np.float32)   # ... while y says all are q - 1
    c2v = np.log(c2v_lin.astype(np.float64))
    ctx, dec = _decoder(jbp, code, K, fr["sigma2"], fr["perm"])
    try:
        ch_g, v2c_g = _step_channel(jbp, torch, dec, fr, c2v_lin, K, n, q)
        weak = dec.log_fallbacks()
    finally:
        dec.close()
        ctx.close()
    ch_o = O.step_channel(code, K, fr["sigma2"], fr["perm"], fr["y"], c2v)
    e = masked_log_err(np.log(ch_g), ch_o)
    print("unresolved rows: %d of %d to the trellis, log err %.2e" % (weak, F * n, e))
    assert weak >= F * n
    assert np.isfinite(ch_g).all()
    assert e <= 1e-4


# (K, q, n, F, SNR dB, T, margin): a converging operating point (2 users x 2 bits per
# channel use need about 21 dB), and the past-capacity config-3 shape over few
# iterations (non-converging BP amplifies any rounding by about 2..10 per iteration).
@pytest.mark.parametrize("K,q,n,F,snr,T,margin", [(2, 16, 64, 60, 24.0, 15, 1e-3),
                                                  (4, 64, 128, 24, 14.0, 3, 2e-2)])
def test_dft_decode_agrees_with_oracle(env, K, q, n, F, snr, T, margin):
    """Whole decodes (step form) with the tensor-core channel node: decisions
    agree with the FP64 oracle wherever its margin exceeds `margin`, and the
    symbol error rates agree within the binomial 95% interval."""
    jbp, O, torch = env
    code = I.make_code(n, q)
    fr = I.make_frames(code, K, snr, F, seed=2026 + K + q)
    ctx, dec = _decoder(jbp, code, K, fr["sigma2"], fr["perm"], iters=T, early_stop=True)
    try:
        got = dec.decode(fr["y"])
        assert dec.tc_timeouts() == 0
    finally:
        dec.close()
        ctx.close()
    ref = O.decode(code, K, fr["sigma2"], fr["perm"], fr["y"], T, early_stop=True, want_margin=True)
    diff = got["hat"] != ref["hat"]
    N = diff.size
    ser_g, ser_o = float((got["hat"] != fr["c"]).mean()), float((ref["hat"] != fr["c"]).mean())
    ci = 1.96 * math.sqrt(max(ser_o * (1 - ser_o), 1.0 / N) / N)
    print("DFT decode K=%d q=%d %.0f dB T=%d: SER gpu %.5f oracle %.5f (CI %.5f); differing %d, at margin > %g: %d; "
          "iterations equal in %d of %d frames"
          % (K, q, snr, T, ser_g, ser_o, ci, int(diff.sum()), margin, int((diff & (ref["margin"] > margin)).sum()),
             int((got["iters"] == ref["iters"]).sum()), F))
    assert abs(ser_g - ser_o) <= ci + 1e-12
    assert not (diff & (ref["margin"] > margin)).any()


def test_dft_channel_routing(env):
    """Handles whose (K, q) has a tensor-core shape run it; the others keep the
    trellis; the fused form refuses the DFT node; AUTO keeps the register-resident
    trellis (q <= 16, K <= 4) and takes the transform elsewhere; a bad option is
    refused."""
    jbp, O, torch = env
    ctx = jbp.Context(iters=4, channel_node=jbp.CHAN_DFT)
    try:
        for K, q, n, want in [(4, 64, 64, jbp.CHAN_DFT), (8, 64, 64, jbp.CHAN_DFT),
                              (2, 4, 32, jbp.CHAN_TRELLIS), (1, 64, 32, jbp.CHAN_TRELLIS),
                              (9, 16, 32, jbp.CHAN_TRELLIS), (7, 32, 32, jbp.CHAN_DFT),
                              (8, 32, 32, jbp.CHAN_DFT), (8, 16, 32, jbp.CHAN_DFT)]:
            code = I.make_code(n, q)
            fr = I.make_frames(code, K, 12.0, 2, seed=1)
            dec = jbp.Decoder(ctx, code, K, fr["sigma2"], fr["perm"])
            try:
                assert dec.channel_node == want, (K, q)
                if want == jbp.CHAN_DFT and dec.fused_ok:
                    with pytest.raises(jbp.JBPError) as ei:
                        dec.decode(fr["y"], form=jbp.FORM_FUSED)
                    assert ei.value.code == jbp.EINVAL
                out = dec.decode(fr["y"])            # AUTO runs the step form for the DFT node
                assert out["hat"].shape == (2, K, n)
            finally:
                dec.close()
    finally:
        ctx.close()
    # AUTO: the transform except where the register-resident trellis applies (q <= 16, K <= 4)
    ctx = jbp.Context(iters=4, channel_node=jbp.CHAN_AUTO)
    try:
        for K, q, n, want in [(4, 16, 64, jbp.CHAN_TRELLIS), (2, 16, 32, jbp.CHAN_TRELLIS),
                              (3, 32, 32, jbp.CHAN_DFT), (2, 64, 32, jbp.CHAN_DFT), (5, 16, 32, jbp.CHAN_DFT)]:
            code = I.make_code(n, q)
            fr = I.make_frames(code, K, 12.0, 2, seed=2)
            dec = jbp.Decoder(ctx, code, K, fr["sigma2"], fr["perm"])
            try:
                assert dec.channel_node == want, (K, q)
            finally:
                dec.close()
    finally:
        ctx.close()
    with pytest.raises(jbp.JBPError) as ei:
        jbp.Context(iters=4, channel_node=3)
    assert ei.value.code == jbp.EINVAL


def test_dft_decode_many_graph_replay_matches_single_decodes(env):
    """Parts of different (n, K, q) in one jbp_decode_many call with the DFT node:
    one and two user passes, one and several chunks, and a GF(4) part that keeps
    the trellis.  The eager call, the captured call and a graph replay equal
    individual decodes bit for bit (each channel use's products are independent
    of the other rows in its tile)."""
    jbp, O, torch = env
    specs = [(128, 16, 3, 14.0, 9), (128, 64, 4, 14.0, 5), (64, 64, 6, 14.0, 3), (64, 4, 2, 12.0, 20)]
    ctx = jbp.Context(iters=6, early_stop=True, channel_node=jbp.CHAN_DFT)
    decs, parts, refs = [], [], []
    try:
        for n, q, K, snr, F in specs:
            code = I.make_code(n, q)
            fr = I.make_frames(code, K, snr, F, seed=7 * n + q + K)
            sig = np.full(F, fr["sigma2"], np.float32)
            d = jbp.Decoder(ctx, code, K, fr["sigma2"], fr["perm"])
            decs.append(d)
            refs.append(d.decode(fr["y"], sigma2=sig))
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            parts.append((d, t(fr["y"]), torch.empty((F, K, n), dtype=torch.uint8, device="cuda"),
                          torch.empty((F,), dtype=torch.int32, device="cuda"),
                          torch.empty((F, K), dtype=torch.uint8, device="cuda"), t(sig)))
        assert [d.channel_node for d in decs] == [jbp.CHAN_DFT] * 3 + [jbp.CHAN_TRELLIS]
        for call in range(3):                  # eager, capture, replay
            for p in parts:
                p[2].fill_(255)
            ctx.decode_many(parts)
            torch.cuda.synchronize()
            for p, r in zip(parts, refs):
                assert np.array_equal(p[2].cpu().numpy(), r["hat"]), call
                assert np.array_equal(p[3].cpu().numpy(), r["iters"]), call
                assert np.array_equal(p[4].cpu().numpy(), r["ok"]), call
        assert all(d.tc_timeouts() == 0 for d in decs)
    finally:
        for d in decs:
            d.close()
        ctx.close()


def test_dft_serving_matches_frames_decoded_alone(env):
    """Serving with the DFT node: frames submitted interleaved to two decoders run
    in resident pools (active masks, admission between blocks) and each result
    equals that frame decoded alone in the step form."""
    jbp, O, torch = env
    ctx = jbp.Context(iters=8, early_stop=True, channel_node=jbp.CHAN_DFT)
    specs = [(64, 64, 2, 30.0, 10), (128, 16, 4, 13.0, 12)]
    decs, frames = [], []
    try:
        for n, q, K, snr, F in specs:
            code = I.make_code(n, q)
            fr = I.make_frames(code, K, snr, F, seed=1300 + n)
            decs.append(jbp.Decoder(ctx, code, K, fr["sigma2"], fr["perm"]))
            frames.append(fr)
        assert all(d.channel_node == jbp.CHAN_DFT for d in decs)
        sig = [np.full(fr["y"].shape[0], np.float32(fr["sigma2"]), np.float32) for fr in frames]
        alone = [[d.decode(fr["y"][i:i + 1], form=jbp.FORM_STEP, sigma2=s[i:i + 1]) for i in range(fr["y"].shape[0])]
                 for d, fr, s in zip(decs, frames, sig)]
        tickets = []
        for i in range(max(fr["y"].shape[0] for fr in frames)):
            for j, (d, fr) in enumerate(zip(decs, frames)):
                if i < fr["y"].shape[0]:
                    tickets.append((j, i, d.submit(fr["y"][i], float(sig[j][i]))))
        pending = list(tickets)
        while pending:
            rest = []
            for j, i, tk in pending:
                res = ctx.poll(tk, decs[j].n, decs[j].K)
                if res is None:
                    rest.append((j, i, tk))
                    continue
                a = alone[j][i]
                assert np.array_equal(res["hat"], a["hat"][0]), (j, i)
                assert res["iters"] == int(a["iters"][0]) and np.array_equal(res["ok"], a["ok"][0])
            pending = rest
    finally:
        for d in decs:
            d.close()
        ctx.close()


def test_dft_per_frame_noise_variance(env):
    """jbp_batch.sigma2 with the DFT node: frames of three SNRs in one batch, each
    decoded with its own noise variance (the kernel scores every channel use with
    its frame's sigma2), against the oracle run at that SNR (step form, few
    iterations of the config-3 shape: decisions above margin 2e-2, iterations equal)."""
    jbp, O, torch = env
    K, q, n, T = 4, 64, 64, 3
    code = I.make_code(n, q)
    snrs = [10.0, 14.0, 18.0]
    parts = [I.make_frames(code, K, s, 6, seed=410 + i, perm_seed=410) for i, s in enumerate(snrs)]
    y = np.concatenate([p["y"] for p in parts])
    sig = np.concatenate([np.full(6, p["sigma2"], np.float32) for p in parts])
    ctx, dec = _decoder(jbp, code, K, 1.0, parts[0]["perm"], iters=T, early_stop=True)
    try:
        assert dec.channel_node == jbp.CHAN_DFT
        got = dec.decode(y, sigma2=sig)
    finally:
        dec.close()
        ctx.close()
    for i, p in enumerate(parts):
        ref = O.decode(code, K, float(np.float32(p["sigma2"])), p["perm"], p["y"], T, early_stop=True,
                       want_margin=True)
        sl = slice(6 * i, 6 * (i + 1))
        diff = got["hat"][sl] != ref["hat"]
        print("per-frame sigma2, %.0f dB: %d decisions differ, %d at margin > 2e-2"
              % (snrs[i], int(diff.sum()), int((diff & (ref["margin"] > 2e-2)).sum())))
        assert not (diff & (ref["margin"] > 2e-2)).any()
        assert (got["iters"][sl] == ref["iters"]).all()


def test_dft_not_built_for_variable_degree_three(env):
    """The transform node gathers two c2v messages per variable; a (3, 4) code keeps
    the trellis under JBP_CHAN_DFT."""
    jbp, O, torch = env
    code = I.make_code(64, 16, dv=3, dc=4)
    fr = I.make_frames(code, 4, 12.0, 2, seed=3)
    ctx, dec = _decoder(jbp, code, 4, fr["sigma2"], fr["perm"], iters=2)
    try:
        assert dec.channel_node == jbp.CHAN_TRELLIS
        assert dec.decode(fr["y"])["hat"].shape == (2, 4, 64)
    finally:
        dec.close()
        ctx.close()


@pytest.mark.parametrize("K,q,n,F", [(4, 64, 128, 200), (8, 64, 48, 500), (4, 16, 256, 100)])
def test_dft_many_tiles_equal_small_batches(env, K, q, n, F):
    """A launch of more tiles than CTAs (each CTA runs several tiles: its shared and
    tensor memory, mbarrier phases and DFT-row prefetch carry over) gives, bit for
    bit, what the same frames give two at a time (one tile each, checked against
    the oracle by the tests above): every channel use's products are independent
    of the other rows of its tile."""
    jbp, O, torch = env
    code = I.make_code(n, q)
    fr = I.make_frames(code, K, 14.0, F, seed=500 + K + q)
    rng = np.random.default_rng(501)
    E = code["P"] * code["dc"]
    c2v = np.exp(I.random_log_messages(rng, (F, K, E), q, spread=3.0)).astype(np.float32)
    ctx, dec = _decoder(jbp, code, K, fr["sigma2"], fr["perm"])
    try:
        y_d = torch.from_numpy(fr["y"]).cuda()
        big_msg = torch.from_numpy(c2v).cuda()
        big_ch = torch.empty((F, K, n, q), dtype=torch.float32, device="cuda")
        dec.step_channel(y_d, big_msg, big_ch)
        small_msg = torch.from_numpy(c2v).cuda()
        small_ch = torch.empty_like(big_ch)
        for f0 in range(0, F, 2):
            dec.step_channel(y_d[f0:f0 + 2], small_msg[f0:f0 + 2], small_ch[f0:f0 + 2])
        torch.cuda.synchronize()
        assert dec.tc_timeouts() == 0
        assert torch.equal(big_ch, small_ch)
        assert torch.equal(big_msg, small_msg)
    finally:
        dec.close()
        ctx.close()


def test_auto_serving_small_and_large_pools_match_the_oracle(env):
    """Serving under AUTO: a pool runs the tensor-core channel node only where it
    is faster for the pool's frame count (measured per decoder when its first
    pool is created), so a frame served alone runs the trellis and frames served
    in a burst run the transform.  Either way the results match the oracle:
    decisions where its margin exceeds 2e-2 (the transform's bar, as for the
    config-3 shape), iterations and syndrome flags, on converging frames."""
    jbp, O, torch = env
    K, q, n, T = 4, 64, 64, 8
    code = I.make_code(n, q)
    fr = I.make_frames(code, K, 30.0, 24, seed=1701)
    ctx = jbp.Context(iters=T, early_stop=True, channel_node=jbp.CHAN_AUTO)
    dec = jbp.Decoder(ctx, code, K, fr["sigma2"], fr["perm"])
    got = {}

    def wait(tk):
        deadline = time.time() + 60.0
        while (res := ctx.poll(tk, n, K)) is None:
            assert time.time() < deadline, "served frame not finished within 60 s"
            time.sleep(1e-4)
        return res

    try:
        assert dec.channel_node == jbp.CHAN_DFT
        # one frame at a time (a pool of one frame), then the rest in one burst
        for i in range(4):
            got[i] = wait(dec.submit(fr["y"][i]))
        tickets = [(i, dec.submit(fr["y"][i])) for i in range(4, 24)]
        for i, tk in tickets:
            got[i] = wait(tk)
        assert dec.tc_timeouts() == 0
    finally:
        dec.close()
        ctx.close()
    ref = O.decode(code, K, fr["sigma2"], fr["perm"], fr["y"], T, early_stop=True, want_margin=True)
    for i in range(24):
        sure = ref["margin"][i] > 2e-2
        assert not ((got[i]["hat"] != ref["hat"][i]) & sure).any(), i
        assert got[i]["iters"] == int(ref["iters"][i]), i
        assert np.array_equal(got[i]["ok"], ref["ok"][i]), i
