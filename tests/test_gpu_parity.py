"""GPU parity: every kernel of the decoder against the FP64 oracle on the same
seeded inputs, through the C ABI.

The kernels store messages as FP32 probabilities scaled to max 1; the tests
feed them exp() of seeded log-messages and compare ln() of their outputs with
the oracle's log-messages computed from the very same float32 inputs.

Tolerances (derived in the design notes, "Parity bar"):
  * channel, v2c and posterior log-messages: |gpu - oracle| <= 1e-4 wherever the
    oracle entry is >= ln(1e-4) (FP32 trellis and sums have no cancellation);
    below that both must be < ln(1e-4) + 1e-4;
  * check-node c2v (FP32 Walsh-Hadamard butterflies): in the linear domain
    |exp(gpu) - exp(oracle)| <= B_q = q (4 log2 q + 2) 2^-24 (forward transform,
    product and inverse transform error relative to the largest entry); in the
    log domain, for every entry with oracle probability rho >= 1e-4 (relative
    to the max), |gpu - oracle| <= 1e-4 + 2 B_q / rho (a linear error B_q is a
    relative error B_q / rho at that entry; the cancellation of the transform
    makes small entries less accurate than large ones);
  * hard decisions bit-exact wherever the FP64 posterior margin p(1) - p(2) > 1e-6;
  * syndromes bit-exact.
"""
import math

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


def wht_bound(q):
    return q * (4 * math.log2(q) + 2) * 2.0 ** -24


def masked_log_err(gpu, ref, thresh=LN_1E4):
    gpu = np.asarray(gpu, dtype=np.float64)
    mask = ref >= thresh
    err_in = np.abs(gpu - ref)[mask].max() if mask.any() else 0.0
    # outside the mask both must be small
    outside_ok = bool(np.all(gpu[~mask] < thresh + 1e-4)) if (~mask).any() else True
    return err_in, outside_ok


@pytest.fixture(scope="module")
def env(jbp_lib, oracle):
    torch = _torch()
    return jbp_lib, oracle, torch


def _decoder(jbp, code, K, sigma2, perm, iters=20, early_stop=True, precision=0):
    ctx = jbp.Context(iters=iters, early_stop=early_stop, precision=precision)
    dec = jbp.Decoder(ctx, code, K, sigma2, perm)
    return ctx, dec


STEP_CASES = [  # (K, q, n)
    (2, 4, 64), (4, 16, 256), (3, 8, 64), (1, 16, 64), (4, 64, 128), (8, 16, 64), (16, 4, 32), (2, 2, 24),
    (5, 32, 40),
]


@pytest.mark.parametrize("K,q,n", STEP_CASES)
def test_step_channel_matches_oracle(env, K, q, n):
    jbp, O, torch = env
    code = I.make_code(n, q)
    fr = I.make_frames(code, K, 12.0, 7, seed=K * 1000 + q + n)
    rng = np.random.default_rng(n + q)
    E = code["P"] * code["dc"]
    c2v_lin = np.exp(I.random_log_messages(rng, (7, K, E), q, spread=3.0)).astype(np.float32)
    c2v = np.log(c2v_lin.astype(np.float64))
    ctx, dec = _decoder(jbp, code, K, fr["sigma2"], fr["perm"])
    try:
        y_d = torch.from_numpy(fr["y"]).cuda()
        msg_d = torch.from_numpy(c2v_lin).cuda()
        ch_d = torch.empty((7, K, n, q), dtype=torch.float32, device="cuda")
        dec.step_channel(y_d, msg_d, ch_d)
        torch.cuda.synchronize()
        ch_g, v2c_g = np.log(ch_d.cpu().numpy().astype(np.float64)), np.log(msg_d.cpu().numpy().astype(np.float64))
    finally:
        dec.close()
        ctx.close()
    ch_o = O.step_channel(code, K, fr["sigma2"], fr["perm"], fr["y"], c2v)
    v2c_o = O.step_v2c(code, K, ch_o, c2v)
    e1, ok1 = masked_log_err(ch_g, ch_o)
    e2, ok2 = masked_log_err(v2c_g, v2c_o)
    print("channel K=%d q=%d n=%d: ch2v err %.2e, v2c err %.2e" % (K, q, n, e1, e2))
    assert e1 <= 1e-4 and ok1
    assert e2 <= 1e-4 and ok2


@pytest.mark.parametrize("K,q,n", STEP_CASES)
def test_step_check_matches_oracle(env, K, q, n):
    jbp, O, torch = env
    code = I.make_code(n, q)
    rng = np.random.default_rng(3 * n + q)
    E = code["P"] * code["dc"]
    v2c_lin = np.exp(I.random_log_messages(rng, (5, K, E), q, spread=3.0)).astype(np.float32)
    ctx, dec = _decoder(jbp, code, K, 1.0, None)
    try:
        msg_d = torch.from_numpy(v2c_lin).cuda()
        dec.step_check(msg_d)
        torch.cuda.synchronize()
        c2v_g = np.log(msg_d.cpu().numpy().astype(np.float64))
    finally:
        dec.close()
        ctx.close()
    c2v_o = O.step_check_v2c(code, K, np.log(v2c_lin.astype(np.float64)))
    B = wht_bound(q)
    lin = np.abs(np.exp(c2v_g) - np.exp(c2v_o)).max()
    rho = np.exp(c2v_o)
    mask = rho >= 1e-4
    ratio = (np.abs(c2v_g - c2v_o)[mask] / (1e-4 + 2 * B / rho[mask])).max()
    e_log4, _ = masked_log_err(c2v_g, c2v_o)
    e_big, _ = masked_log_err(c2v_g, c2v_o, thresh=math.log(0.5))
    print("check K=%d q=%d: linear err %.2e (bound %.2e), log err %.2e (rho>=0.5), %.2e (rho>=1e-4), "
          "err/allowed %.3f" % (K, q, lin, B, e_big, e_log4, ratio))
    assert lin <= B
    assert ratio <= 1.0
    assert np.allclose(c2v_g.max(-1), 0.0, atol=1e-6)
    assert c2v_g.min() >= math.log(1e-12) - 1e-3


@pytest.mark.parametrize("K,q,n", [(2, 4, 64), (4, 16, 256), (3, 64, 64), (1, 2, 16)])
def test_step_var_and_syndrome_match_oracle(env, K, q, n):
    jbp, O, torch = env
    code = I.make_code(n, q)
    rng = np.random.default_rng(5 * n + q)
    E = code["P"] * code["dc"]
    ch2v_lin = np.exp(I.random_log_messages(rng, (6, K, n), q, spread=2.0)).astype(np.float32)
    c2v_lin = np.exp(I.random_log_messages(rng, (6, K, E), q, spread=2.0)).astype(np.float32)
    ch2v, c2v = np.log(ch2v_lin.astype(np.float64)), np.log(c2v_lin.astype(np.float64))
    ctx, dec = _decoder(jbp, code, K, 1.0, None)
    try:
        ch_d, msg_d = torch.from_numpy(ch2v_lin).cuda(), torch.from_numpy(c2v_lin).cuda()
        post_d = torch.empty_like(ch_d)
        hat_d = torch.empty((6, K, n), dtype=torch.uint8, device="cuda")
        dec.step_var(ch_d, msg_d, post_d, hat_d)
        # syndromes of the decisions and of true codewords
        cw = I.make_frames(code, K, 10.0, 6, seed=1)["c"]
        cw_d = torch.from_numpy(cw).cuda()
        ok_hat = torch.empty((6, K), dtype=torch.uint8, device="cuda")
        ok_cw = torch.empty((6, K), dtype=torch.uint8, device="cuda")
        dec.step_syndrome(hat_d, ok_hat)
        dec.step_syndrome(cw_d, ok_cw)
        torch.cuda.synchronize()
        post_g, hat_g = post_d.cpu().numpy(), hat_d.cpu().numpy()
        okh, okc = ok_hat.cpu().numpy(), ok_cw.cpu().numpy()
    finally:
        dec.close()
        ctx.close()
    post_o, hat_o = O.step_var(code, K, ch2v, c2v)
    e, _ = masked_log_err(post_g, post_o)
    assert e <= 1e-4
    p = np.exp(post_o)
    p /= p.sum(-1, keepdims=True)
    ps = np.sort(p, -1)
    sure = (ps[..., -1] - ps[..., -2]) > 1e-6
    assert (hat_g[sure] == hat_o[sure]).all()
    assert (okh == O.syndrome_ok(code, K, hat_g)).all()
    assert okc.all()


def _margin_mismatch(got, ref):
    sure = ref["margin"] > 1e-6
    return int(((got["hat"] != ref["hat"]) & sure).sum()), int(sure.sum())


@pytest.mark.parametrize("form", ["fused", "step"])
def test_decode_config1_matches_oracle(env, form):
    """K=2, GF(4), n=64, SNR 10 dB, 20 flooding iterations, 1,000 frames."""
    jbp, O, torch = env
    code = I.make_code(64, 4)
    fr = I.make_frames(code, 2, 10.0, 1000, seed=1_000_000_000)
    ctx, dec = _decoder(jbp, code, 2, fr["sigma2"], fr["perm"], iters=20, early_stop=False)
    try:
        got = dec.decode(fr["y"], form=jbp.FORM_FUSED if form == "fused" else jbp.FORM_STEP)
    finally:
        dec.close()
        ctx.close()
    ref = O.decode(code, 2, fr["sigma2"], fr["perm"], fr["y"], 20, early_stop=False, want_margin=True)
    bad, total = _margin_mismatch(got, ref)
    frames_bad = int(((got["hat"] != ref["hat"]) & (ref["margin"] > 1e-6)).any((1, 2)).sum())
    ser_g = (got["hat"] != fr["c"]).mean()
    ser_o = (ref["hat"] != fr["c"]).mean()
    print("config1 %s: %d/%d confident decisions differ (%d frames); SER gpu %.5f oracle %.5f"
          % (form, bad, total, frames_bad, ser_g, ser_o))
    assert (got["iters"] == 20).all()
    assert bad == 0
    assert (got["ok"] == ref["ok"]).all()


def test_forms_agree(env):
    """STEP and PLAIN run the same kernels: bit-identical.  FUSED runs the
    register-resident thread shape (another association order of the same sums):
    its decisions equal the oracle's wherever the FP64 margin exceeds 1e-6."""
    jbp, O, torch = env
    code = I.make_code(64, 16)
    fr = I.make_frames(code, 3, 12.0, 37, seed=77)
    ctx, dec = _decoder(jbp, code, 3, fr["sigma2"], fr["perm"], iters=15, early_stop=True)
    try:
        a = dec.decode(fr["y"], form=jbp.FORM_FUSED, want_post=True)
        b = dec.decode(fr["y"], form=jbp.FORM_STEP, want_post=True)
        c = dec.decode(fr["y"][:5], form=jbp.FORM_PLAIN, want_post=True)
    finally:
        dec.close()
        ctx.close()
    for key in ("hat", "iters", "ok", "post"):
        assert np.array_equal(b[key][:5], c[key]), key
    ref = O.decode(code, 3, fr["sigma2"], fr["perm"], fr["y"], 15, early_stop=True, want_margin=True)
    for got in (a, b):
        bad, _ = _margin_mismatch(got, ref)
        assert bad == 0
        assert (got["iters"] == ref["iters"]).all()


@pytest.mark.parametrize("K,q,n,F,T", [(1, 2, 12, 1, 3), (4, 16, 256, 153, 6), (16, 4, 32, 9, 4),
                                       (3, 64, 64, 5, 3), (2, 8, 12, 40, 8), (6, 32, 48, 3, 3)])
def test_decode_edge_shapes_match_oracle(env, K, q, n, F, T):
    """Single frame, ragged batches, K = 1 and K = 16, q = 2 and q = 64, tiny n."""
    jbp, O, torch = env
    code = I.make_code(n, q)
    fr = I.make_frames(code, K, 14.0, F, seed=F * 7 + K)
    ctx, dec = _decoder(jbp, code, K, fr["sigma2"], fr["perm"], iters=T, early_stop=True)
    try:
        got = dec.decode(fr["y"])
        empty = dec.decode(np.zeros((0, n), np.float32))
    finally:
        dec.close()
        ctx.close()
    ref = O.decode(code, K, fr["sigma2"], fr["perm"], fr["y"], T, early_stop=True, want_margin=True)
    bad, _ = _margin_mismatch(got, ref)
    assert bad == 0
    assert (got["iters"] == ref["iters"]).all()
    assert empty["hat"].shape == (0, K, n)


def test_literal_channel_mode(env):
    """interleave = 0 (every pi_k the identity): the users are exchangeable, so
    their posteriors are identical and often nearly tied; decisions must agree
    where the FP64 margin exceeds 1e-4 (FP32 rounding accumulated over the
    iterations can flip a near-tie between 1e-6 and 1e-4; the count is printed)."""
    jbp, O, torch = env
    code = I.make_code(64, 4)
    fr = I.make_frames(code, 2, 12.0, 50, seed=5, interleave=False)
    ctx = jbp.Context(iters=10, early_stop=False)
    dec = jbp.Decoder(ctx, code, 2, fr["sigma2"], None, interleave=False)
    try:
        got = dec.decode(fr["y"])
    finally:
        dec.close()
        ctx.close()
    ref = O.decode(code, 2, fr["sigma2"], None, fr["y"], 10, early_stop=False, want_margin=True)
    diff = got["hat"] != ref["hat"]
    print("literal mode: differing decisions at FP64 margins", np.sort(ref["margin"][diff])[:10])
    assert not (diff & (ref["margin"] > 1e-4)).any()
    assert (got["hat"][:, 0] == got["hat"][:, 1]).all()   # symmetric users, identical decisions


def tc_bound(prec, q):
    """Linear error bound (relative to the largest entry) of the tensor-core check
    node: the FP32 butterfly bound plus the operand split error.  One BF16 term
    keeps 8 significant bits (2^-9 relative), two keep 16 (2^-17), three about
    24; the split error enters the forward input, the product (three factors,
    to first order one each) and the inverse input: 4 q u_split."""
    u = {3: 2.0 ** -25, 1: 2.0 ** -17, 2: 2.0 ** -9}[prec]
    return 2 * wht_bound(q) + 4 * q * u


@pytest.mark.parametrize("prec", [3, 1, 2])
@pytest.mark.parametrize("K,q,n", [(4, 16, 256), (2, 64, 128), (3, 32, 64), (1, 16, 40)])
def test_step_check_tensor_cores(env, prec, K, q, n):
    """tcgen05 check node (BF16X3 / BF16X2 / BF16 operand splits) against the oracle."""
    jbp, O, torch = env
    code = I.make_code(n, q)
    rng = np.random.default_rng(11 * n + q + prec)
    E = code["P"] * code["dc"]
    F = 5
    v2c_lin = np.exp(I.random_log_messages(rng, (F, K, E), q, spread=3.0)).astype(np.float32)
    ctx, dec = _decoder(jbp, code, K, 1.0, None)
    try:
        msg_d = torch.from_numpy(v2c_lin).cuda()
        dec.step_check(msg_d, precision=prec)
        torch.cuda.synchronize()
        c2v_g = np.log(msg_d.cpu().numpy().astype(np.float64))
        assert dec.tc_timeouts() == 0
    finally:
        dec.close()
        ctx.close()
    c2v_o = O.step_check_v2c(code, K, np.log(v2c_lin.astype(np.float64)))
    lin = np.abs(np.exp(c2v_g) - np.exp(c2v_o)).max()
    e_big, _ = masked_log_err(c2v_g, c2v_o, thresh=math.log(0.5))
    e_log4, _ = masked_log_err(c2v_g, c2v_o)
    B = tc_bound(prec, q)
    print("tensor-core check prec=%d K=%d q=%d: linear err %.2e (bound %.2e), log err %.2e (rho>=0.5), %.2e (rho>=1e-4)"
          % (prec, K, q, lin, B, e_big, e_log4))
    assert np.isfinite(c2v_g).all()
    assert lin <= B
    assert np.allclose(c2v_g.max(-1), 0.0, atol=1e-5)


@pytest.mark.parametrize("prec", [3, 1, 2])
def test_decode_precision_variants(env, prec):
    """Whole decodes with the tensor-core check node (step form): BF16X3 keeps the
    decisions of the FP32 oracle wherever the margin exceeds 1e-3; BF16X2 and BF16
    are reported (SER against the oracle's)."""
    jbp, O, torch = env
    code = I.make_code(64, 16)
    fr = I.make_frames(code, 2, 16.0, 60, seed=91)
    ctx, dec = _decoder(jbp, code, 2, fr["sigma2"], fr["perm"], iters=12, early_stop=True, precision=prec)
    try:
        got = dec.decode(fr["y"])
    finally:
        dec.close()
        ctx.close()
    ref = O.decode(code, 2, fr["sigma2"], fr["perm"], fr["y"], 12, early_stop=True, want_margin=True)
    diff = got["hat"] != ref["hat"]
    ser_g, ser_o = (got["hat"] != fr["c"]).mean(), (ref["hat"] != fr["c"]).mean()
    print("precision %d: SER gpu %.5f oracle %.5f; decisions differing at margin > 1e-3: %d"
          % (prec, ser_g, ser_o, int((diff & (ref["margin"] > 1e-3)).sum())))
    if prec == 3:
        assert not (diff & (ref["margin"] > 1e-3)).any()


def test_per_frame_noise_variance_matches_oracle(env):
    """jbp_batch.sigma2: each frame decoded with its own SNR equals the oracle run
    at that SNR."""
    jbp, O, torch = env
    code = I.make_code(64, 4)
    snrs = [9.0, 12.0, 15.0]
    parts = [I.make_frames(code, 2, s, 20, seed=300 + i, perm_seed=300) for i, s in enumerate(snrs)]
    y = np.concatenate([p["y"] for p in parts])
    sig = np.concatenate([np.full(20, p["sigma2"], np.float32) for p in parts])
    ctx, dec = _decoder(jbp, code, 2, 1.0, parts[0]["perm"], iters=15, early_stop=True)
    try:
        got = dec.decode(y, sigma2=sig)
        got_step = dec.decode(y, sigma2=sig, form=jbp.FORM_STEP)
    finally:
        dec.close()
        ctx.close()
    for i, p in enumerate(parts):
        ref = O.decode(code, 2, float(np.float32(p["sigma2"])), p["perm"], p["y"], 15, early_stop=True,
                       want_margin=True)
        for g in (got, got_step):
            sl = slice(20 * i, 20 * (i + 1))
            diff = g["hat"][sl] != ref["hat"]
            assert not (diff & (ref["margin"] > 1e-6)).any()
            assert (g["iters"][sl] == ref["iters"]).all()


def test_decode_many_graph_replay_matches_single_decodes(env):
    """Three decoders of different (n, K, q) -- two fused, one in the HBM step form --
    in one jbp_decode_many call: the eager call, the captured call and a graph
    replay all equal individual decodes, bit for bit."""
    jbp, O, torch = env
    specs = [(64, 4, 2, 12.0, 40), (128, 16, 3, 14.0, 25), (256, 64, 4, 14.0, 6)]
    ctx = jbp.Context(iters=8, early_stop=True)
    decs, parts, refs = [], [], []
    try:
        for n, q, K, snr, F in specs:
            code = I.make_code(n, q)
            fr = I.make_frames(code, K, snr, F, seed=n + q + K)
            sig = np.full(F, fr["sigma2"], np.float32)
            d = jbp.Decoder(ctx, code, K, fr["sigma2"], fr["perm"])
            decs.append(d)
            refs.append(d.decode(fr["y"], sigma2=sig))
            t = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            parts.append((d, t(fr["y"]), torch.empty((F, K, n), dtype=torch.uint8, device="cuda"),
                          torch.empty((F,), dtype=torch.int32, device="cuda"),
                          torch.empty((F, K), dtype=torch.uint8, device="cuda"), t(sig)))
        assert not decs[2].fused_ok
        for call in range(3):                  # eager, capture, replay
            for p in parts:
                p[2].fill_(255)
            ctx.decode_many(parts)
            torch.cuda.synchronize()
            for p, r in zip(parts, refs):
                assert np.array_equal(p[2].cpu().numpy(), r["hat"]), call
                assert np.array_equal(p[3].cpu().numpy(), r["iters"]), call
                assert np.array_equal(p[4].cpu().numpy(), r["ok"]), call
    finally:
        for d in decs:
            d.close()
        ctx.close()


def test_serving_results_are_the_same_alone_and_in_the_mix(env):
    """Requests of two decoders submitted interleaved (resident pools re-batched
    every block of iterations, the two pools' blocks overlapping) give, frame by
    frame, exactly the result of decoding that frame alone in the form its pool
    runs -- the fused form here (GF(q <= 16), K <= 4, variable degree 2: the pool
    keeps each slot's state in the fused kernel's layout); unknown or consumed
    tickets poll JBP_ECLOSED."""
    jbp, O, torch = env
    ctx = jbp.Context(iters=10, early_stop=True)
    specs = [(64, 4, 2, 11.0, 24), (128, 16, 3, 13.0, 16)]
    decs, frames = [], []
    try:
        for n, q, K, snr, F in specs:
            code = I.make_code(n, q)
            fr = I.make_frames(code, K, snr, F, seed=900 + n)
            decs.append(jbp.Decoder(ctx, code, K, fr["sigma2"], fr["perm"]))
            frames.append(fr)
        sig = [np.full(fr["y"].shape[0], np.float32(fr["sigma2"]), np.float32) for fr in frames]
        alone = [[d.decode(fr["y"][i:i + 1], form=jbp.FORM_FUSED, sigma2=s[i:i + 1]) for i in range(fr["y"].shape[0])]
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
        with pytest.raises(jbp.JBPError) as ei:
            ctx.poll(tickets[0][2], decs[0].n, decs[0].K)
        assert ei.value.code == jbp.ECLOSED
        st = ctx.serving_stats()
        assert st["completed"] == len(tickets) and st["p99_us"] >= st["p50_us"] > 0
    finally:
        for d in decs:
            d.close()
        ctx.close()


def test_serving_admits_frames_between_blocks(env):
    """Frames submitted while earlier frames of the same decoder are part-way
    through their iterations join the resident pool at the next block boundary;
    every result equals the frame decoded alone (fused form, which the pool of
    this decoder runs, its slots' state stored between blocks of 2 iterations),
    and the iteration counts show the early frames were not restarted."""
    import time
    jbp, O, torch = env
    ctx = jbp.Context(iters=30, early_stop=False, block_iters=2)
    code = I.make_code(256, 16)
    fr = I.make_frames(code, 4, 10.0, 48, seed=1234)
    dec = jbp.Decoder(ctx, code, 4, fr["sigma2"], fr["perm"])
    try:
        alone = [dec.decode(fr["y"][i:i + 1], form=jbp.FORM_FUSED) for i in range(48)]
        first = [dec.submit(fr["y"][i]) for i in range(16)]
        time.sleep(0.002)
        second = [dec.submit(fr["y"][i]) for i in range(16, 48)]
        for i, tk in enumerate(first + second):
            while True:
                res = ctx.poll(tk, 256, 4)
                if res is not None:
                    break
                time.sleep(0.0005)
            assert np.array_equal(res["hat"], alone[i]["hat"][0]), i
            assert res["iters"] == 30 and np.array_equal(res["ok"], alone[i]["ok"][0])
        assert ctx.serving_stats()["completed"] == 48
    finally:
        dec.close()
        ctx.close()


@pytest.mark.parametrize("form", ["auto", "step"])
def test_variable_degree_three_matches_oracle(env, form):
    """A regular (3, 4) code: every variable has three checks, so the channel
    node's incoming message is the product of three c2v and each v2c leaves one
    of three out (the step form's team path and generic variable node)."""
    jbp, O, torch = env
    code = I.make_code(64, 16, dv=3, dc=4)
    fr = I.make_frames(code, 3, 12.0, 24, seed=31)
    ctx, dec = _decoder(jbp, code, 3, fr["sigma2"], fr["perm"], iters=15, early_stop=True)
    try:
        got = dec.decode(fr["y"], form=jbp.FORM_STEP if form == "step" else jbp.FORM_AUTO)
    finally:
        dec.close()
        ctx.close()
    ref = O.decode(code, 3, fr["sigma2"], fr["perm"], fr["y"], 15, early_stop=True, want_margin=True)
    bad, _ = _margin_mismatch(got, ref)
    assert bad == 0
    assert (got["iters"] == ref["iters"]).all()


@pytest.mark.timeout(120)
def test_serving_destroy_with_frames_in_flight(env):
    """jbp_destroy of a decoder whose frames are queued or part-way through
    their iterations returns once its pool has drained; a frame it cancelled
    polls JBP_ECLOSED, one it finished polls its result; another decoder's
    frames are unaffected and the context then closes."""
    jbp, O, torch = env
    ctx = jbp.Context(iters=50, early_stop=False, block_iters=5)
    code_a = I.make_code(512, 16)
    fr_a = I.make_frames(code_a, 6, 10.0, 64, seed=71)
    code_b = I.make_code(64, 4)
    fr_b = I.make_frames(code_b, 2, 12.0, 8, seed=72)
    dec_a = jbp.Decoder(ctx, code_a, 6, fr_a["sigma2"], fr_a["perm"])
    dec_b = jbp.Decoder(ctx, code_b, 2, fr_b["sigma2"], fr_b["perm"])
    try:
        alone_b = [dec_b.decode(fr_b["y"][i:i + 1], form=jbp.FORM_FUSED) for i in range(8)]   # its pool's form
        ta = [dec_a.submit(fr_a["y"][i]) for i in range(64)]
        tb = [dec_b.submit(fr_b["y"][i]) for i in range(8)]
        dec_a.close()
        done = cancelled = 0
        for tk in ta:
            try:
                res = ctx.poll(tk, 512, 6)
            except jbp.JBPError as e:
                assert e.code == jbp.ECLOSED
                cancelled += 1
                continue
            assert res is not None and res["iters"] == 50
            done += 1
        assert done + cancelled == 64
        for i, tk in enumerate(tb):
            while True:
                res = ctx.poll(tk, 64, 2)
                if res is not None:
                    break
            assert np.array_equal(res["hat"], alone_b[i]["hat"][0])
    finally:
        dec_a.close()
        dec_b.close()
        ctx.close()


@pytest.mark.parametrize("T,snr", [(1, 20.0), (2, 20.0), (4, 16.0), (12, 16.0)])
def test_fused_iteration_boundaries_and_early_stop(env, T, snr):
    """The fused form folds each iteration's decisions into the next channel
    phase and its syndromes into the next check phase; at T = 1 and T = 2 and
    with frames stopping at different iterations, iteration counts and syndrome
    flags equal the oracle's (and the step form's) for every frame, and the
    decisions of every frame the oracle decodes to codewords are bit-exact
    where the FP64 margin exceeds 1e-6.  Frames that never converge at this SNR
    are compared on iterations and flags only: their BP trajectory is chaotic,
    and the FP32 transform's rounding grows by a factor of about 2-10 per
    iteration until, after a dozen iterations, a final decision can flip."""
    jbp, O, torch = env
    code = I.make_code(64, 4)
    fr = I.make_frames(code, 2, snr, 200, seed=4252)
    ctx, dec = _decoder(jbp, code, 2, fr["sigma2"], fr["perm"], iters=T, early_stop=True)
    try:
        fused = dec.decode(fr["y"], form=jbp.FORM_FUSED)
        step = dec.decode(fr["y"], form=jbp.FORM_STEP)
    finally:
        dec.close()
        ctx.close()
    ref = O.decode(code, 2, fr["sigma2"], fr["perm"], fr["y"], T, early_stop=True, want_margin=True)
    conv = ref["ok"].all(axis=1)
    for got in (fused, step):
        assert (got["iters"] == ref["iters"]).all()
        assert (got["ok"] == ref["ok"]).all()
        sure = ref["margin"] > 1e-6
        if T > 4:
            sure &= conv[:, None, None]
        assert int(((got["hat"] != ref["hat"]) & sure).sum()) == 0
    print("T=%d: iterations run %s, converged %d" % (T, np.bincount(ref["iters"]).tolist(), int(conv.sum())))
    if T == 12:
        assert conv.sum() > 10 and len(set(ref["iters"].tolist())) > 4   # frames stop at many iterations


def test_step_entry_points_refuse_misaligned_buffers(env):
    """The step kernels move messages with 16-byte loads and bulk copies; a
    misaligned device pointer is refused on the host with JBP_EINVAL."""
    jbp, O, torch = env
    code = I.make_code(64, 16)
    fr = I.make_frames(code, 2, 10.0, 2, seed=3)
    ctx, dec = _decoder(jbp, code, 2, fr["sigma2"], fr["perm"])
    try:
        dev = torch.device("cuda:0")
        E = code["P"] * 4
        big = torch.ones(2 * 2 * E * 16 + 1, dtype=torch.float32, device=dev)
        msg = big[1:].view(2, 2, E, 16)            # 4 bytes off a 16-byte boundary
        ch2v = torch.empty((2, 2, 64, 16), dtype=torch.float32, device=dev)
        y = torch.from_numpy(fr["y"]).to(dev)
        for call in (lambda: dec.step_check(msg), lambda: dec.step_channel(y, msg, ch2v),
                     lambda: dec.step_var(ch2v, msg, None, torch.empty((2, 2, 64), dtype=torch.uint8, device=dev))):
            with pytest.raises(jbp.JBPError) as ei:
                call()
            assert ei.value.code == jbp.EINVAL
        torch.cuda.synchronize()
    finally:
        dec.close()
        ctx.close()


@pytest.mark.parametrize("K,q,n,F", [(4, 16, 256, 200), (4, 64, 128, 60), (3, 32, 64, 150)])
def test_step_kernels_many_tiles_equal_small_batches(env, K, q, n, F):
    """Persistent step kernels over more tiles than CTAs -- the TMA-staged check
    (double-buffered tiles carry over from one tile to the next), the tensor-core
    check variants, the team-shape and thread-shape channel node and the variable
    node -- give, bit for bit, what the same frames give two at a time (one tile
    per CTA, the case the oracle comparisons above cover): no unit reads another
    unit's data."""
    jbp, O, torch = env
    code = I.make_code(n, q)
    fr = I.make_frames(code, K, 12.0, F, seed=600 + K + q)
    rng = np.random.default_rng(601)
    E = code["P"] * code["dc"]
    msg0 = np.exp(I.random_log_messages(rng, (F, K, E), q, spread=3.0)).astype(np.float32)
    precs = [0, 3, 1] if q >= 16 else [0]
    ctx, dec = _decoder(jbp, code, K, fr["sigma2"], fr["perm"])
    try:
        y_d = torch.from_numpy(fr["y"]).cuda()

        def run(frames):
            outs = []
            msg = torch.from_numpy(msg0).cuda()
            ch = torch.zeros((F, K, n, q), dtype=torch.float32, device="cuda")
            hat = torch.zeros((F, K, n), dtype=torch.uint8, device="cuda")
            for f0 in range(0, F, frames):
                sl = slice(f0, min(F, f0 + frames))
                dec.step_channel(y_d[sl], msg[sl], ch[sl])
            outs += [msg.clone(), ch.clone()]
            for prec in precs:
                m = msg.clone()
                for f0 in range(0, F, frames):
                    dec.step_check(m[f0:f0 + frames], precision=prec)
                outs.append(m)
            for f0 in range(0, F, frames):
                sl = slice(f0, min(F, f0 + frames))
                dec.step_var(ch[sl], outs[2][sl], None, hat[sl])
            outs.append(hat)
            torch.cuda.synchronize()
            return outs

        big, small = run(F), run(2)
        assert dec.tc_timeouts() == 0
        for i, (a, b) in enumerate(zip(big, small)):
            assert torch.equal(a, b), i
    finally:
        dec.close()
        ctx.close()


@pytest.mark.parametrize("K,q,n,fpc", [(4, 16, 256, 1), (2, 4, 64, 2), (3, 8, 64, 4)])
def test_fused_many_groups_equal_small_batches(env, K, q, n, fpc):
    """The fused kernel over more frame groups than CTAs (each CTA re-initialises its
    shared-memory state between groups; fpc frames per group, the last group partly
    filled) gives, bit for bit, what the same frames give two at a time: frames
    never share arithmetic, and the oracle comparisons above use one group per CTA."""
    jbp, O, torch = env
    code = I.make_code(n, q)
    F = 152 * fpc * 2 + 6            # every CTA runs at least two groups, the last one partly filled
    fr = I.make_frames(code, K, 12.0, F, seed=700 + K + q)
    ctx, dec = _decoder(jbp, code, K, fr["sigma2"], fr["perm"], iters=12, early_stop=True)
    try:
        dec.set_launch(256, fpc)
        big = dec.decode(fr["y"], form=jbp.FORM_FUSED)
        small = [dec.decode(fr["y"][f0:f0 + 2], form=jbp.FORM_FUSED) for f0 in range(0, F, 2)]
    finally:
        dec.close()
        ctx.close()
    for key in ("hat", "iters", "ok"):
        assert np.array_equal(big[key], np.concatenate([s[key] for s in small])), key


def test_serving_step_form_pools_match_frames_decoded_alone(env):
    """Decoders outside the fused position-major form (variable degree 3 here)
    keep step-form pools: each served frame equals the frame decoded alone in
    the step form, early-stopping frames included."""
    import time
    jbp, O, torch = env
    ctx = jbp.Context(iters=12, early_stop=True, block_iters=3)
    code = I.make_code(64, 16, dv=3, dc=4)
    fr = I.make_frames(code, 2, 14.0, 20, seed=3141)
    dec = jbp.Decoder(ctx, code, 2, fr["sigma2"], fr["perm"])
    try:
        alone = [dec.decode(fr["y"][i:i + 1], form=jbp.FORM_STEP) for i in range(20)]
        tickets = [dec.submit(fr["y"][i]) for i in range(20)]
        for i, tk in enumerate(tickets):
            deadline = time.time() + 60.0
            while (res := ctx.poll(tk, 64, 2)) is None:
                assert time.time() < deadline
                time.sleep(1e-4)
            assert np.array_equal(res["hat"], alone[i]["hat"][0]), i
            assert res["iters"] == int(alone[i]["iters"][0]) and np.array_equal(res["ok"], alone[i]["ok"][0])
    finally:
        dec.close()
        ctx.close()


@pytest.mark.parametrize("form,want_post,per_frame_sigma", [("FORM_FUSED", False, False), ("FORM_STEP", True, True),
                                                            ("FORM_AUTO", False, True)])
def test_host_decode_in_parts_equals_device_decode(env, form, want_post, per_frame_sigma):
    """A host-buffer decode of a large batch runs in parts whose copies overlap the
    other parts' decodes (9,001 frames: eight parts of unequal size).  Every output
    must equal the one-launch decode of the same frames on device buffers, bit for
    bit, and the decisions the oracle's on a sample above the margin."""
    jbp, O, torch = env
    K, q, n, F, T = 2, 4, 64, 9001, 12
    code = I.make_code(n, q)
    fr = I.make_frames(code, K, 10.0, F, seed=88_000 + len(form))
    sig = (fr["sigma2"] * (1.0 + 0.25 * np.random.default_rng(5).random(F))).astype(np.float32) \
        if per_frame_sigma else None
    ctx, dec = _decoder(jbp, code, K, fr["sigma2"], fr["perm"], iters=T, early_stop=True)
    f = getattr(jbp, form)
    try:
        host = dec.decode(fr["y"], form=f, want_post=want_post, sigma2=sig)
        dev = torch.device("cuda", 0)
        y_d = torch.from_numpy(fr["y"]).to(dev)
        hat = torch.full((F, K, n), 255, dtype=torch.uint8, device=dev)
        it = torch.zeros((F,), dtype=torch.int32, device=dev)
        ok = torch.full((F, K), 7, dtype=torch.uint8, device=dev)
        post = torch.empty((F, K, n, q), dtype=torch.float32, device=dev) if want_post else None
        sig_d = torch.from_numpy(sig).to(dev) if sig is not None else None
        torch.cuda.synchronize()
        dec.decode_device(y_d, hat, it, ok, post=post, form=f, sigma2=sig_d)
        torch.cuda.synchronize()
        ref = {"hat": hat.cpu().numpy(), "iters": it.cpu().numpy(), "ok": ok.cpu().numpy()}
        if want_post:
            ref["post"] = post.cpu().numpy()
    finally:
        dec.close()
        ctx.close()
    for key in ref:
        assert np.array_equal(host[key], ref[key]), key
    for f in [0, 1125, 1126, 4500, F - 1]:   # both sides of the first part boundary, the ends
        s2 = fr["sigma2"] if sig is None else float(sig[f])
        o = O.decode(code, K, s2, fr["perm"], fr["y"][f:f + 1], T, early_stop=True, want_margin=True)
        bad, _ = _margin_mismatch({"hat": host["hat"][f:f + 1]}, o)
        assert bad == 0, f
        assert host["iters"][f] == o["iters"][0], f
