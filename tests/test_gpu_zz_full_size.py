"""Parity at the headline workload's full size, in the launch configuration the
benchmark times: 65,536 frames of K = 4 users, GF(16), n = 256, 50 iterations
with early stop, one fused launch with the autotuned launch shape.

The oracle decodes a sample of frames one by one (the first and last frames,
both sides of the first frame-group boundary, the middle, and random frames):
their decisions must equal the oracle's wherever the FP64 posterior margin
exceeds 1e-6, with equal iteration counts and syndrome flags.  Every frame of
the batch is checked against what holds at any size: `ok` is the oracle's
syndrome test of the returned decisions, iteration counts lie in 1..50, and a
frame that stopped early has every user's syndrome zero.  (Runs last: it is the
slowest GPU test.)"""
import os

import numpy as np
import pytest

from paper_2605_26580_gb300 import inputs as I

pytestmark = pytest.mark.gpu

F, K, Q, N, T = 65536, 4, 16, 256, 50


def test_headline_batch_full_size(jbp_lib, oracle):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    jbp, O = jbp_lib, oracle
    dev = torch.device("cuda", 0)
    code = I.make_code(N, Q)
    fr = I.make_frames(code, K, 10.0, F, seed=9_000_000_001, device=dev)
    ctx = jbp.Context(iters=T, early_stop=True)
    dec = jbp.Decoder(ctx, code, K, fr["sigma2"], fr["perm"])
    try:
        y = torch.from_numpy(fr["y"]).to(dev)
        hat = torch.empty((F, K, N), dtype=torch.uint8, device=dev)
        it = torch.empty((F,), dtype=torch.int32, device=dev)
        ok = torch.empty((F, K), dtype=torch.uint8, device=dev)
        st = torch.cuda.Stream(device=dev)
        torch.cuda.synchronize()                  # inputs on the device before the decoder's stream reads them
        threads, fpc = dec.tune(y, hat, it, ok, stream=st)
        st.synchronize()
        hat.fill_(255)                            # every decision must be written by the decode below
        torch.cuda.synchronize()
        dec.decode_device(y, hat, it, ok, form=jbp.FORM_FUSED, stream=st)
        st.synchronize()
        g = {"hat": hat.cpu().numpy(), "iters": it.cpu().numpy(), "ok": ok.cpu().numpy()}
        assert dec.tc_timeouts() == 0
    finally:
        dec.close()
        ctx.close()
    assert threads > 0 and fpc >= 1
    # every frame: properties that hold at any size
    assert (g["hat"] < Q).all()
    assert ((g["iters"] >= 1) & (g["iters"] <= T)).all()
    assert np.array_equal(g["ok"], O.syndrome_ok(code, K, g["hat"]))
    early = g["iters"] < T
    assert (g["ok"][early] == 1).all()
    # sampled frames against the oracle, decoded one by one
    rng = np.random.default_rng(2)
    idx = sorted({0, fpc - 1, fpc, F // 2, F - fpc - 1, F - 1} | set(int(i) for i in rng.integers(0, F, 4)))
    ref = O.decode(code, K, fr["sigma2"], fr["perm"], fr["y"][idx], T, early_stop=True, want_margin=True,
                   threads=os.cpu_count() or 1)
    sure = ref["margin"] > 1e-6
    bad = int(((g["hat"][idx] != ref["hat"]) & sure).sum())
    print("full size: launch %d threads x %d frames per CTA; %d sampled frames, %d of %d confident decisions differ; "
          "SER %.4f" % (threads, fpc, len(idx), bad, int(sure.sum()), float((g["hat"] != fr["c"]).mean())))
    assert bad == 0
    assert np.array_equal(g["iters"][idx], ref["iters"])
    assert np.array_equal(g["ok"][idx], ref["ok"])
