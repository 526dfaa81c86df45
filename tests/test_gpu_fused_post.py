"""GPU parity of the fused (shared-memory resident) decode kernel's
log-messages, and of its two code paths.

* The fused kernel's log-posterior after T iterations (eq. app_ldpc_marginal:
  the channel message times the variable's two c2v messages, max-normalised)
  against the FP64 oracle's on the same float32 inputs, element by element:
  |gpu - oracle| <= 1e-4 wherever the oracle entry is >= ln(1e-4), and both
  below ln(1e-4) + 1e-4 elsewhere.  Shapes: the headline shape (K = 4, GF(16),
  n = 256) and two smaller ones, a few iterations (early stop off, so both
  sides run exactly T iterations).
* Without a log-posterior output the kernel folds the decision phase of
  iteration t into the channel phase of iteration t + 1 and the syndrome test
  into the next check phase (the path the benchmark times); with one it keeps
  separate phases.  Both must give bit-identical decisions, iteration counts and
  syndrome flags on the same frames, in each launch shape, and every launch
  shape (one thread per channel use, or a lane pair per use at 512 threads)
  the same outputs as the first.
"""
import math

import numpy as np
import pytest

from paper_2605_26580_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LN_1E4 = math.log(1e-4)


@pytest.fixture(scope="module")
def env(jbp_lib, oracle):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return jbp_lib, oracle, torch


def _fused_device(jbp, torch, dec, y, K, n, q, want_post, launch=None):
    F = y.shape[0]
    dev = torch.device("cuda", 0)
    y_d = torch.from_numpy(y).to(dev)
    hat = torch.full((F, K, n), 255, dtype=torch.uint8, device=dev)
    it = torch.zeros((F,), dtype=torch.int32, device=dev)
    ok = torch.full((F, K), 7, dtype=torch.uint8, device=dev)
    post = torch.empty((F, K, n, q), dtype=torch.float32, device=dev) if want_post else None
    if launch:
        dec.set_launch(*launch)
    torch.cuda.synchronize()
    dec.decode_device(y_d, hat, it, ok, post=post, form=jbp.FORM_FUSED)
    torch.cuda.synchronize()
    out = {"hat": hat.cpu().numpy(), "iters": it.cpu().numpy(), "ok": ok.cpu().numpy()}
    if want_post:
        out["post"] = post.cpu().numpy()
    return out


@pytest.mark.parametrize("K,q,n,T,snr,launch", [(4, 16, 256, 3, 10.0, None), (4, 16, 256, 6, 12.0, None),
                                                (2, 4, 64, 5, 10.0, None), (3, 8, 64, 4, 12.0, None),
                                                (4, 16, 256, 1, 16.0, None), (4, 16, 256, 4, 10.0, (512, 1))])
def test_fused_logpost_matches_oracle(env, K, q, n, T, snr, launch):
    jbp, O, torch = env
    code = I.make_code(n, q)
    F = 6
    fr = I.make_frames(code, K, snr, F, seed=40_000 + 100 * K + q + T)
    ctx = jbp.Context(iters=T, early_stop=False)
    dec = jbp.Decoder(ctx, code, K, fr["sigma2"], fr["perm"])
    try:
        assert dec.fused_ok
        got = _fused_device(jbp, torch, dec, fr["y"], K, n, q, want_post=True, launch=launch)
    finally:
        dec.close()
        ctx.close()
    ref = O.decode(code, K, fr["sigma2"], fr["perm"], fr["y"], T, early_stop=False, want_post=True)
    g = got["post"].astype(np.float64)
    r = ref["post"]
    mask = r >= LN_1E4
    err = np.abs(g - r)
    e_in = float(err[mask].max())
    e_big = float(err[r >= math.log(0.5)].max())
    outside_ok = bool(np.all(g[~mask] < LN_1E4 + 1e-4))
    print("fused logpost K=%d q=%d n=%d T=%d %.0f dB: max err %.2e (oracle >= ln 1e-4, %d entries), "
          "%.2e (>= ln 0.5); %d entries below" % (K, q, n, T, snr, e_in, int(mask.sum()), e_big,
                                                   int((~mask).sum())))
    assert np.allclose(g.max(-1), 0.0, atol=1e-6)
    assert (got["iters"] == T).all()
    assert e_in <= 1e-4
    assert outside_ok


@pytest.mark.parametrize("K,q,n,snr,T,launches", [
    (4, 16, 256, 10.0, 50, [(256, 1), (128, 2), (192, 1), (512, 1), (512, 2)]),
    (2, 4, 64, 12.0, 20, [(256, 1), (128, 4)]),
    (3, 8, 64, 14.0, 15, [(256, 1), (64, 3)]),
])
def test_fused_folded_path_equals_unfolded(env, K, q, n, snr, T, launches):
    jbp, O, torch = env
    code = I.make_code(n, q)
    F = 40
    fr = I.make_frames(code, K, snr, F, seed=50_000 + 100 * K + q)
    ctx = jbp.Context(iters=T, early_stop=True)
    dec = jbp.Decoder(ctx, code, K, fr["sigma2"], fr["perm"])
    first = None
    try:
        for launch in launches:
            folded = _fused_device(jbp, torch, dec, fr["y"], K, n, q, want_post=False, launch=launch)
            if first is None:
                first = folded
            for key in ("hat", "iters", "ok"):   # the launch shape changes no arithmetic
                assert np.array_equal(folded[key], first[key]), (launch, key)
            unfolded = _fused_device(jbp, torch, dec, fr["y"], K, n, q, want_post=True, launch=launch)
            for key in ("hat", "iters", "ok"):
                assert np.array_equal(folded[key], unfolded[key]), (launch, key)
            assert (folded["hat"] < q).all() and ((folded["iters"] >= 1) & (folded["iters"] <= T)).all()
            assert np.array_equal(folded["ok"], O.syndrome_ok(code, K, folded["hat"]))
            print("K=%d q=%d launch %s: folded == unfolded on %d frames; iterations %d..%d"
                  % (K, q, launch, F, int(folded["iters"].min()), int(folded["iters"].max())))
    finally:
        dec.close()
        ctx.close()
