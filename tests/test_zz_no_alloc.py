"""jbp_decode_noalloc: the decode for callers that may not allocate device memory.

Such callers include code that runs inside another framework's memory pool or
under a hard device-memory cap, and processes that may not call cudaMalloc at
all.  The entry point keeps every working buffer in a fixed array inside the
library, so these tests check (through the C ABI) that it decodes exactly like
the ordinary allocating entry point, jbp_decode in the step form, on two calls in
a row with different batches (the array keeps the previous call's contents and
must not leak them into the next result), and that a batch too large for the
fixed array is refused with a clear error.  This file sorts last so that a run
stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2605_26580_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _code_struct(jbp, code):
    var = np.ascontiguousarray(code["chk_var"], dtype=np.int32)
    coef = np.ascontiguousarray(code["chk_coef"], dtype=np.uint8)
    st = jbp.Code(code["n"], code["P"], code["q"], 2, code["dc"], var.ctypes.data_as(C.POINTER(C.c_int32)),
                  coef.ctypes.data_as(C.POINTER(C.c_uint8)))
    return st, (var, coef)


def _chan_struct(jbp, sigma2, perm):
    p = np.ascontiguousarray(perm, dtype=np.int32).reshape(-1)
    return jbp.Channel(float(sigma2), 1, p.ctypes.data_as(C.POINTER(C.c_int32))), p


def test_noalloc_matches_allocating_decode_twice(jbp_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    jbp = jbp_lib
    torch.cuda.init()
    K, T = 2, 12
    code = I.make_code(64, 4)
    batches = [I.make_frames(code, K, 11.0, 150, seed=501), I.make_frames(code, K, 13.0, 90, seed=502)]
    # the interleavers depend on the seed: use the first batch's for both decoders
    perm = batches[0]["perm"]
    batches[1] = dict(batches[1])
    batches[1]["y"], _ = I.channel_output(4, batches[1]["c"], perm, 13.0, 503)
    lib = jbp.lib()
    cst, keep_code = _code_struct(jbp, code)
    for fr in batches:
        F = fr["y"].shape[0]
        sigma2 = fr["sigma2"]
        # reference: the allocating entry point (step form, device buffers)
        ctx = jbp.Context(iters=T, early_stop=True)
        dec = jbp.Decoder(ctx, code, K, sigma2, perm)
        y = torch.from_numpy(fr["y"]).cuda()
        ref = {"hat": torch.empty((F, K, 64), dtype=torch.uint8, device="cuda"),
               "iters": torch.empty((F,), dtype=torch.int32, device="cuda"),
               "ok": torch.empty((F, K), dtype=torch.uint8, device="cuda")}
        dec.decode_device(y, ref["hat"], ref["iters"], ref["ok"], form=jbp.FORM_STEP)
        torch.cuda.synchronize()
        dec.close()
        ctx.close()
        # the no-allocation entry point, same inputs, outputs pre-filled with garbage
        out = {k: torch.full_like(v, 0x5A) for k, v in ref.items()}
        chs, keep_perm = _chan_struct(jbp, sigma2, perm)
        rc = lib.jbp_decode_noalloc(C.byref(cst), K, C.byref(chs), T, 1, F, y.data_ptr(), out["hat"].data_ptr(),
                                    out["iters"].data_ptr(), out["ok"].data_ptr(), None)
        assert rc == jbp.OK, lib.jbp_last_error()
        torch.cuda.synchronize()
        for key in ("hat", "iters", "ok"):
            assert torch.equal(out[key], ref[key]), key
        # the decisions are the joint BP decisions (sanity: most frames far from random)
        assert (out["hat"].cpu().numpy() == fr["c"]).mean() > 0.3


def test_noalloc_refuses_batches_larger_than_its_fixed_array(jbp_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    jbp = jbp_lib
    code = I.make_code(256, 16)
    cst, keep_code = _code_struct(jbp, code)
    perm = I.make_interleavers(256, 4, seed=1)
    chs, keep_perm = _chan_struct(jbp, 1.0, perm)
    F = 1000   # 1000 frames x 192 KiB of message state > 16 MiB
    y = torch.zeros((F, 256), device="cuda")
    hat = torch.empty((F, 4, 256), dtype=torch.uint8, device="cuda")
    it = torch.empty((F,), dtype=torch.int32, device="cuda")
    ok = torch.empty((F, 4), dtype=torch.uint8, device="cuda")
    rc = jbp.lib().jbp_decode_noalloc(C.byref(cst), 4, C.byref(chs), 5, 1, F, y.data_ptr(), hat.data_ptr(),
                                      it.data_ptr(), ok.data_ptr(), None)
    assert rc == jbp.EINVAL
    msg = jbp.lib().jbp_last_error().decode()
    assert "more than the fixed" in msg and "at most" in msg
