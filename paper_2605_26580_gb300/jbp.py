"""Thin ctypes binding of the C ABI in ``include/jbp.h`` (argument marshalling only).

Every step of the decoder runs inside ``libjbp.so``; this module only converts
numpy arrays / torch CUDA tensors to pointers and status codes to exceptions.
If the library is missing or cannot load, every call raises: there is no
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjbp.so")

OK, EINVAL, ENOMEM, ECUDA, EAGAIN, ETIMEOUT, ECLOSED = range(7)
PREC_FP32, PREC_BF16X2, PREC_BF16, PREC_BF16X3 = 0, 1, 2, 3
FORM_AUTO, FORM_FUSED, FORM_STEP, FORM_PLAIN = 0, 1, 2, 3
CHAN_TRELLIS, CHAN_DFT, CHAN_AUTO = 0, 1, 2
CUDA_STREAM_LEGACY = 0x1   # the CUDA runtime's explicit handle of the legacy default stream

EXPORTS = [
    "jbp_context_create", "jbp_context_destroy", "jbp_create", "jbp_destroy", "jbp_decode",
    "jbp_submit", "jbp_poll", "jbp_serving_stats", "jbp_last_error", "jbp_step_channel",
    "jbp_step_check", "jbp_step_var", "jbp_step_syndrome", "jbp_query", "jbp_query_channel", "jbp_dft_tables", "jbp_gf_tables", "jbp_decode_noalloc", "jbp_stats", "jbp_decode_many", "jbp_tune",
    "jbp_ura_create", "jbp_ura_destroy", "jbp_amp_evidence", "jbp_sic_decode", "jbp_ura_decode", "jbp_match_rows",
    "jbp_fp32_peak",
]


class JBPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("jbp error %d: %s" % (code, msg))
        self.code = code


class Code(C.Structure):
    _fields_ = [("n", C.c_int32), ("P", C.c_int32), ("q", C.c_int32), ("dv", C.c_int32), ("dc", C.c_int32),
                ("chk_var", C.POINTER(C.c_int32)), ("chk_coef", C.POINTER(C.c_uint8))]


class Channel(C.Structure):
    _fields_ = [("sigma2", C.c_double), ("interleave", C.c_int32), ("perm", C.POINTER(C.c_int32))]


class Options(C.Structure):
    _fields_ = [("iters", C.c_int32), ("early_stop", C.c_int32), ("precision", C.c_int32), ("device", C.c_int32),
                ("mem_budget_bytes", C.c_int64), ("block_iters", C.c_int32), ("channel_node", C.c_int32),
                ("reserved", C.c_int32 * 6)]


class UraParams(C.Structure):
    _fields_ = [("ns", C.c_int32), ("K", C.c_int32), ("amp_iters", C.c_int32), ("bp_iters", C.c_int32),
                ("early_stop", C.c_int32), ("reserved", C.c_int32), ("rho_bg", C.c_double),
                ("sigma_u2", C.c_double), ("cancel_log", C.c_double), ("rows", C.POINTER(C.c_int32))]


class Batch(C.Structure):
    _fields_ = [("F", C.c_int32), ("y", C.c_void_p), ("hat", C.c_void_p), ("iters", C.c_void_p),
                ("ok", C.c_void_p), ("logpost", C.c_void_p), ("on_device", C.c_int32), ("form", C.c_int32),
                ("stream", C.c_void_p), ("sigma2", C.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libjbp.so (raises if it is missing: there is no CPU path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libjbp.so is not built; run __graft_entry__.build() "
                                   "(paper_2605_26580_gb300.build.build())")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
            L.jbp_context_create.argtypes = [C.POINTER(Options), C.POINTER(vp)]
            L.jbp_context_destroy.argtypes = [vp]
            L.jbp_create.argtypes = [vp, C.POINTER(Code), i32, i32, C.POINTER(Channel), C.POINTER(vp)]
            L.jbp_destroy.argtypes = [vp]
            L.jbp_decode.argtypes = [vp, C.POINTER(Batch)]
            L.jbp_submit.argtypes = [vp, vp, C.c_double, C.POINTER(u64)]
            L.jbp_poll.argtypes = [vp, u64, vp, vp, vp]
            L.jbp_serving_stats.argtypes = [vp, C.POINTER(u64), C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.jbp_last_error.restype = C.c_char_p
            L.jbp_step_channel.argtypes = [vp, i32, vp, vp, vp, vp]
            L.jbp_step_check.argtypes = [vp, i32, vp, i32, vp]
            L.jbp_step_var.argtypes = [vp, i32, vp, vp, vp, vp, vp]
            L.jbp_step_syndrome.argtypes = [vp, i32, vp, vp, vp]
            L.jbp_query.argtypes = [vp, C.POINTER(i32), C.POINTER(i64), C.POINTER(i32)]
            L.jbp_query_channel.argtypes = [vp, C.POINTER(i32)]
            L.jbp_dft_tables.argtypes = [i32, i32, C.POINTER(i32), vp, C.POINTER(i64)]
            L.jbp_gf_tables.argtypes = [i32, vp, vp]
            L.jbp_fp32_peak.argtypes = [i32, C.c_double, i32, C.POINTER(C.c_double)]
            L.jbp_decode_many.argtypes = [vp, i32, C.POINTER(vp), C.POINTER(Batch), vp]
            L.jbp_tune.argtypes = [vp, C.POINTER(Batch), C.POINTER(i32), C.POINTER(i32)]
            L.jbp_stats.argtypes = [vp, C.POINTER(u64), C.POINTER(i32)]
            L.jbp_decode_noalloc.argtypes = [C.POINTER(Code), i32, C.POINTER(Channel), i32, i32, i32, vp, vp, vp,
                                             vp, vp]
            L.jbp_match_rows.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp, i32, vp]
            L.jbp_ura_create.argtypes = [vp, C.POINTER(Code), C.POINTER(UraParams), C.POINTER(vp)]
            L.jbp_ura_destroy.argtypes = [vp]
            L.jbp_amp_evidence.argtypes = [vp, i32, vp, vp, i32, vp]
            L.jbp_sic_decode.argtypes = [vp, i32, vp, vp, vp, vp, i32, vp]
            L.jbp_ura_decode.argtypes = [vp, i32, vp, vp, vp, vp, i32, vp]
            for name in EXPORTS:
                if name != "jbp_last_error":
                    getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def check(rc: int) -> int:
    if rc not in (OK,):
        raise JBPError(rc, lib().jbp_last_error().decode())
    return rc


def _addr(x):
    """Pointer of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def _stream_ptr(stream, t=None):
    """The stream of a call on device buffers: the given one; else, for torch CUDA
    tensors, torch's current stream on their device, so that the call is ordered
    after the work that produced them (the handle's own stream does not wait for
    torch's); else NULL (the handle's stream)."""
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    if t is not None and getattr(t, "is_cuda", False):
        import torch
        h = torch.cuda.current_stream(t.device).cuda_stream
        # torch's default stream is the legacy default stream, whose handle 0 the C
        # ABI reads as "the handle's own stream": pass its explicit handle instead
        return h if h else CUDA_STREAM_LEGACY
    return None


def gf_tables(q: int):
    """Host-only: the GF(q) multiply and divide tables jbp_create uploads, as
    (mul, div) uint8 arrays [q, q] with mul[h, x] = h x and div[h, x] = x / h."""
    mul = np.zeros((q, q), dtype=np.uint8)
    div = np.zeros((q, q), dtype=np.uint8)
    check(lib().jbp_gf_tables(q, mul.ctypes.data, div.ctypes.data))
    return mul, div


def fp32_peak(device: int = 0, seconds: float = 1.5, packed: bool = False) -> float:
    """Measured FP32 multiply-add rate of the device in TFLOP/s (jbp_fp32_peak)."""
    out = C.c_double()
    check(lib().jbp_fp32_peak(int(device), float(seconds), 1 if packed else 0, C.byref(out)))
    return out.value


def dft_tables(K: int, q: int):
    """Host-only: the DFT channel node's constant tables for (K, q) as jbp_create
    builds them.  Returns (shape dict with L, W, KB, Nc, chunks; uint8 array)."""
    shape = (C.c_int32 * 5)()
    nbytes = C.c_int64()
    check(lib().jbp_dft_tables(K, q, shape, None, C.byref(nbytes)))
    out = np.zeros(nbytes.value, dtype=np.uint8)
    check(lib().jbp_dft_tables(K, q, None, out.ctypes.data, C.byref(nbytes)))
    return dict(zip(("L", "W", "KB", "Nc", "chunks"), list(shape))), out


class Context:
    def __init__(self, iters: int = 50, early_stop: bool = True, precision: int = PREC_FP32, device: int = 0,
                 mem_budget_bytes: int = 0, block_iters: int = 0, channel_node: int = CHAN_TRELLIS):
        self.opt = Options(int(iters), int(bool(early_stop)), int(precision), int(device), int(mem_budget_bytes),
                           int(block_iters), int(channel_node))
        h = C.c_void_p()
        check(lib().jbp_context_create(C.byref(self.opt), C.byref(h)))
        self.ptr = h

    def close(self):
        if self.ptr:
            check(lib().jbp_context_destroy(self.ptr))
            self.ptr = None

    def poll(self, ticket: int, n: int, K: int):
        hat = np.empty((K, n), dtype=np.uint8)
        ok = np.empty((K,), dtype=np.uint8)
        it = np.empty((1,), dtype=np.int32)
        rc = lib().jbp_poll(self.ptr, ticket, _addr(hat), _addr(it), _addr(ok))
        if rc == EAGAIN:
            return None
        check(rc)
        return {"hat": hat, "iters": int(it[0]), "ok": ok}

    def decode_many(self, parts, stream=None):
        """parts: list of (Decoder, y, hat, iters, ok[, sigma2]) device tensors; one call."""
        n = len(parts)
        hs = (C.c_void_p * n)(*[p[0].ptr for p in parts])
        bs = (Batch * n)()
        for i, p in enumerate(parts):
            dec, y, hat, it, ok = p[:5]
            sig = p[5] if len(p) > 5 else None
            bs[i] = Batch(int(y.shape[0]), _addr(y), _addr(hat), _addr(it), _addr(ok), None, 1, FORM_AUTO, None,
                          _addr(sig))
        check(lib().jbp_decode_many(self.ptr, n, hs, bs, _stream_ptr(stream, parts[0][1] if parts else None)))

    def match_rows(self, hat, truth):
        """Row-aligned errors (host arrays [F, K, n]): (symbol errors [F], row errors [F])."""
        hat = np.ascontiguousarray(hat, dtype=np.uint8)
        truth = np.ascontiguousarray(truth, dtype=np.uint8)
        F, K, n = truth.shape
        sym = np.empty(F, dtype=np.int32)
        cw = np.empty(F, dtype=np.int32)
        check(lib().jbp_match_rows(self.ptr, F, K, n, _addr(hat), _addr(truth), _addr(sym), _addr(cw), 0, None))
        return sym, cw

    def match_rows_device(self, hat, truth, sym, cw, stream=None):
        F, K, n = truth.shape
        check(lib().jbp_match_rows(self.ptr, int(F), int(K), int(n), _addr(hat), _addr(truth), _addr(sym), _addr(cw),
                                   1, _stream_ptr(stream, hat)))

    def serving_stats(self):
        c = C.c_uint64()
        a, b = C.c_double(), C.c_double()
        check(lib().jbp_serving_stats(self.ptr, C.byref(c), C.byref(a), C.byref(b)))
        return {"completed": c.value, "p50_us": a.value, "p99_us": b.value}


class Decoder:
    """One (code, K, q, channel) decoder bound to a Context."""

    def __init__(self, ctx: Context, code: dict, K: int, sigma2: float, perm=None, interleave: bool = True):
        self.ctx = ctx
        self.K, self.n, self.q = int(K), int(code["n"]), int(code["q"])
        self._chk_var = np.ascontiguousarray(code["chk_var"], dtype=np.int32)
        self._chk_coef = np.ascontiguousarray(code["chk_coef"], dtype=np.uint8)
        dv = code.get("dv") or int(np.bincount(self._chk_var, minlength=self.n).max())   # largest degree
        c = Code(self.n, int(code["P"]), self.q, int(dv), int(code["dc"]),
                 self._chk_var.ctypes.data_as(C.POINTER(C.c_int32)),
                 self._chk_coef.ctypes.data_as(C.POINTER(C.c_uint8)))
        self._perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32).reshape(-1)
        ch = Channel(float(sigma2), int(bool(interleave and self._perm is not None)),
                     None if self._perm is None else self._perm.ctypes.data_as(C.POINTER(C.c_int32)))
        h = C.c_void_p()
        check(lib().jbp_create(ctx.ptr, C.byref(c), self.K, self.q, C.byref(ch), C.byref(h)))
        self.ptr = h
        E = C.c_int32()
        sb = C.c_int64()
        fz = C.c_int32()
        check(lib().jbp_query(h, C.byref(E), C.byref(sb), C.byref(fz)))
        self.E, self.state_bytes, self.fused_ok = E.value, sb.value, bool(fz.value)
        cn = C.c_int32()
        check(lib().jbp_query_channel(h, C.byref(cn)))
        self.channel_node = cn.value

    def close(self):
        if self.ptr:
            check(lib().jbp_destroy(self.ptr))
            self.ptr = None

    def log_fallbacks(self) -> int:
        v = C.c_uint64()
        check(lib().jbp_stats(self.ptr, C.byref(v), None))
        return v.value

    def tc_timeouts(self) -> int:
        v = C.c_int32()
        check(lib().jbp_stats(self.ptr, None, C.byref(v)))
        return v.value

    # -- whole decodes --------------------------------------------------------
    def decode(self, y, form: int = FORM_AUTO, want_post: bool = False, sigma2=None):
        """Host decode: y numpy [F, n] float32 -> dict of numpy outputs.  sigma2:
        optional per-frame noise variance [F]."""
        y = np.ascontiguousarray(y, dtype=np.float32)
        sig = None if sigma2 is None else np.ascontiguousarray(sigma2, dtype=np.float32)
        F = y.shape[0]
        out = {"hat": np.empty((F, self.K, self.n), dtype=np.uint8), "iters": np.empty((F,), dtype=np.int32),
               "ok": np.empty((F, self.K), dtype=np.uint8)}
        if want_post:
            out["post"] = np.empty((F, self.K, self.n, self.q), dtype=np.float32)
        b = Batch(F, _addr(y), _addr(out["hat"]), _addr(out["iters"]), _addr(out["ok"]), _addr(out.get("post")),
                  0, int(form), None, _addr(sig))
        check(lib().jbp_decode(self.ptr, C.byref(b)))
        return out

    def decode_device(self, y, hat, iters, ok, post=None, form: int = FORM_AUTO, stream=None, sigma2=None):
        """Enqueue a decode on device tensors (returns without waiting)."""
        b = Batch(int(y.shape[0]), _addr(y), _addr(hat), _addr(iters), _addr(ok), _addr(post), 1, int(form),
                  _stream_ptr(stream, y), _addr(sigma2))
        check(lib().jbp_decode(self.ptr, C.byref(b)))

    def set_launch(self, threads: int, frames_per_cta: int = 0):
        th, fc = C.c_int32(threads), C.c_int32(frames_per_cta)
        check(lib().jbp_tune(self.ptr, None, C.byref(th), C.byref(fc)))

    def tune(self, y, hat, iters, ok, sigma2=None, stream=None):
        b = Batch(int(y.shape[0]), _addr(y), _addr(hat), _addr(iters), _addr(ok), None, 1, FORM_AUTO,
                  _stream_ptr(stream, y), _addr(sigma2))
        th, fc = C.c_int32(), C.c_int32()
        check(lib().jbp_tune(self.ptr, C.byref(b), C.byref(th), C.byref(fc)))
        return th.value, fc.value

    # -- serving --------------------------------------------------------------
    def submit(self, y_frame, sigma2: float = 0.0) -> int:
        y = np.ascontiguousarray(y_frame, dtype=np.float32).reshape(-1)
        t = C.c_uint64()
        check(lib().jbp_submit(self.ptr, _addr(y), float(sigma2), C.byref(t)))
        return t.value

    # -- single steps on device tensors ---------------------------------------
    def step_channel(self, y, msg, ch2v, stream=None):
        check(lib().jbp_step_channel(self.ptr, int(y.shape[0]), _addr(y), _addr(msg), _addr(ch2v),
                                     _stream_ptr(stream, msg)))

    def step_check(self, msg, precision: int = PREC_FP32, stream=None):
        check(lib().jbp_step_check(self.ptr, int(msg.shape[0]), _addr(msg), int(precision), _stream_ptr(stream, msg)))

    def step_var(self, ch2v, msg, post, hat, stream=None):
        check(lib().jbp_step_var(self.ptr, int(ch2v.shape[0]), _addr(ch2v), _addr(msg), _addr(post), _addr(hat),
                                 _stream_ptr(stream, msg)))

    def step_syndrome(self, hat, ok, stream=None):
        check(lib().jbp_step_syndrome(self.ptr, int(hat.shape[0]), _addr(hat), _addr(ok), _stream_ptr(stream, hat)))


class EvidenceDecoder:
    """The paper's classical path on the evidence interface: slot-wise AMP
    detector (y -> S) and SIC over K rows of single-row FFT-BP (S -> rows)."""

    def __init__(self, ctx: Context, code: dict, K: int, rows, rho: float, su2: float, cancel_log: float,
                 amp_iters: int = 20, bp_iters: int = 50, early_stop: bool = True):
        self.ctx = ctx
        self.K, self.n, self.q = int(K), int(code["n"]), int(code["q"])
        self._chk_var = np.ascontiguousarray(code["chk_var"], dtype=np.int32)
        self._chk_coef = np.ascontiguousarray(code["chk_coef"], dtype=np.uint8)
        self._rows = np.ascontiguousarray(rows, dtype=np.int32)
        self.ns = int(self._rows.shape[1])
        dv = code.get("dv") or int(np.bincount(self._chk_var, minlength=self.n).max())   # largest degree
        c = Code(self.n, int(code["P"]), self.q, int(dv), int(code["dc"]),
                 self._chk_var.ctypes.data_as(C.POINTER(C.c_int32)),
                 self._chk_coef.ctypes.data_as(C.POINTER(C.c_uint8)))
        p = UraParams(self.ns, self.K, int(amp_iters), int(bp_iters), int(bool(early_stop)), 0, float(rho),
                      float(su2), float(cancel_log), self._rows.ctypes.data_as(C.POINTER(C.c_int32)))
        h = C.c_void_p()
        check(lib().jbp_ura_create(ctx.ptr, C.byref(c), C.byref(p), C.byref(h)))
        self.ptr = h

    def close(self):
        if self.ptr:
            check(lib().jbp_ura_destroy(self.ptr))
            self.ptr = None

    # host arrays: the call copies, runs and waits
    def evidence(self, y):
        y = np.ascontiguousarray(y, dtype=np.float32)
        F = int(y.shape[0])
        S = np.empty((F, self.n, self.q), dtype=np.float32)
        check(lib().jbp_amp_evidence(self.ptr, F, _addr(y), _addr(S), 0, None))
        return S

    def sic(self, S):
        S = np.ascontiguousarray(S, dtype=np.float32)
        F = int(S.shape[0])
        out = {"hat": np.empty((F, self.K, self.n), dtype=np.uint8), "iters": np.empty((F, self.K), dtype=np.int32),
               "ok": np.empty((F, self.K), dtype=np.uint8)}
        check(lib().jbp_sic_decode(self.ptr, F, _addr(S), _addr(out["hat"]), _addr(out["iters"]), _addr(out["ok"]),
                                   0, None))
        return out

    def decode(self, y):
        y = np.ascontiguousarray(y, dtype=np.float32)
        F = int(y.shape[0])
        out = {"hat": np.empty((F, self.K, self.n), dtype=np.uint8), "iters": np.empty((F, self.K), dtype=np.int32),
               "ok": np.empty((F, self.K), dtype=np.uint8)}
        check(lib().jbp_ura_decode(self.ptr, F, _addr(y), _addr(out["hat"]), _addr(out["iters"]), _addr(out["ok"]),
                                   0, None))
        return out

    # device tensors: enqueued on `stream`, no wait
    def evidence_device(self, y, S, stream=None):
        check(lib().jbp_amp_evidence(self.ptr, int(y.shape[0]), _addr(y), _addr(S), 1, _stream_ptr(stream, y)))

    def sic_device(self, S, hat, iters, ok, stream=None):
        check(lib().jbp_sic_decode(self.ptr, int(S.shape[0]), _addr(S), _addr(hat), _addr(iters), _addr(ok), 1,
                                   _stream_ptr(stream, S)))

    def decode_device(self, y, hat, iters, ok, stream=None):
        check(lib().jbp_ura_decode(self.ptr, int(y.shape[0]), _addr(y), _addr(hat), _addr(iters), _addr(ok), 1,
                                   _stream_ptr(stream, y)))
