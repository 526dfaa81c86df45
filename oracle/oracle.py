"""Python access to the FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It compiles ``jbp_oracle.c`` with gcc
(OpenMP over frames) into ``oracle/_build/`` and wraps it with ctypes.  It
shares nothing with the CUDA library: no headers, tables or helpers.

All arrays follow the layouts documented in ``jbp_oracle.h``: frame-major,
check-major edges ``e = j*dc + d``, messages as max-normalised FP64 log vectors.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD, "libjbp_oracle.so")

CHECK_WHT, CHECK_DIRECT, CHECK_LITERAL = 0, 1, 2
REL_FLOOR = 1e-12                 # c2v floor relative to the message max
LOG_FLOOR = math.log(REL_FLOOR)   # clip of every stored log-message

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain C11, -O2, OpenMP)."""
    src = os.path.join(HERE, "jbp_oracle.c")
    hdr = os.path.join(HERE, "jbp_oracle.h")
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return LIB_PATH
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Code(C.Structure):
    _fields_ = [("n", C.c_int), ("P", C.c_int), ("dc", C.c_int), ("m", C.c_int),
                ("chk_var", C.POINTER(C.c_int)), ("chk_coef", C.POINTER(C.c_int))]


class _Chan(C.Structure):
    _fields_ = [("K", C.c_int), ("sigma2", C.c_double), ("perm", C.POINTER(C.c_int))]


class _Opts(C.Structure):
    _fields_ = [("iters", C.c_int), ("early_stop", C.c_int), ("check_method", C.c_int),
                ("rel_floor", C.c_double), ("log_floor", C.c_double), ("threads", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            d, i, u8, i32 = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_uint8), C.POINTER(C.c_int32)
            f32 = C.POINTER(C.c_float)
            _lib.or_gf_mul.argtypes = [C.c_int, C.c_int, C.c_int]
            _lib.or_gf_poly.argtypes = [C.c_int]
            _lib.or_channel_node.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, d, C.c_double, d]
            _lib.or_channel_node_brute.argtypes = _lib.or_channel_node.argtypes
            _lib.or_check_node.argtypes = [C.c_int, C.c_int, i, d, C.c_int, C.c_double, d]
            _lib.or_step_channel.argtypes = [C.POINTER(_Code), C.POINTER(_Chan), C.c_int, f32, d, C.c_double, d]
            _lib.or_step_check.argtypes = [C.POINTER(_Code), C.c_int, C.c_int, d, d, C.c_int, C.c_double, d]
            _lib.or_step_var.argtypes = [C.POINTER(_Code), C.c_int, C.c_int, d, d, d, u8]
            _lib.or_step_v2c.argtypes = [C.POINTER(_Code), C.c_int, C.c_int, d, d, d]
            _lib.or_step_check_v2c.argtypes = [C.POINTER(_Code), C.c_int, C.c_int, d, C.c_int, C.c_double, d]
            _lib.or_syndrome.argtypes = [C.POINTER(_Code), C.c_int, C.c_int, u8, u8]
            _lib.or_decode.argtypes = [C.POINTER(_Code), C.POINTER(_Chan), C.c_int, f32, C.POINTER(_Opts),
                                       u8, i32, u8, d, d, d, d]
            _lib.or_brute_marginals.argtypes = [C.POINTER(_Code), C.POINTER(_Chan), f32, d]
            _lib.or_brute_marginals.restype = C.c_long
            for fn in (_lib.or_bg_log_activity, _lib.or_bg_gain, _lib.or_bg_deriv):
                fn.argtypes = [C.c_double] * 4
                fn.restype = C.c_double
            _lib.or_amp_slot.argtypes = [C.c_int, C.c_int, i, f32, C.c_int, C.c_double, C.c_double, d, d, d]
            _lib.or_amp_dict.argtypes = [C.c_int, C.c_int, d, d, f32, C.c_int, C.c_double, C.c_double, d, d, d]
            _lib.or_amp_evidence.argtypes = [C.c_int, C.c_int, C.c_int, i, C.c_int, f32, C.c_int, C.c_double,
                                             C.c_double, d, C.c_int]
            _lib.or_bp_prior.argtypes = [C.POINTER(_Code), C.c_int, d, C.POINTER(_Opts), u8, i32, u8, d, d]
            _lib.or_sic_decode.argtypes = [C.POINTER(_Code), C.c_int, C.c_double, C.c_int, d, C.POINTER(_Opts),
                                           u8, i32, u8, d]
    return _lib


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


class _Pinned:
    """Keeps the numpy arrays behind a ctypes struct alive."""

    def __init__(self, code, K=None, sigma2=None, perm=None):
        self.chk_var = np.ascontiguousarray(code["chk_var"], dtype=np.int32)
        self.chk_coef = np.ascontiguousarray(code["chk_coef"], dtype=np.int32)
        self.code = _Code(int(code["n"]), int(code["P"]), int(code["dc"]), int(code["m"]),
                          _ptr(self.chk_var, C.c_int), _ptr(self.chk_coef, C.c_int))
        if K is not None:
            self.perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32).reshape(-1)
            self.chan = _Chan(int(K), float(sigma2), _ptr(self.perm, C.c_int))


def gf_mul(m: int, a: int, b: int) -> int:
    return lib().or_gf_mul(m, a, b)


def gf_poly(m: int) -> int:
    return lib().or_gf_poly(m)


def channel_node(K, m, sigma2, y, logmu, log_floor=LOG_FLOOR, brute=False):
    logmu = np.ascontiguousarray(logmu, dtype=np.float64).reshape(K, 1 << m)
    out = np.empty_like(logmu)
    fn = lib().or_channel_node_brute if brute else lib().or_channel_node
    fn(K, m, float(sigma2), float(y), _ptr(logmu, C.c_double), float(log_floor), _ptr(out, C.c_double))
    return out


def check_node(m, coef, logv2c, method=CHECK_WHT, rel_floor=REL_FLOOR):
    coef = np.ascontiguousarray(coef, dtype=np.int32)
    dc = coef.shape[0]
    logv2c = np.ascontiguousarray(logv2c, dtype=np.float64).reshape(dc, 1 << m)
    out = np.empty_like(logv2c)
    lib().or_check_node(m, dc, _ptr(coef, C.c_int), _ptr(logv2c, C.c_double), method,
                        float(rel_floor), _ptr(out, C.c_double))
    return out


def step_channel(code, K, sigma2, perm, y, c2v, log_floor=LOG_FLOOR):
    pin = _Pinned(code, K, sigma2, perm)
    y = np.ascontiguousarray(y, dtype=np.float32)
    F = y.shape[0]
    c2v = np.ascontiguousarray(c2v, dtype=np.float64)
    ch2v = np.empty((F, K, code["n"], 1 << code["m"]), dtype=np.float64)
    lib().or_step_channel(C.byref(pin.code), C.byref(pin.chan), F, _ptr(y, C.c_float),
                          _ptr(c2v, C.c_double), float(log_floor), _ptr(ch2v, C.c_double))
    return ch2v


def step_check(code, K, ch2v, c2v_old, method=CHECK_WHT, rel_floor=REL_FLOOR):
    pin = _Pinned(code)
    ch2v = np.ascontiguousarray(ch2v, dtype=np.float64)
    c2v_old = np.ascontiguousarray(c2v_old, dtype=np.float64)
    out = np.empty_like(c2v_old)
    lib().or_step_check(C.byref(pin.code), K, ch2v.shape[0], _ptr(ch2v, C.c_double),
                        _ptr(c2v_old, C.c_double), method, float(rel_floor), _ptr(out, C.c_double))
    return out


def step_v2c(code, K, ch2v, c2v):
    pin = _Pinned(code)
    ch2v = np.ascontiguousarray(ch2v, dtype=np.float64)
    c2v = np.ascontiguousarray(c2v, dtype=np.float64)
    out = np.empty_like(c2v)
    lib().or_step_v2c(C.byref(pin.code), K, ch2v.shape[0], _ptr(ch2v, C.c_double),
                      _ptr(c2v, C.c_double), _ptr(out, C.c_double))
    return out


def step_check_v2c(code, K, v2c, method=CHECK_WHT, rel_floor=REL_FLOOR):
    pin = _Pinned(code)
    v2c = np.ascontiguousarray(v2c, dtype=np.float64)
    out = np.empty_like(v2c)
    lib().or_step_check_v2c(C.byref(pin.code), K, v2c.shape[0], _ptr(v2c, C.c_double), method,
                            float(rel_floor), _ptr(out, C.c_double))
    return out


def step_var(code, K, ch2v, c2v):
    pin = _Pinned(code)
    ch2v = np.ascontiguousarray(ch2v, dtype=np.float64)
    c2v = np.ascontiguousarray(c2v, dtype=np.float64)
    F = ch2v.shape[0]
    post = np.empty_like(ch2v)
    hat = np.empty((F, K, code["n"]), dtype=np.uint8)
    lib().or_step_var(C.byref(pin.code), K, F, _ptr(ch2v, C.c_double), _ptr(c2v, C.c_double),
                      _ptr(post, C.c_double), _ptr(hat, C.c_uint8))
    return post, hat


def syndrome_ok(code, K, hat):
    pin = _Pinned(code)
    hat = np.ascontiguousarray(hat, dtype=np.uint8)
    F = hat.shape[0]
    ok = np.empty((F, K), dtype=np.uint8)
    lib().or_syndrome(C.byref(pin.code), K, F, _ptr(hat, C.c_uint8), _ptr(ok, C.c_uint8))
    return ok


def decode(code, K, sigma2, perm, y, iters, early_stop=True, check_method=CHECK_WHT,
           rel_floor=REL_FLOOR, log_floor=LOG_FLOOR, threads=0, want_post=False,
           want_margin=False, want_msgs=False):
    """Full joint BP decode of F frames.  Returns a dict of numpy arrays."""
    pin = _Pinned(code, K, sigma2, perm)
    y = np.ascontiguousarray(y, dtype=np.float32)
    F, n, Q = y.shape[0], int(code["n"]), 1 << int(code["m"])
    E = int(code["P"]) * int(code["dc"])
    out = {
        "hat": np.empty((F, K, n), dtype=np.uint8),
        "iters": np.empty((F,), dtype=np.int32),
        "ok": np.empty((F, K), dtype=np.uint8),
    }
    if want_post:
        out["post"] = np.empty((F, K, n, Q), dtype=np.float64)
    if want_margin:
        out["margin"] = np.empty((F, K, n), dtype=np.float64)
    if want_msgs:
        out["ch2v"] = np.empty((F, K, n, Q), dtype=np.float64)
        out["c2v"] = np.empty((F, K, E, Q), dtype=np.float64)
    o = _Opts(int(iters), int(bool(early_stop)), int(check_method), float(rel_floor),
              float(log_floor), int(threads))
    lib().or_decode(C.byref(pin.code), C.byref(pin.chan), F, _ptr(y, C.c_float), C.byref(o),
                    _ptr(out["hat"], C.c_uint8), _ptr(out["iters"], C.c_int32), _ptr(out["ok"], C.c_uint8),
                    _ptr(out.get("post"), C.c_double), _ptr(out.get("margin"), C.c_double),
                    _ptr(out.get("ch2v"), C.c_double), _ptr(out.get("c2v"), C.c_double))
    return out


def brute_marginals(code, K, sigma2, perm, y):
    """Exact max-normalised log marginals [K, n, Q] and the codebook size."""
    pin = _Pinned(code, K, sigma2, perm)
    y = np.ascontiguousarray(y, dtype=np.float32).reshape(-1)
    out = np.empty((K, int(code["n"]), 1 << int(code["m"])), dtype=np.float64)
    size = lib().or_brute_marginals(C.byref(pin.code), C.byref(pin.chan), _ptr(y, C.c_float),
                                    _ptr(out, C.c_double))
    if size < 0:
        raise ValueError("case too large for enumeration")
    return out, int(size)


# ---- evidence interface: AMP detector and SIC FFT-BP ----

def bg_log_activity(s, nu, rho, su2):
    return lib().or_bg_log_activity(float(s), float(nu), float(rho), float(su2))


def bg_gain(s, nu, rho, su2):
    return lib().or_bg_gain(float(s), float(nu), float(rho), float(su2))


def bg_deriv(s, nu, rho, su2):
    return lib().or_bg_deriv(float(s), float(nu), float(rho), float(su2))


def amp_slot(Q, rows, y, iters, rho, su2):
    """One slot: returns (S [Q], R [Q] complex, nu)."""
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.float32).reshape(-1)
    S = np.empty(Q, dtype=np.float64)
    R = np.empty(2 * Q, dtype=np.float64)
    nu = C.c_double()
    lib().or_amp_slot(int(Q), rows.size, _ptr(rows, C.c_int), _ptr(y, C.c_float), int(iters), float(rho),
                      float(su2), _ptr(S, C.c_double), _ptr(R, C.c_double), C.byref(nu))
    return S, R[0::2] + 1j * R[1::2], nu.value


def amp_dict(A, y, iters, rho, su2):
    """AMP with a given complex dictionary A [ns, Q]: returns (S [Q], R [Q], nu)."""
    ns, Q = A.shape
    Ar = np.ascontiguousarray(A.real, dtype=np.float64)
    Ai = np.ascontiguousarray(A.imag, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float32).reshape(-1)
    S = np.empty(Q, dtype=np.float64)
    R = np.empty(2 * Q, dtype=np.float64)
    nu = C.c_double()
    lib().or_amp_dict(int(Q), int(ns), _ptr(Ar, C.c_double), _ptr(Ai, C.c_double), _ptr(y, C.c_float), int(iters),
                      float(rho), float(su2), _ptr(S, C.c_double), _ptr(R, C.c_double), C.byref(nu))
    return S, R[0::2] + 1j * R[1::2], nu.value


def amp_evidence(Q, rows, y, iters, rho, su2, threads=0):
    """y [F, L, ns, 2] float32, rows [L, ns] -> S [F, L, Q] float64."""
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    L, ns = rows.shape
    y = np.ascontiguousarray(y, dtype=np.float32)
    F = y.shape[0]
    S = np.empty((F, L, Q), dtype=np.float64)
    lib().or_amp_evidence(int(Q), ns, L, _ptr(rows, C.c_int), F, _ptr(y, C.c_float), int(iters), float(rho),
                          float(su2), _ptr(S, C.c_double), int(threads))
    return S


def _opts(iters, early_stop, check_method, rel_floor, log_floor, threads):
    return _Opts(int(iters), int(bool(early_stop)), int(check_method), float(rel_floor), float(log_floor),
                 int(threads))


def bp_prior(code, S, iters, early_stop=True, check_method=CHECK_WHT, rel_floor=REL_FLOOR,
             log_floor=LOG_FLOOR, threads=0, want_post=False):
    """Single-row FFT-BP from evidence S [F, n, Q]."""
    pin = _Pinned(code)
    S = np.ascontiguousarray(S, dtype=np.float64)
    F, n, Q = S.shape
    out = {"hat": np.empty((F, n), dtype=np.uint8), "iters": np.empty((F,), dtype=np.int32),
           "ok": np.empty((F,), dtype=np.uint8), "margin": np.empty((F, n), dtype=np.float64)}
    if want_post:
        out["post"] = np.empty((F, n, Q), dtype=np.float64)
    o = _opts(iters, early_stop, check_method, rel_floor, log_floor, threads)
    lib().or_bp_prior(C.byref(pin.code), F, _ptr(S, C.c_double), C.byref(o), _ptr(out["hat"], C.c_uint8),
                      _ptr(out["iters"], C.c_int32), _ptr(out["ok"], C.c_uint8), _ptr(out.get("post"), C.c_double),
                      _ptr(out["margin"], C.c_double))
    return out


def sic_decode(code, K, S, iters, cancel_log, early_stop=True, check_method=CHECK_WHT,
               rel_floor=REL_FLOOR, log_floor=LOG_FLOOR, threads=0):
    """SIC over K rows from evidence S [F, n, Q]: hat [F, K, n], iters/ok [F, K], margin."""
    pin = _Pinned(code)
    S = np.ascontiguousarray(S, dtype=np.float64)
    F, n, Q = S.shape
    out = {"hat": np.empty((F, K, n), dtype=np.uint8), "iters": np.empty((F, K), dtype=np.int32),
           "ok": np.empty((F, K), dtype=np.uint8), "margin": np.empty((F, K, n), dtype=np.float64)}
    o = _opts(iters, early_stop, check_method, rel_floor, log_floor, threads)
    lib().or_sic_decode(C.byref(pin.code), int(K), float(cancel_log), F, _ptr(S, C.c_double), C.byref(o),
                        _ptr(out["hat"], C.c_uint8), _ptr(out["iters"], C.c_int32), _ptr(out["ok"], C.c_uint8),
                        _ptr(out["margin"], C.c_double))
    return out


def host_threads() -> int:
    return os.cpu_count() or 1
