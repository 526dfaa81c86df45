"""The C-ABI library loads and exports every entry point declared in include/jbp.h;
host-side argument checks work without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    with open(os.path.join(ROOT, "include", "jbp.h")) as f:
        for m in re.finditer(r"^\s*(?:int|const char \*)\s*(jbp_\w+)\s*\(", f.read(), re.M):
            names.append(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = set(_declared())
    for required in ["jbp_context_create", "jbp_create", "jbp_decode", "jbp_submit", "jbp_poll",
                     "jbp_destroy", "jbp_context_destroy", "jbp_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(jbp_lib):
    lib = C.CDLL(jbp_lib.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared()) <= set(jbp_lib.EXPORTS) | {"jbp_last_error"}


def test_null_arguments_are_rejected(jbp_lib):
    lib = jbp_lib.lib()
    assert lib.jbp_context_create(None, None) == jbp_lib.EINVAL
    assert b"NULL" in lib.jbp_last_error()
    assert lib.jbp_decode(None, None) == jbp_lib.EINVAL
    assert lib.jbp_destroy(None) == jbp_lib.EINVAL
    assert lib.jbp_poll(None, 1, None, None, None) == jbp_lib.EINVAL
    assert lib.jbp_step_check(None, 1, None, 0, None) == jbp_lib.EINVAL
    assert lib.jbp_ura_create(None, None, None, None) == jbp_lib.EINVAL
    assert lib.jbp_ura_destroy(None) == jbp_lib.EINVAL
    assert lib.jbp_amp_evidence(None, 1, None, None, 0, None) == jbp_lib.EINVAL
    assert lib.jbp_sic_decode(None, 1, None, None, None, None, 0, None) == jbp_lib.EINVAL
    assert lib.jbp_ura_decode(None, 1, None, None, None, None, 0, None) == jbp_lib.EINVAL
    assert lib.jbp_match_rows(None, 1, 2, 3, None, None, None, None, 0, None) == jbp_lib.EINVAL


def test_bad_options_are_rejected_before_touching_the_gpu(jbp_lib):
    opt = jbp_lib.Options(0, 1, 0, 0, 0, 0)          # iters = 0
    h = C.c_void_p()
    assert jbp_lib.lib().jbp_context_create(C.byref(opt), C.byref(h)) == jbp_lib.EINVAL
    opt = jbp_lib.Options(10, 1, 9, 0, 0, 0)         # precision 9
    assert jbp_lib.lib().jbp_context_create(C.byref(opt), C.byref(h)) == jbp_lib.EINVAL


def test_no_gpu_fails_loudly(jbp_lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(jbp_lib.JBPError) as ei:
        jbp_lib.Context(iters=5)
    assert ei.value.code in (jbp_lib.ECUDA, jbp_lib.EINVAL)


def _prototypes():
    """name -> parameter type strings, parsed from the header's declarations."""
    src = open(os.path.join(ROOT, "include", "jbp.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    out = {}
    for m in re.finditer(r"^\s*int\s+(jbp_\w+)\s*\(([^)]*)\)\s*;", src, re.M):
        params = [" ".join(p.split()) for p in m.group(2).split(",") if p.strip() and p.strip() != "void"]
        out[m.group(1)] = params
    return out


def _null_args(params):
    """Every pointer NULL, every integer 1, every double 1.0 (typed for the C ABI)."""
    args = []
    for p in params:
        if "*" in p:
            args.append(None)
        elif p.startswith("double"):
            args.append(C.c_double(1.0))
        elif "int64_t" in p:
            args.append(C.c_uint64(1) if p.startswith("uint") else C.c_int64(1))
        else:
            args.append(C.c_int32(1))
    return args


def test_every_entry_point_refuses_null_pointers(jbp_lib):
    """Each entry point called with all pointers NULL returns EINVAL and sets a
    message, before any device work (this host has no GPU)."""
    lib = C.CDLL(jbp_lib.LIB_PATH)
    lib.jbp_last_error.restype = C.c_char_p
    protos = _prototypes()
    assert set(protos) | {"jbp_last_error"} == set(_declared())
    for name, params in protos.items():
        fn = getattr(lib, name)
        fn.restype = C.c_int
        rc = fn(*_null_args(params))
        assert rc == jbp_lib.EINVAL, (name, rc)
        assert lib.jbp_last_error(), name


def test_plain_c_program_links_and_calls_the_library(jbp_lib, tmp_path):
    """The boundary is usable from C99 as declared: a C program includes jbp.h,
    links libjbp.so and calls two host-only entry points and an argument check."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_jbp.c"
    src.write_text(r"""
#include <stdio.h>
#include "jbp.h"
int main(void) {
    uint8_t mul[16 * 16], div[16 * 16];
    int32_t shape[5];
    int64_t bytes = 0;
    if (jbp_gf_tables(16, mul, div) != JBP_OK) return 1;
    if (jbp_dft_tables(4, 64, shape, NULL, &bytes) != JBP_OK) return 2;
    if (jbp_decode(NULL, NULL) != JBP_EINVAL) return 3;
    printf("%d %d %d %lld %s\n", mul[2 * 16 + 8], div[3 * 16 + 3], shape[0], (long long)bytes,
           jbp_last_error()[0] ? "msg" : "nomsg");
    return 0;
}
""")
    lib_dir = os.path.dirname(jbp_lib.LIB_PATH)
    exe = tmp_path / "use_jbp"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", lib_dir, "-ljbp", "-Wl,-rpath," + lib_dir], check=True, capture_output=True, timeout=120)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    a, b, L, nbytes, msg = out.stdout.split()
    assert int(a) == 3          # x * x^3 = x^4 = x + 1 in GF(16) with x^4 + x + 1
    assert int(b) == 1          # 3 / 3
    assert int(L) == 256        # first multiple of 16 >= 4 * 63 + 1
    assert int(nbytes) > 0 and msg == "msg"
