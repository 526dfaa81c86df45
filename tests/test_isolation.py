"""The oracle and the CUDA path share no code, and only the test suite, the smoke
test and the bench's CPU legs reach the oracle (static checks of the sources)."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2605_26580_gb300")


def _files(folder, exts):
    for dirpath, dirnames, names in os.walk(folder):
        dirnames[:] = [d for d in dirnames if not d.startswith(("_", "."))]
        for n in names:
            if n.endswith(exts):
                yield os.path.join(dirpath, n)


def _imports(path):
    """(module name, enclosing function or None) of every import in a Python file."""
    tree = ast.parse(open(path).read(), path)
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)):
                visit(child, fn or child.name)
                continue
            if isinstance(child, ast.Import):
                out.extend((a.name, fn) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                out.append(((child.module or ""), fn))
            visit(child, fn)

    visit(tree, None)
    return out


def _includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', open(path).read(), re.M)


def test_package_never_imports_the_oracle():
    for path in _files(PKG, (".py",)):
        for mod, _ in _imports(path):
            assert not mod.split(".")[0] == "oracle", (path, mod)


def test_cuda_sources_include_nothing_of_the_oracle():
    for path in list(_files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h"))) + \
            list(_files(os.path.join(ROOT, "include"), (".h",))):
        for inc in _includes(path):
            assert "oracle" not in inc, (path, inc)


def test_oracle_uses_nothing_of_the_cuda_path():
    for inc in _includes(os.path.join(ROOT, "oracle", "jbp_oracle.c")):
        # its own header, else only C library headers: nothing of the CUDA side (jbp*.h, csrc, include)
        assert inc == "jbp_oracle.h" or ("/" not in inc and not inc.startswith("jbp")), inc
    for path in _files(os.path.join(ROOT, "oracle"), (".py",)):
        for mod, _ in _imports(path):
            assert not mod.startswith("paper_2605_26580_gb300"), (path, mod)


def test_oracle_is_reached_only_from_the_allowed_places():
    # bench.py: the reference arm, the CPU-baseline leg, and the workloads that time
    # the oracle on a sample beside the GPU and report each variant's error against it
    allowed = {"bench.py": {"run_reference", "cpu_baseline_leg", "wl_small", "wl_precision", "wl_ura"},
               "__graft_entry__.py": {"build", "smoke"}}
    for name, fns in allowed.items():
        users = {fn for mod, fn in _imports(os.path.join(ROOT, name)) if mod.split(".")[0] == "oracle"}
        assert users and users <= fns, (name, users)


def test_shared_input_module_holds_no_decoder_arithmetic():
    """The seeded input generators are the one module both sides use; they build
    codes, codewords and channel outputs but import no decoder."""
    mods = {m.split(".")[0] for m, _ in _imports(os.path.join(PKG, "inputs.py"))}
    # (torch may run the binary encoder's product on a device; it loads no decoder)
    assert not mods & {"oracle", "ctypes", "paper_2605_26580_gb300"}, mods
    src = open(os.path.join(PKG, "inputs.py")).read()
    for word in ("channel_node", "check_node", "wht", "hadamard", "decode("):
        assert word not in src.lower(), word
