"""The C ABI library loads and exports every entry point of include/fmmlu.h.

CPU only: no compute call is made; host-side argument checks are exercised.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fmmlu.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(fmmlu_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_07325_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    import paper_2201_07325_gb300 as pkg
    return pkg.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("fmmlu_build_tree", "fmmlu_factor", "fmmlu_solve", "fmmlu_solve_adjoint",
                 "fmmlu_free", "fmmlu_stats", "fmmlu_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), f"{name} declared in fmmlu.h but not exported"


def test_host_side_argument_checks(lib):
    import paper_2201_07325_gb300 as pkg
    o = pkg.fmmlu_default_opts()
    assert o.leaf_size == 64 and o.n_proxy == 300 and o.proxy_radius_factor == 1.5
    out = ctypes.c_void_p()
    rc = lib.fmmlu_factor(None, None, None, None, 1.0, 1e-6, None, None, ctypes.byref(out))
    assert rc == -1 and "null" in pkg.fmmlu_last_error()
    assert lib.fmmlu_solve(None, None, None, 1, None) == -1
    assert lib.fmmlu_solve_adjoint(None, None, None, 1, None) == -1
    assert lib.fmmlu_stats(None, None, 0) == -1
    assert lib.fmmlu_build_tree(None, 0, None, None, ctypes.byref(out)) == -1
    assert lib.fmmlu_matvec(0, None, None, None, 1.0, 1.0, None, None, 1, None) == -1
    lib.fmmlu_free(None)
    bad = pkg.fmmlu_default_opts(proxy_radius_factor=0.9)
    rc = lib.fmmlu_build_tree(ctypes.c_void_p(8), 10, ctypes.byref(bad), None, ctypes.byref(out))
    assert rc == -1 and "proxy_radius_factor" in pkg.fmmlu_last_error()


def test_python_opts_layout_matches_the_header(tmp_path):
    """The ctypes mirror of fmmlu_opts has the C struct's size and field
    offsets (a C program compiled against include/fmmlu.h prints them)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2201_07325_gb300.binding import fmmlu_opts
    fields = [f for f, _ in fmmlu_opts._fields_]
    prog = tmp_path / "layout.c"
    body = "\n".join(f'  printf("{f} %zu\\n", offsetof(fmmlu_opts, {f}));' for f in fields)
    prog.write_text(
        "#include <stddef.h>\n#include <stdio.h>\n#include <stdint.h>\n"
        f'#include "{HEADER}"\n'
        "int main(void) {\n"
        '  printf("sizeof %zu\\n", sizeof(fmmlu_opts));\n'
        f"{body}\n  return 0;\n}}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(prog)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    assert int(out["sizeof"]) == ctypes.sizeof(fmmlu_opts)
    for f in fields:
        assert int(out[f]) == getattr(fmmlu_opts, f).offset, f


def test_solve_and_tuning_options(lib):
    import paper_2201_07325_gb300 as pkg
    o = pkg.fmmlu_default_opts()
    assert o.solve_chunk == 0 and o.solve_graph == 1 and o.autotune == 1
    assert o.autotune_cache is None
    out = ctypes.c_void_p()
    for field, value in (("solve_chunk", 40), ("solve_chunk", 8192), ("solve_graph", 3),
                         ("autotune", 2), ("schur_emulation", 3), ("id_method", -1),
                         ("proxy_rule", 2)):
        bad = pkg.fmmlu_default_opts(**{field: value})
        rc = lib.fmmlu_build_tree(ctypes.c_void_p(8), 10, ctypes.byref(bad), None,
                                  ctypes.byref(out))
        assert rc == -1, (field, value)
    ok = pkg.fmmlu_default_opts(autotune_cache="/nonexistent/dir/tune.txt", solve_chunk=4096)
    assert ok.autotune_cache == b"/nonexistent/dir/tune.txt"
