"""The C-ABI library builds, loads without a GPU, and exports every function
include/meb.h declares (no compute call is made here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "meb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(meb_[a-z_0-9]+)\s*\(", src)))


def test_header_symbols_exported():
    from paper_2605_31425_gb300 import build
    lib = ctypes.CDLL(build.build())
    names = declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_params_default_without_gpu():
    import paper_2605_31425_gb300 as meb
    p = meb.params_default()
    assert p.tol == 1e-10 and p.rho == 0.5 and p.tau == 10.0 and p.dense_max_d == 224


def test_binding_constants_match_header():
    """The ctypes binding's option, screen-mode and server-flag values are the
    header's, and its structs have the header's sizes (no GPU needed)."""
    import ctypes as ct
    from paper_2605_31425_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "meb.h")).read()
    defs = {k: int(v.rstrip("u"), 0) for k, v in re.findall(r"#define\s+(MEB_[A-Z0-9_]+)\s+(\w+)", src)
            if re.fullmatch(r"(0x)?[0-9a-fA-F]+u?", v)}
    checked = 0
    for name, val in defs.items():
        if hasattr(_lib, name):
            assert getattr(_lib, name) == val, name
            checked += 1
    assert checked >= 10
    for k, v in _lib.SCREEN_MODES.items():
        assert defs["MEB_SCREEN_" + k.upper()] == v
    lib = ct.CDLL(__import__("paper_2605_31425_gb300.build", fromlist=["build"]).build())
    p = _lib.MebParams()
    lib.meb_params_default(ct.byref(p))
    assert p.max_cg == 500 and p.max_readd == 8


def test_binding_struct_layouts_match_header(tmp_path):
    """sizeof and field offsets of the header's structs, from a C program
    compiled against include/meb.h, equal the ctypes binding's."""
    import ctypes as ct
    import shutil
    import subprocess
    from paper_2605_31425_gb300 import _lib
    if shutil.which("gcc") is None:
        import pytest
        pytest.skip("no C compiler")
    structs = {"meb_params": _lib.MebParams, "meb_info": _lib.MebInfo, "meb_stats": _lib.MebStats,
               "meb_batch_item": _lib.MebBatchItem, "meb_server_config": _lib.MebServerConfig,
               "meb_server_stats": _lib.MebServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "meb.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for cname, py in structs.items():
        assert int(out[cname]) == ct.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(out[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)
