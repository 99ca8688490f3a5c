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
