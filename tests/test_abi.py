"""The C-ABI library builds, loads and exports every entry point of include/elmfb.h.

No compute call is made (no GPU needed).
"""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared():
    names = set()
    for hp in HEADERS:
        src = open(hp).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(elmfb_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2409_01949_gb300 import build as B
    if not os.path.exists(B.LIB) and shutil.which("nvcc") is None and \
            not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no nvcc to build libelmfb.so")
    return B.build()


def test_every_declared_symbol_is_exported(libpath):
    lib = ctypes.CDLL(libpath)
    declared = _declared()
    assert len(declared) >= 15
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_declared_symbols(libpath):
    import paper_2409_01949_gb300 as E
    assert set(E.exported_symbols()) <= _declared()
    E.lib()   # loads with the declared signatures


def test_default_solve_options_without_gpu(libpath):
    import paper_2409_01949_gb300 as E
    o = E.default_solve_opts()
    assert o.method == E.SOLVE_LSQR and o.max_iter == 15000 and o.check_every == 50
