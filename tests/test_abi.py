"""libhawkes builds for sm_103a, loads without a GPU, and exports every
function include/hawkes.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_2407_11349_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(hawkes_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return ctypes.CDLL(libbuild.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hawkes_create", "hawkes_destroy", "hawkes_set_events", "hawkes_set_counties",
                     "hawkes_resample_locations", "hawkes_loglik_grad", "hawkes_loglik_grad_async"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_the_header():
    from paper_2407_11349_gb300 import hawkes
    missing = [n for n in declared_functions() if n not in hawkes._SIGS]
    assert not missing


def test_strerror(lib):
    lib.hawkes_strerror.restype = ctypes.c_char_p
    assert lib.hawkes_strerror(0) == b"ok"
    assert b"sorted" in lib.hawkes_strerror(-2) or b"decreasing" in lib.hawkes_strerror(-2)


def test_library_is_sm_103a():
    # the fat binary must carry sm_103a code: nvcc was asked for nothing else
    assert libbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _declared_arities():
    """Parameter count of every function include/*.h declares."""
    out = {}
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(hawkes_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
            args = m.group(2).strip()
            out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_signatures_match_the_header():
    """The ctypes binding passes exactly as many arguments as each C
    declaration takes."""
    from paper_2407_11349_gb300 import hawkes
    arity = _declared_arities()
    assert len(arity) >= 40
    wrong = {n: (arity[n], len(hawkes._SIGS[n][1])) for n in arity
             if n in hawkes._SIGS and arity[n] != len(hawkes._SIGS[n][1])}
    assert not wrong, f"argument counts differ (header, binding): {wrong}"
