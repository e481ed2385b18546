"""The C-ABI library builds, loads and exports every function include/*.h
declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return sorted(set(re.findall(r"\b(dmn_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2109_14403_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions("dmn.h") + declared_functions("dmn_mlp.h") + declared_functions("dmn_linear.h")
    assert "dmn_eval" in names and "dmn_create" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in dmn.h but not exported"


def test_binding_covers_the_headers():
    from paper_2109_14403_gb300 import dmn
    assert set(declared_functions("dmn.h") + declared_functions("dmn_mlp.h")
               + declared_functions("dmn_linear.h")) == set(dmn.SIGNATURES)


def test_default_options_and_error_string(lib):
    from paper_2109_14403_gb300 import dmn
    L = dmn.load()
    o = dmn.dmn_options()
    L.dmn_default_options(ctypes.byref(o))
    assert o.tol == 1e-10 and o.maxit == 50 and o.maxbacktrack == 8 and o.gamma == 0.5
    assert L.dmn_last_error() == b""


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    """Argument validation happens before any CUDA call."""
    import numpy as np
    from paper_2109_14403_gb300 import dmn, synthetic as syn
    L = dmn.load()
    w, n, ph = syn.tree(3)
    mats = dmn.materials_from_rows(syn.materials())
    h = ctypes.c_void_p()
    P = ctypes.c_void_p

    def create(K, w_, n_, ph_, nm=2):
        return L.dmn_create(ctypes.byref(h), K, w_.ctypes.data_as(P), n_.ctypes.data_as(P),
                            ph_.ctypes.data_as(P), ctypes.cast(mats, P), nm, None)

    assert create(11, w, n, ph) == 1
    assert b"outside 1..10" in L.dmn_last_error()
    bad = w.copy()
    bad[0] += 1e-6
    assert create(3, bad, n, ph) == 1
    assert b"sum" in L.dmn_last_error()
    bad = w.copy()
    bad[1] = 0.0
    bad[0] += w[1]
    assert create(3, bad, n, ph) == 1
    nz = n.copy()
    nz[2] = 0.0
    assert create(3, w, nz, ph) == 1
    bp = ph.copy()
    bp[0] = 7
    assert create(3, w, n, bp) == 1
    assert create(3, w, n, ph, nm=0) == 1


def test_release_library_has_no_bounds_log():
    """The index-check log exists only in the debug build; the release
    library says so (no CUDA call is made)."""
    from paper_2109_14403_gb300 import dmn
    if dmn.library_path().endswith("libdmn_debug.so"):
        pytest.skip("debug library selected in this process")
    with pytest.raises(RuntimeError, match="debug library"):
        dmn.bounds_log()
