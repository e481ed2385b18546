"""Host-side checks of the PA66 material (kind 3) that need no GPU: the
allocation-free entry point refuses it before touching the device, and bad
PA66 constants are rejected by the argument checks."""
import ctypes

import numpy as np

from paper_2109_14403_gb300 import dmn, synthetic as syn


def test_noalloc_rejects_pa66_leaves():
    L = dmn.load()
    K = 3
    w, n, ph = syn.tree(K)
    mats = dmn.materials_from_rows(syn.materials_pa66())
    P = ctypes.c_void_p
    rc = L.dmn_eval_noalloc(K, w.ctypes.data_as(P), n.ctypes.data_as(P), ph.ctypes.data_as(P),
                            ctypes.cast(mats, P), 2, None, None, 1, P(16), P(16), 1.0, P(16), P(32),
                            P(48), P(64), P(80))
    assert rc == 1 and b"PA66" in L.dmn_last_error()


def test_invalid_pa66_constants_are_rejected():
    L = dmn.load()
    K = 2
    w, n, ph = syn.tree(K)
    P = ctypes.c_void_p
    for col, bad, word in ((7, 1.5, b"hardening"), (8, 2.5, b"rate law"), (14, -1.0, b"WLF"),
                           (28, -1.0, b"Maxwell")):
        rows = syn.materials_pa66().copy()
        rows[1, col] = bad
        mats = dmn.materials_from_rows(rows)
        o = dmn.dmn_options()
        L.dmn_default_options(ctypes.byref(o))
        h = ctypes.c_void_p()
        rc = L.dmn_create(ctypes.byref(h), K, w.ctypes.data_as(P), n.ctypes.data_as(P), ph.ctypes.data_as(P),
                          ctypes.cast(mats, P), 2, ctypes.byref(o))
        assert rc == 1 and word in L.dmn_last_error(), (col, L.dmn_last_error())
    # and a PA66 tree deeper than 8 levels
    w9, n9, ph9 = syn.tree(9)
    mats = dmn.materials_from_rows(syn.materials_pa66())
    h = ctypes.c_void_p()
    o = dmn.dmn_options()
    L.dmn_default_options(ctypes.byref(o))
    rc = L.dmn_create(ctypes.byref(h), 9, w9.ctypes.data_as(P), n9.ctypes.data_as(P), ph9.ctypes.data_as(P),
                      ctypes.cast(mats, P), 2, ctypes.byref(o))
    assert rc == 1 and b"K <= 8" in L.dmn_last_error()
    assert np.isfinite(syn.MATRIX_PA66).all()
