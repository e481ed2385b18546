"""Host logic of the autotuner: selection and the JSON table (no GPU)."""
import json

from paper_2109_14403_gb300 import autotune


def test_choose_takes_the_fastest_and_breaks_ties_low():
    assert autotune.choose({2: 15.4, 3: 12.6, 4: 13.0}) == 3
    assert autotune.choose({2: 10.0, 3: 10.0, 4: 11.0}) == 2


def test_lookup_reads_the_table(tmp_path):
    p = tmp_path / "t.json"
    p.write_text(json.dumps({autotune.key(8, "mixed"): {"variant": 4}}))
    assert autotune.lookup(8, "mixed", str(p)) == 4
    assert autotune.lookup(7, "mixed", str(p)) == 0
    assert autotune.lookup(8, "mixed", str(tmp_path / "missing.json")) == 0


def test_variants_are_accepted_by_the_library():
    """Every variant the tuner may choose passes dmn_create's check (the
    check runs before any CUDA call, so a rejected one fails here on CPU)."""
    import ctypes
    import numpy as np
    from paper_2109_14403_gb300 import dmn, synthetic as syn
    L = dmn.load()
    w, n, ph = syn.tree(8)  # every form serves K = 8
    mats = dmn.materials_from_rows(syn.materials())
    P = ctypes.c_void_p
    for prec, vs in autotune.VARIANTS.items():
        for v in vs + (99,):
            if prec == "fp64" and v >= 22:
                continue
            o = dmn.dmn_options()
            L.dmn_default_options(ctypes.byref(o))
            o.precision = {"fp64": dmn.PREC_FP64, "mixed": dmn.PREC_MIXED}[prec]
            o.solve_variant = v
            h = ctypes.c_void_p()
            rc = L.dmn_create(ctypes.byref(h), 8, w.ctypes.data_as(P), n.ctypes.data_as(P),
                              ph.ctypes.data_as(P), ctypes.cast(mats, P), 2, ctypes.byref(o))
            msg = L.dmn_last_error()
            if v == 99:
                assert rc == 1 and b"solve_variant" in msg
            else:  # past the argument checks: fails (no device here) or succeeds (GPU)
                assert b"solve_variant" not in msg
                if rc == 0:
                    L.dmn_destroy(h)


def test_workload_keys_fall_back_to_the_random_walk(tmp_path):
    p = tmp_path / "t.json"
    p.write_text(json.dumps({autotune.key(8, "mixed"): {"variant": 13},
                             autotune.key(8, "mixed", "plastic"): {"variant": 23}}))
    assert autotune.key(8, "mixed") == "K=8,mixed"
    assert autotune.key(8, "mixed", "uneven") == "K=8,mixed,uneven"
    assert autotune.lookup(8, "mixed", str(p), workload="plastic") == 23
    assert autotune.lookup(8, "mixed", str(p), workload="uneven") == 13
    assert autotune.lookup(8, "mixed", str(p)) == 13


def test_warp_variants_rejected_for_unsupported_trees():
    """The warp form serves 6 <= K <= 8 in mixed precision; elsewhere
    dmn_create refuses it before any CUDA call (the tuner skips it)."""
    import ctypes
    from paper_2109_14403_gb300 import dmn, synthetic as syn
    L = dmn.load()
    P = ctypes.c_void_p
    mats = dmn.materials_from_rows(syn.materials())
    for K, prec in ((5, dmn.PREC_MIXED), (8, dmn.PREC_FP64), (9, dmn.PREC_MIXED)):
        w, n, ph = syn.tree(K)
        o = dmn.dmn_options()
        L.dmn_default_options(ctypes.byref(o))
        o.precision, o.solve_variant = prec, 23
        h = ctypes.c_void_p()
        rc = L.dmn_create(ctypes.byref(h), K, w.ctypes.data_as(P), n.ctypes.data_as(P),
                          ph.ctypes.data_as(P), ctypes.cast(mats, P), 2, ctypes.byref(o))
        assert rc == dmn.DMN_ERR_ARG and b"one warp per point" in L.dmn_last_error()
