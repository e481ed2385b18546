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
    w, n, ph = syn.tree(3)
    mats = dmn.materials_from_rows(syn.materials())
    P = ctypes.c_void_p
    for prec, vs in autotune.VARIANTS.items():
        for v in vs + (99,):
            o = dmn.dmn_options()
            L.dmn_default_options(ctypes.byref(o))
            o.precision = {"fp64": dmn.PREC_FP64, "mixed": dmn.PREC_MIXED}[prec]
            o.solve_variant = v
            h = ctypes.c_void_p()
            rc = L.dmn_create(ctypes.byref(h), 3, w.ctypes.data_as(P), n.ctypes.data_as(P),
                              ph.ctypes.data_as(P), ctypes.cast(mats, P), 2, ctypes.byref(o))
            msg = L.dmn_last_error()
            if v == 99:
                assert rc == 1 and b"solve_variant" in msg
            else:  # past the argument checks: fails (no device here) or succeeds (GPU)
                assert b"solve_variant" not in msg
                if rc == 0:
                    L.dmn_destroy(h)
