"""The index-checking build of the library (libdmn_debug.so, compiled with
DMN_BOUNDS_CHECK): every node, leaf, state-offset and shared-memory slot index
of the solve kernels is checked, a bad one is counted, replaced by 0 and
flagged on its point (status bit DMN_PT_BOUNDS) instead of trapping.  The
oracle cases of depth 1-3 run through it -- the owner-mapped and the compact
form, both precisions, with plastic increments -- plus the warp form at K = 6
and a PA66 tree; every point must match the oracle with no bounds bit and the
log must stay empty.  A child process loads the debug library
(DMN_LIBRARY=debug): this process has the release library loaded."""
import os
import subprocess
import sys
import textwrap

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import numpy as np, torch
    import oracle
    from paper_2109_14403_gb300 import DMN, dmn, synthetic as syn
    dmn.load()
    assert dmn.library_path().endswith("libdmn_debug.so")
    dev = torch.device("cuda:0")
    dmn.bounds_log(clear=True)

    def case(K, prec, variant, mats, scale, n=37, dt=0.7, seed=0):
        rng = np.random.default_rng(400 + K + seed)
        deps = rng.normal(0, scale, size=(2, n, 6))
        theta = 293.0 + np.cumsum(rng.uniform(0, 5, size=(2, n)), axis=0)
        w, nrm, ph = syn.tree(K)
        d = DMN(K, w, nrm, ph, mats, tol=1e-12, precision=prec, solve_variant=variant)
        tree = oracle.Tree(K, w, nrm, ph, mats)
        s = d.init_state(torch.full((n,), syn.THETA_START, dtype=torch.float64, device=dev))
        so = tree.init_state(n, syn.THETA_START)
        for k in range(2):
            s, out, st, it = d.eval(torch.tensor(deps[k], device=dev), torch.tensor(theta[k], device=dev), dt, s)
            so, oo, sto, _ = oracle.eval_batch(tree, deps[k], theta[k], dt, so)
            st = st.cpu().numpy()
            assert (st == 0).all(), (K, prec, variant, np.unique(st))
            g = out.cpu().numpy()[:, :6]
            rel = np.linalg.norm(g - oo[:, :6], axis=1) / np.maximum(np.linalg.norm(oo[:, :6], axis=1), 1e-3)
            assert rel.max() < (1e-10 if prec == "fp64" else 1e-8), (K, prec, variant, rel.max())
        d.close()

    j2 = syn.materials()
    for K in (1, 2, 3):
        for prec, variants in (("fp64", (0, 11)), ("mixed", (0, 13))):
            for v in variants:
                case(K, prec, v, j2, 3e-3)
    case(6, "mixed", 22, j2, 3e-3)
    case(2, "mixed", 0, syn.materials_pa66(), 2e-3, dt=0.01)
    count, index, bound, line = dmn.bounds_log(clear=True)
    assert count == 0, f"{count} bad indices, first {index} of {bound} at line {line}"
    print("debug build ok")
""")


def test_debug_build_runs_the_small_oracle_cases_clean():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, DMN_LIBRARY="debug", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "debug build ok" in r.stdout

