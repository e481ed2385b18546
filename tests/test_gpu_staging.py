"""State staging of the compact solve.  A point's state block goes into shared
memory by bulk copies (cp.async.bulk on an mbarrier); the copies need the
caller's state 16-byte aligned, which every entry point checks before any
launch (a misaligned state is an argument error, nothing runs).  The staged
solve must match the oracle (the parity tests) and never report a staging
timeout (status bit 32) on a normal batch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2109_14403_gb300 import DMN, synthetic as syn  # noqa: E402

STAGING_TIMEOUT = 32


def _misaligned_copy(s):
    """The same values in a buffer that starts 8 bytes past a 16-byte boundary."""
    n, sw = s.shape
    buf = torch.empty(n * sw + 1, dtype=torch.float64, device=s.device)
    v = buf[1:].view(n, sw)
    v.copy_(s)
    assert v.data_ptr() % 16 == 8
    return v


@pytest.mark.parametrize("K,prec,variant", [(8, "mixed", 13), (5, "fp64", 11), (3, "mixed", 13)])
def test_staged_state_loads(K, prec, variant):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    n = 97
    rng = np.random.default_rng(900 + K)
    w, nrm, ph = syn.tree(K)
    mats = syn.materials()
    d = DMN(K, w, nrm, ph, mats, tol=1e-12, precision=prec, solve_variant=variant)
    tree = oracle.Tree(K, w, nrm, ph, mats)
    s = d.init_state(torch.full((n,), syn.THETA_START, dtype=torch.float64, device=dev))
    so = tree.init_state(n, syn.THETA_START)
    for k in range(3):
        deps = rng.normal(0, 3e-3, size=(n, 6))
        theta = syn.THETA_START + 2.0 * (k + 1) + rng.uniform(0, 1, n)
        s, out, st, it = d.eval(torch.tensor(deps, device=dev), torch.tensor(theta, device=dev), 0.5, s)
        so, oo, sto, _ = oracle.eval_batch(tree, deps, theta, 0.5, so)
        st = st.cpu().numpy()
        assert ((st & STAGING_TIMEOUT) == 0).all()
        assert (st == 0).all(), np.unique(st)
        g = out.cpu().numpy()[:, :6]
        rel = np.linalg.norm(g - oo[:, :6], axis=1) / np.maximum(np.linalg.norm(oo[:, :6], axis=1), 1e-3)
        assert rel.max() < (1e-10 if prec == "fp64" else 1e-8), rel.max()
    with pytest.raises(RuntimeError, match="16-byte aligned"):
        d.eval(torch.tensor(deps, device=dev), torch.tensor(theta, device=dev), 0.5, _misaligned_copy(s))
    d.close()
