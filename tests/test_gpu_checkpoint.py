"""Checkpoint and resume: the device state (eps_bar^n, theta^n, a^n and the
leaves' internal variables) is the whole history of a Gauss point.  Saving it
to host memory, creating a new handle (as a restarted program would) and
loading it back must continue the load path with identical bits."""
import numpy as np
import pytest

from paper_2109_14403_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("mats_name", ["j2", "pa66"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_resume_after_restore_is_bit_identical(prec, mats_name):
    from paper_2109_14403_gb300 import DMN
    dev = _dev()
    K, n = 5, 64
    w, nrm, ph = syn.tree(K)
    mats = syn.materials() if mats_name == "j2" else syn.materials_pa66()
    rng = np.random.default_rng(9)
    deps = torch.tensor(rng.normal(0, 2e-3, (6, n, 6)), device=dev)
    theta = torch.tensor(293.0 + np.cumsum(rng.uniform(0, 2, (6, n)), axis=0), device=dev)
    dt = 0.01
    d = DMN(K, w, nrm, ph, mats, tol=1e-12, precision=prec)
    s = d.init_state(torch.full((n,), syn.THETA_START, dtype=torch.float64, device=dev))
    outs = []
    for k in range(6):
        s, out, st, it = d.eval(deps[k], theta[k], dt, s)
        outs.append(out.clone())
        if k == 2:
            saved = s.cpu().clone()  # checkpoint after three increments
    d.close()
    # a restarted program: new handle, state loaded from the checkpoint
    d2 = DMN(K, w, nrm, ph, mats, tol=1e-12, precision=prec)
    s2 = saved.to(dev)
    for k in range(3, 6):
        s2, out2, st2, it2 = d2.eval(deps[k], theta[k], dt, s2)
        assert torch.equal(out2, outs[k])
    assert torch.equal(s2, s)
    d2.close()
