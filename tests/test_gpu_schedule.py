"""Scheduling paths on the GPU: CUDA-graph increments, the uneven batch of
three trees (K = 6, 7, 8) against the oracle, and the autotuner."""
import numpy as np
import pytest

import oracle
from paper_2109_14403_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def test_graph_replay_equals_direct_launches():
    from paper_2109_14403_gb300 import DMN
    from paper_2109_14403_gb300.graph import IncrementGraph
    dev = _dev()
    n = 2000
    w, nrm, ph = syn.tree(8)
    d = DMN(8, w, nrm, ph, syn.materials(), precision="mixed")
    deps, theta = syn.random_walk_k8(n_points=n, n_incr=3)
    s = d.init_state(torch.full((n,), 293.0, dtype=torch.float64, device=dev))
    g = IncrementGraph([(d, n)])
    g.set_state(0, s)
    for k in range(3):
        g.deps[0].copy_(torch.tensor(deps[k] * 5, device=dev))
        g.theta[0].copy_(torch.tensor(theta[k], device=dev))
        g.step()
        s, out, st, it = d.eval(torch.tensor(deps[k] * 5, device=dev),
                                torch.tensor(theta[k], device=dev), 1.0, s)
        torch.cuda.synchronize()
        assert torch.equal(out, g.out[0]) and torch.equal(s, g.current_state(0))
        assert torch.equal(it, g.iters[0])
    d.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_uneven_batch_three_depths_against_oracle(prec):
    from paper_2109_14403_gb300 import DMN
    dev = _dev()
    n = 3000
    tid, deps, theta = syn.uneven_batch(n_points=n, n_incr=2)
    trees = syn.uneven_trees()
    mats = syn.materials()
    tol = {"fp64": 1e-10, "mixed": 1e-8}[prec]
    iters_all = []
    for i, K in enumerate(syn.UNEVEN_DEPTHS):
        w, nrm, ph = trees[i]
        sel = np.nonzero(tid == i)[0]
        d = DMN(K, w, nrm, ph, mats, tol=1e-12, precision=prec)
        s = d.init_state(torch.full((len(sel),), 293.0, dtype=torch.float64, device=dev))
        ot = oracle.Tree(K, w, nrm, ph, mats)
        chk = sel[:: max(1, len(sel) // 40)]
        pos = np.searchsorted(sel, chk)
        so = ot.init_state(len(chk), 293.0)
        for k in range(2):
            s, out, st, it = d.eval(torch.tensor(deps[k][sel], device=dev),
                                    torch.tensor(theta[k][sel], device=dev), 1.0, s)
            so, oo, sto, _ = oracle.eval_batch(ot, deps[k][chk], theta[k][chk], 1.0, so)
            g = out.cpu().numpy()[pos]
            assert (st.cpu().numpy() == 0).all() and (sto == 0).all()
            rel = np.linalg.norm(g[:, :6] - oo[:, :6], axis=1) / np.linalg.norm(oo[:, :6], axis=1)
            assert rel.max() < tol
            iters_all.append(it.cpu().numpy())
        d.close()
    it = np.concatenate(iters_all)
    assert it.max() >= 3 * it.min()  # uneven Newton iteration counts


def test_autotuner_writes_a_choice(tmp_path):
    from paper_2109_14403_gb300 import autotune
    _dev()
    p = str(tmp_path / "tuning.json")
    e = autotune.tune(K=6, n_points=4096, n_steps=2, warmup=1, path=p)
    assert e["variant"] in autotune.VARIANTS["mixed"]
    assert autotune.lookup(6, "mixed", p) == e["variant"]


@pytest.mark.parametrize("variant", [13, 23])
def test_warm_graph_replay_equals_direct_launches(variant):
    """The headline increment (network input, four GEMMs, warm-started solve)
    replayed as a CUDA graph gives the bits of the same launches made
    directly, over three increments (every rotation phase of the state
    buffers), for the compact and the warp form of the solve."""
    from paper_2109_14403_gb300 import DMN
    from paper_2109_14403_gb300.graph import WarmIncrementGraph
    from paper_2109_14403_gb300.mlp import MLP
    dev = _dev()
    n = 2048
    w, nrm, ph = syn.tree(8)
    d = DMN(8, w, nrm, ph, syn.materials(), precision="mixed", tol=1e-12, solve_variant=variant)
    net = MLP(K=8, hidden=512, n_hidden=3, max_batch=n, seed=0)
    p = net.params()
    din, dout = net.layer_dims()[-1]
    p[-(din * dout + dout):] *= 1e-6  # small predicted increments
    net.set_params(p)
    deps, theta = syn.random_walk_k8(n_points=n, n_incr=5)
    D = torch.tensor(deps * 5, device=dev)
    T = torch.tensor(theta, device=dev)
    s0 = d.init_state(torch.full((n,), 293.0, dtype=torch.float64, device=dev))
    s1, _, _, _ = d.eval(D[0], T[0], 1.0, s0)
    g = WarmIncrementGraph(d, net, n, s0, s1)
    prev, cur = s0, s1
    for k in range(1, 5):
        g.deps.copy_(D[k])
        g.theta.copy_(T[k])
        g.step()
        x = net.input(D[k], T[k], cur, prev)
        da = net.predict(x)
        nxt, out, st, it = d.eval_warm(D[k], T[k], 1.0, cur, da)
        torch.cuda.synchronize()
        assert torch.equal(da, g.da)
        assert torch.equal(out, g.out) and torch.equal(st, g.status) and torch.equal(it, g.iters)
        assert torch.equal(nxt, g.current_state())
        prev, cur = cur, nxt
    net.close()
    d.close()
