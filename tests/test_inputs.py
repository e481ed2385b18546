"""Properties of the synthetic workloads that the GPU tests rely on (CPU only)."""
import numpy as np

import oracle
from paper_2109_14403_gb300 import synthetic as syn


def test_scaled_walk_exercises_the_line_search():
    """The K=8 walk scaled by 20 (used by the GPU backtracking test): in its
    second increment some points take a different path when backtracking is
    switched off, i.e. the oracle rejected full Newton steps there."""
    K, n = 8, 200
    w, nrm, ph = syn.tree(K)
    tree = oracle.Tree(K, w, nrm, ph, syn.materials())
    deps, theta = syn.random_walk_k8(n_points=n, n_incr=2)
    s = tree.init_state(n, syn.THETA_START)
    s, _, st, _ = oracle.eval_batch(tree, deps[0] * 20.0, theta[0], 1.0, s)
    assert (st == 0).all()
    _, _, st1, it1 = oracle.eval_batch(tree, deps[1] * 20.0, theta[1], 1.0, s)
    _, _, _, it0 = oracle.eval_batch(tree, deps[1] * 20.0, theta[1], 1.0, s, maxbacktrack=0)
    assert (st1 == 0).all()
    assert int(np.sum(it1 != it0)) >= 5
