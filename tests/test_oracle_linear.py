"""Pins of the oracle's linear homogenization function DMN^L and of the
offline-training objective (``oracle.linear``, Sec. 3.2):

  * one laminate by Milton's formula (eq. laminate) equals the laminate solved
    from its jump conditions directly: strains e_1 = E + c2 sym(a (x) n),
    e_2 = E - c1 sym(a (x) n), traction continuity (sigma_1 - sigma_2) n = 0;
  * the laminate does not depend on lam once lam is large enough;
  * equal phases give that phase back for any normals and weights;
  * Voigt and Reuss bounds (Loewner order) for every sample;
  * DMN^L of elastic phases equals the algorithmic tangent of the online
    oracle (Algorithm 1) on the same tree;
  * the gradients of J by automatic differentiation against central finite
    differences; weights with v < 0 get no gradient (w = <v>_+);
  * J at exact targets is the penalty term alone.
"""
import numpy as np
import pytest

import oracle
import oracle.linear as lin
from paper_2109_14403_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
SQ2 = np.sqrt(2.0)


def bmat(n):
    B = np.zeros((6, 3))
    r = 1 / SQ2
    B[0, 0], B[1, 1], B[2, 2] = n
    B[3, 1], B[3, 2] = r * n[2], r * n[1]
    B[4, 0], B[4, 2] = r * n[2], r * n[0]
    B[5, 0], B[5, 1] = r * n[1], r * n[0]
    return B


def laminate_by_jump_conditions(C1, C2, n, c1):
    c2 = 1 - c1
    B = bmat(n)
    # unknown jump a (3) for each unit macro strain: B^T (C1 e1 - C2 e2) = 0
    A = B.T @ (c2 * C1 + c1 * C2) @ B
    Cb = np.zeros((6, 6))
    for k in range(6):
        E = np.eye(6)[k]
        a = np.linalg.solve(A, -B.T @ (C1 - C2) @ E)
        e1, e2 = E + c2 * B @ a, E - c1 * B @ a
        Cb[:, k] = c1 * C1 @ e1 + c2 * C2 @ e2
    return Cb


def test_milton_laminate_equals_jump_conditions():
    C1s, C2s = syn.stiffness_pairs(4, seed=1)
    rng = np.random.default_rng(2)
    for s in range(4):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        c1 = rng.uniform(0.1, 0.9)
        lam = 2 * max(np.linalg.eigvalsh(C1s[s]).max(), np.linalg.eigvalsh(C2s[s]).max())
        Cm = lin.laminate(torch.tensor(C1s[s]), torch.tensor(C2s[s]), torch.tensor(n), c1, lam).numpy()
        Cj = laminate_by_jump_conditions(C1s[s], C2s[s], n, c1)
        np.testing.assert_allclose(Cm, Cj, rtol=1e-10, atol=1e-12 * np.abs(Cj).max())
        Cm5 = lin.laminate(torch.tensor(C1s[s]), torch.tensor(C2s[s]), torch.tensor(n), c1,
                           2.5 * lam).numpy()
        np.testing.assert_allclose(Cm5, Cm, rtol=1e-10, atol=1e-12 * np.abs(Cj).max())


def test_equal_phases_and_bounds():
    K = 4
    normals, v = syn.linear_params(K)
    C1s, C2s = syn.stiffness_pairs(6, seed=3)
    out = lin.forward(C1s, C1s, normals, v)
    np.testing.assert_allclose(out, C1s, rtol=1e-11, atol=1e-12)
    out = lin.forward(C1s, C2s, normals, v)
    w = np.maximum(v, 0)
    # volume fractions of the two phases (even leaves phase 1, odd leaves phase 2)
    f1 = w[0::2].sum() / w.sum()
    for s in range(6):
        voigt = f1 * C1s[s] + (1 - f1) * C2s[s]
        reuss = np.linalg.inv(f1 * np.linalg.inv(C1s[s]) + (1 - f1) * np.linalg.inv(C2s[s]))
        assert np.linalg.eigvalsh(voigt - out[s]).min() > -1e-10 * np.abs(voigt).max()
        assert np.linalg.eigvalsh(out[s] - reuss).min() > -1e-10 * np.abs(voigt).max()
        np.testing.assert_allclose(out[s], out[s].T, atol=1e-12 * np.abs(out[s]).max())


@pytest.mark.parametrize("K", [2, 4])
def test_linear_dmn_equals_online_tangent(K):
    """Elastic phases: the algorithmic tangent of Algorithm 1 is DMN^L."""
    w, n, ph = syn.tree(K)
    mats = syn.materials().copy()
    mats[1, 5] = 1e12  # never yields
    t = oracle.Tree(K, w, n, ph, mats)
    _, out, st, _ = oracle.eval_batch(t, np.full((1, 6), 1e-4), [300.0], 1.0, t.init_state(1, 293.0))
    C1 = syn.iso_mandel(72000.0, 0.22)
    C2 = syn.iso_mandel(2500.0, 0.38)
    ref = lin.forward(C1[None], C2[None], n, w)[0]
    np.testing.assert_allclose(oracle.split_out(out[0])["C"], ref, rtol=1e-10, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("p,q", [(1.0, 10.0), (2.0, 2.0)])
def test_gradients_match_finite_differences(p, q):
    K = 3
    normals, v = syn.linear_params(K, seed=11)
    v[2] = -0.05  # a dead leaf: w = 0
    C1s, C2s = syn.stiffness_pairs(5, seed=4)
    tn, tv = syn.linear_params(K, seed=12)
    Ct = lin.forward(C1s, C2s, tn, tv)
    J, gn, gv = lin.loss_grad(C1s, C2s, Ct, normals, v, p=p, q=q, penalty=10.0)
    assert gv[2] == 0.0
    h = 1e-6
    for i in range(normals.shape[0]):
        for c in range(3):
            a, b = normals.copy(), normals.copy()
            a[i, c] += h
            b[i, c] -= h
            fd = (lin.loss(C1s, C2s, Ct, a, v, p, q, 10.0)[0] - lin.loss(C1s, C2s, Ct, b, v, p, q, 10.0)[0]) / (2 * h)
            assert abs(fd - gn[i, c]) <= 1e-6 * max(np.abs(gn).max(), 1e-3)
    for j in range(v.size):
        if j == 2:
            continue
        a, b = v.copy(), v.copy()
        a[j] += h
        b[j] -= h
        fd = (lin.loss(C1s, C2s, Ct, normals, a, p, q, 10.0)[0] - lin.loss(C1s, C2s, Ct, normals, b, p, q, 10.0)[0]) / (2 * h)
        assert abs(fd - gv[j]) <= 1e-6 * max(np.abs(gv).max(), 1e-3)


def test_loss_at_exact_targets_is_the_penalty():
    K = 2
    normals, v = syn.linear_params(K, seed=5)
    v = v * 1.2
    C1s, C2s = syn.stiffness_pairs(3, seed=6)
    Ct = lin.forward(C1s, C2s, normals, v)
    J, d, pen, e = lin.loss(C1s, C2s, Ct, normals, v, penalty=7.0)
    assert d < 1e-14 and abs(pen - 7.0 * (v.sum() - 1) ** 2) < 1e-14
