"""Pins of the oracle's mixed strain / stress control with adiabatic heating
(``oracle.eval_mixed``): closed forms on homogeneous trees, where every leaf
carries the same isotropic material and the DMN reduces to that material.

  * uniaxial stress, isothermal, linear thermoelastic: Hooke's law,
    eps_11 = s/E + alpha dT, eps_22 = eps_33 = -nu s/E + alpha dT;
  * uniaxial stress, adiabatic, linear thermoelastic: the implicit heat
    balance c dT = -3 K alpha theta tr(eps) (eq. macro_heat without source and
    flux; coupling term of Sec. 4 with psi linear in theta) with
    tr(eps) = s/(3K) + 3 alpha dT gives the quadratic
    9 K alpha^2 dT^2 + (c + 9 K alpha^2 theta_0 + alpha s) dT + alpha theta_0 s = 0
    (Kelvin's thermoelastic effect: tension cools);
  * uniaxial stress beyond yield, J2 with linear hardening: p = (s - sigma_Y)/H,
    eps_11 = s/E + p, eps_22 = -nu s/E - p/2; adiabatic, the scalar balance
    c dT = -alpha theta s - 9 K alpha^2 theta dT + sigma_Y(theta) p(theta)
    solved by bracketing (scipy.optimize.brentq);
  * an all-strain mask reproduces eval_batch bit for bit;
  * a composite tree: the returned state meets every prescribed stress and the
    heat balance when evaluated again with eval_batch;
  * the tangent predictor: exact (one evaluation) for a linear thermoelastic
    composite under isothermal mixed control; on the cyclic path the same
    solution with fewer evaluations.
"""
import numpy as np
import pytest

import oracle
from paper_2109_14403_gb300 import synthetic as syn

TH0 = 293.0
ALL_STRESS, ADIABATIC = 0x3F, 0x40


def homogeneous(row, K=3):
    w, n, ph = syn.tree(K)
    return oracle.Tree(K, w, n, np.zeros_like(ph), [row])


def uniaxial(s, n=1):
    t = np.zeros((n, 6))
    t[:, 0] = s
    return t


@pytest.mark.parametrize("theta", [TH0, 340.0])
def test_uniaxial_stress_hooke(theta):
    E, nu, al = 70000.0, 0.22, 5e-6
    t = homogeneous([0, E, nu, al, TH0, 0, 0, 0])
    s = 120.0
    de, th, so, out, st, outer = oracle.eval_mixed(t, [ALL_STRESS], uniaxial(s), np.zeros((1, 6)),
                                                   theta, 1.0, 2.0, t.init_state(1, TH0))
    assert st[0] == 0 and th[0] == theta
    dT = theta - TH0
    ref = np.array([s / E + al * dT, -nu * s / E + al * dT, -nu * s / E + al * dT, 0, 0, 0])
    np.testing.assert_allclose(de[0], ref, rtol=0, atol=1e-15)
    np.testing.assert_allclose(out[0, :6], uniaxial(s)[0], rtol=0, atol=1e-10 * s)


def test_uniaxial_stress_adiabatic_kelvin():
    E, nu, al, c, dt = 70000.0, 0.22, 5e-6, 2.0, 0.01
    t = homogeneous([0, E, nu, al, TH0, 0, 0, 0])
    K = E / (3 * (1 - 2 * nu))
    for s in (100.0, -250.0):
        de, th, so, out, st, outer = oracle.eval_mixed(t, [ALL_STRESS | ADIABATIC], uniaxial(s),
                                                       np.zeros((1, 6)), TH0, dt, c,
                                                       t.init_state(1, TH0), tol_outer=1e-13)
        A, B, C = 9 * K * al**2, c + 9 * K * al**2 * TH0 + al * s, al * TH0 * s
        dT = (-B + np.sqrt(B * B - 4 * A * C)) / (2 * A)
        assert st[0] == 0
        assert np.sign(dT) == -np.sign(s)
        assert abs(th[0] - TH0 - dT) <= 1e-9 * abs(dT)
        np.testing.assert_allclose(de[0, :3], [s / E + al * dT, -nu * s / E + al * dT,
                                               -nu * s / E + al * dT], rtol=1e-10)


def test_uniaxial_stress_j2_isothermal_and_adiabatic():
    from scipy.optimize import brentq
    E, nu, al, sy0, dsy, H = 2500.0, 0.38, 8e-5, 50.0, -0.3, 300.0
    t = homogeneous([1, E, nu, al, TH0, sy0, dsy, H])
    K = E / (3 * (1 - 2 * nu))
    s, c, dt = 80.0, 1.5, 1.0
    de, th, so, out, st, outer = oracle.eval_mixed(
        t, [ALL_STRESS, ALL_STRESS | ADIABATIC], uniaxial(s, 2), np.zeros((2, 6)), TH0, dt, c,
        t.init_state(2, TH0), max_outer=50, tol_outer=1e-13)
    assert (st == 0).all()
    p = (s - sy0) / H
    np.testing.assert_allclose(de[0, :3], [s / E + p, -nu * s / E - p / 2, -nu * s / E - p / 2],
                               rtol=1e-12)

    def heat(d):
        th_ = TH0 + d
        sy = sy0 + dsy * d
        return c * d + al * th_ * s + 9 * K * al**2 * th_ * d - sy * (s - sy) / H
    dT = brentq(heat, -50.0, 50.0, xtol=1e-14)
    p = (s - (sy0 + dsy * dT)) / H
    assert abs(th[1] - TH0 - dT) <= 1e-9 * abs(dT)
    np.testing.assert_allclose(de[1, :3], [s / E + p + al * dT, -nu * s / E - p / 2 + al * dT,
                                           -nu * s / E - p / 2 + al * dT], rtol=1e-10)
    # the plastic strain stored in the state: (p, -p/2, -p/2) and accumulated p
    z = so[1, 8 + 3 * t.nnode:]
    np.testing.assert_allclose(z[:3], [p, -p / 2, -p / 2], rtol=1e-10)
    assert abs(z[6] - p) <= 1e-10 * p


def test_all_strain_mask_is_eval_batch():
    K = 4
    w, n, ph = syn.tree(K)
    t = oracle.Tree(K, w, n, ph, syn.materials())
    deps, theta = syn.single_increment(5, seed=3, scale=2e-3)
    s0 = t.init_state(5, TH0)
    de, th, so, out, st, outer = oracle.eval_mixed(t, np.zeros(5, np.uint8), deps, np.zeros((5, 6)),
                                                   theta, 0.5, 2.0, s0)
    so2, out2, st2, _ = oracle.eval_batch(t, deps, theta, 0.5, s0)
    assert (outer == 1).all() and (st == st2).all()
    assert np.array_equal(de, deps) and np.array_equal(th, theta)
    assert np.array_equal(out, out2) and np.array_equal(so, so2)


def test_composite_meets_the_prescribed_conditions():
    K = 5
    w, n, ph = syn.tree(K)
    t = oracle.Tree(K, w, n, ph, syn.materials_cyclic())
    c = syn.effective_heat_capacity(w, ph)
    rng = np.random.default_rng(5)
    m = 6
    mask = np.array([0x7F, 0x3F, 0x06, 0x46, 0x40, 0x7E], np.uint8)
    target = rng.normal(0, 40.0, (m, 6))
    strain = ((mask[:, None] >> np.arange(6)) & 1) == 0
    target[strain] = rng.normal(0, 3e-3, strain.sum())
    dt = 0.01
    s0 = t.init_state(m, TH0)
    de, th, so, out, st, outer = oracle.eval_mixed(t, mask, target, np.zeros((m, 6)), TH0, dt, c, s0,
                                                   max_outer=40, tol_outer=1e-11)
    assert (st == 0).all() and (outer >= 2).all()
    _, o2, st2, _ = oracle.eval_batch(t, de, th, dt, s0)
    assert (st2 == 0).all()
    for i in range(m):
        for comp in range(6):
            if (mask[i] >> comp) & 1:
                assert abs(o2[i, comp] - target[i, comp]) <= 1e-9 * max(1.0, np.abs(o2[i, :6]).max())
            else:
                assert de[i, comp] == target[i, comp]
        if mask[i] & ADIABATIC:
            assert abs(c * (th[i] - TH0) / dt - o2[i, 48]) <= 1e-9 * c / dt
        else:
            assert th[i] == TH0


def test_not_converged_flag():
    t = homogeneous([1, 2500.0, 0.38, 8e-5, TH0, 50.0, -0.3, 300.0])
    de, th, so, out, st, outer = oracle.eval_mixed(t, [ALL_STRESS], uniaxial(80.0), np.zeros((1, 6)),
                                                   TH0, 1.0, 1.9, t.init_state(1, TH0), max_outer=2)
    assert st[0] == 8 and outer[0] == 2


def test_predictor_is_exact_for_linear_phases():
    K = 4
    w, n, ph = syn.tree(K)
    t = oracle.Tree(K, w, n, ph, [[0, 72000.0, 0.22, 5e-6, TH0, 0, 0, 0],
                                  [0, 2500.0, 0.38, 8e-5, TH0, 0, 0, 0]])
    m = 4
    s0 = t.init_state(m, TH0)
    # previous increment: a strain-controlled step to a nonzero state
    rng = np.random.default_rng(11)
    d1 = rng.normal(0, 1e-3, (m, 6))
    s1, o1, st1, _ = oracle.eval_batch(t, d1, 300.0, 1.0, s0)
    mask = np.array([ALL_STRESS, 0x06, 0x3E, 0x01], np.uint8)
    target = rng.normal(0, 30.0, (m, 6))
    strain = ((mask[:, None] >> np.arange(6)) & 1) == 0
    target[strain] = rng.normal(0, 1e-3, strain.sum())
    de, th, so, out, st, outer = oracle.eval_mixed(t, mask, target, np.zeros((m, 6)), 310.0, 1.0,
                                                   2.0, s1, out_prev=o1, tol_outer=1e-9)
    assert (st == 0).all() and (outer == 1).all()


def test_predictor_saves_evaluations_on_the_cyclic_path():
    K = 4
    w, n, ph = syn.tree(K)
    t = oracle.Tree(K, w, n, ph, syn.materials_cyclic())
    c = syn.effective_heat_capacity(w, ph)
    mask, target, dt, amp, direction = syn.cyclic_stress(6, 1, seed=5)
    runs = []
    for predict in (False, True):
        s = t.init_state(mask.size, TH0)
        de, th, out = np.zeros((mask.size, 6)), np.full(mask.size, TH0), None
        total = 0
        for k in range(target.shape[0]):
            de, th, s, out, st, outer = oracle.eval_mixed(
                t, mask, target[k], de, th, dt, c, s, tol_outer=1e-11,
                out_prev=out if predict else None)
            assert (st == 0).all()
            total += outer.sum()
        runs.append((total, de, th))
    assert runs[1][0] < runs[0][0]
    np.testing.assert_allclose(runs[1][1], runs[0][1], rtol=0, atol=1e-9 * np.abs(runs[0][1]).max())
    np.testing.assert_allclose(runs[1][2], runs[0][2], rtol=0, atol=1e-9)
