"""Pins of the oracle's PA66 leaf (kind 3, Sec. 4 of the paper: eq. PA66 psi,
the Maxwell branches with thermorheologically simple viscosities and the WLF
shift, J2 viscoplasticity with power-law hardening and thermal softening Gamma,
the coupling term D and the dissipation), each against something other than
the oracle's own formulas:

  * the complex-step derivatives (d sigma/d eps, d sigma/d theta, dD/d eps,
    dD/d theta) against central finite differences;
  * frozen branches (tau_i -> infinity): the linear thermoelastic law with
    E_inf + sum E_i, built from the projector formulas C = 3K P1 + 2G P2;
  * relaxed branches (tau_i -> 0): the same law with E_inf alone;
  * one Maxwell branch under held strain: after k steps the branch stresses
    are 3 K_1 e r_K^k and 2 G_1 e' r_G^k with r = 1 / (1 + dt / (a tau)),
    tau_K = tau E/K and tau_G = tau E/G (implicit Euler of the branch ODE),
    and for dt -> 0 the exponential relaxation exp(-t K / (tau E));
  * thermorheological simplicity: at temperature theta the viscoelastic
    response equals the one at theta_ref with every tau_i scaled by a_theta;
  * the coupling term: D - Diss = theta psi_{theta eps} : eps_dot +
    theta psi_{theta z} . z_dot with psi of eq. (PA66 psi) differentiated
    numerically;
  * the viscoplastic step: dp = dt (sigma_Y/eta) <(q - sigma_Y - H)/sigma_Y>^m
    at the returned stress, flow along the returned deviator (normality),
    and q -> sigma_Y + H as eta_0 -> 0;
  * a homogeneous PA66 tree reproduces the leaf (all 79 internal variables).
"""
import numpy as np
import pytest

import oracle
from paper_2109_14403_gb300 import synthetic as syn

ROW = np.array(syn.MATRIX_PA66, dtype=np.float64)
M1 = np.array([1.0, 1, 1, 0, 0, 0])
SQ32 = np.sqrt(1.5)


def row_with(**kw):
    r = ROW.copy()
    idx = dict(E=1, nu=2, alpha=3, theta0=4, sy0=5, k=6, n=7, m=8, eta0=9, beta1=10, beta2=11,
               theta_ref=12, C1=13, C2=14)
    for key, v in kw.items():
        if key == "Ei":
            r[16:28] = v
        elif key == "taui":
            r[28:40] = v
        else:
            r[idx[key]] = v
    return r


def iso_C(E, nu):
    K, G = E / (3 * (1 - 2 * nu)), E / (2 * (1 + nu))
    P1 = np.outer(M1, M1) / 3.0
    return 3 * K * P1 + 2 * G * (np.eye(6) - P1)


def zn_random(rng, scale=2e-3, p=0.01):
    z = np.zeros(79)
    ep = rng.normal(0, scale, 6)
    ep[:3] -= ep[:3].mean()  # viscoplastic strain is deviatoric
    z[:6], z[6] = ep, p
    z[7:] = rng.normal(0, scale, 72)
    return z


STATES = [  # (eps, theta, zn seed, trn, dt)
    (np.array([0.02, -0.008, -0.008, 0.001, 0.0, 0.002]), 300.0, None, 0.0, 0.005),
    (np.array([0.004, 0.001, -0.002, 0.0005, -0.001, 0.0]), 310.0, 1, 0.002, 0.01),
    (np.array([-0.03, 0.012, 0.011, 0.0, 0.004, -0.003]), 330.0, 2, -0.004, 1.0),
    (np.array([1e-4, 0.0, 0.0, 0.0, 0.0, 0.0]), 293.15, None, 0.0, 0.1),  # elastic
]


def leaf_state(i):
    eps, th, seed, trn, dt = STATES[i]
    zn = None if seed is None else zn_random(np.random.default_rng(seed))
    return eps, th, zn, trn, dt


@pytest.mark.parametrize("i", range(len(STATES)))
def test_complex_step_derivatives_match_finite_differences(i):
    eps, th, zn, trn, dt = leaf_state(i)
    o = oracle.leaf(ROW, eps, th, zn, trn, dt)
    h = 1e-8
    for j in range(6):
        e1, e2 = eps.copy(), eps.copy()
        e1[j] += h
        e2[j] -= h
        a, b = oracle.leaf(ROW, e1, th, zn, trn, dt), oracle.leaf(ROW, e2, th, zn, trn, dt)
        np.testing.assert_allclose(o["C"][:, j], (a["sig"] - b["sig"]) / (2 * h), rtol=0,
                                   atol=1e-6 * np.abs(o["C"]).max())
        assert abs(o["d"][j] - (a["D"] - b["D"]) / (2 * h)) <= 1e-6 * max(np.abs(o["d"]).max(), 1.0)
    ht = 1e-5
    a, b = oracle.leaf(ROW, eps, th + ht, zn, trn, dt), oracle.leaf(ROW, eps, th - ht, zn, trn, dt)
    np.testing.assert_allclose(o["tau"], (a["sig"] - b["sig"]) / (2 * ht), rtol=0,
                               atol=1e-6 * max(np.abs(o["tau"]).max(), 1e-3))
    assert abs(o["g"] - (a["D"] - b["D"]) / (2 * ht)) <= 1e-6 * max(abs(o["g"]), 1e-3)


@pytest.mark.parametrize("limit", ["frozen", "relaxed"])
def test_branch_limits_are_linear_thermoelastic(limit):
    tau = 1e30 if limit == "frozen" else 1e-30
    r = row_with(sy0=1e9, taui=np.full(12, tau))
    E = ROW[1] + (ROW[16:28].sum() if limit == "frozen" else 0.0)
    rng = np.random.default_rng(3)
    eps, th = rng.normal(0, 2e-3, 6), 320.0
    o = oracle.leaf(r, eps, th, None, 0.0, 0.01)
    ref = iso_C(E, ROW[2]) @ (eps - ROW[3] * (th - ROW[4]) * M1)
    np.testing.assert_allclose(o["sig"], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(o["C"], iso_C(E, ROW[2]), rtol=1e-10, atol=1e-9)
    assert o["znew"][6] == 0.0


def test_single_maxwell_branch_relaxation():
    """Held strain, one branch (E_1 = 300, tau_1 = 0.2 s), theta = theta_ref
    (a = 1), no long-term stiffness worth speaking of, no plasticity."""
    E1, tau1, nu = 300.0, 0.2, ROW[2]
    Ei = np.zeros(12)
    Ei[0] = E1
    r = row_with(E=1e-9, sy0=1e9, alpha=0.0, Ei=Ei, taui=np.full(12, tau1), theta_ref=300.0)
    K1, G1 = E1 / (3 * (1 - 2 * nu)), E1 / (2 * (1 + nu))
    tauK, tauG = tau1 * E1 / K1, tau1 * E1 / G1
    e = np.array([1e-3, 1e-3, 1e-3, 0, 0, 0]) + np.array([0, 0, 0, 2e-3, 0, 0])
    for dt, nsteps in ((0.01, 40), (1e-4, 4000)):
        z = np.zeros(79)
        for k in range(1, nsteps + 1):
            o = oracle.leaf(r, e, 300.0, z, e[:3].sum(), dt)
            z = o["znew"]
        rK, rG = 1 / (1 + dt / tauK), 1 / (1 + dt / tauG)
        # minus the (negligible) long-term branch
        mean_sig = o["sig"][:3].mean() - 1e-9 / (1 - 2 * nu) * 1e-3
        o["sig"][3] -= 1e-9 / (1 + nu) * 2e-3
        if dt == 0.01:  # the implicit Euler recursion, exactly
            assert abs(mean_sig - 3 * K1 * 1e-3 * rK ** nsteps) <= 1e-12 * 3 * K1 * 1e-3
            assert abs(o["sig"][3] - 2 * G1 * 2e-3 * rG ** nsteps) <= 1e-12 * 2 * G1 * 2e-3
        else:  # the ODE's exponential relaxation, to O(dt)
            t = dt * nsteps
            assert abs(mean_sig / (3 * K1 * 1e-3) - np.exp(-t / tauK)) < 1e-3
            assert abs(o["sig"][3] / (2 * G1 * 2e-3) - np.exp(-t / tauG)) < 1e-3


def test_thermorheological_simplicity():
    th = 330.0
    x = th - ROW[12]
    a = 10.0 ** (-ROW[13] * x / (ROW[14] + x))
    base = dict(sy0=1e9, alpha=0.0, beta1=0.0)
    r_hot = row_with(**base)
    r_ref = row_with(**base, taui=ROW[28:40] * a)
    rng = np.random.default_rng(4)
    eps, z = rng.normal(0, 2e-3, 6), zn_random(rng, p=0.0)
    z[:7] = 0.0
    o1 = oracle.leaf(r_hot, eps, th, z, 0.0, 0.05)
    o2 = oracle.leaf(r_ref, eps, ROW[12], z, 0.0, 0.05)
    np.testing.assert_allclose(o1["sig"], o2["sig"], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(o1["znew"], o2["znew"], rtol=1e-12, atol=1e-16)


def psi_mech(r, eps, th, z):
    """eq. (PA66 psi): long-term branch, hardening energy, Maxwell branches."""
    E, nu, al, th0, k, n = r[1], r[2], r[3], r[4], r[6], r[7]
    G1 = np.exp(-r[10] * (th - r[12]))
    evp, p = z[:6], z[6]
    e = eps - evp
    psi = 0.5 * e @ iso_C(E, nu) @ e - e @ iso_C(E, nu) @ (al * (th - th0) * M1)
    psi += G1 * k * p ** (n + 1) / (n + 1)
    for i in range(12):
        Ci = iso_C(r[16 + i], nu)
        ei = e - z[7 + 6 * i:13 + 6 * i]
        psi += 0.5 * ei @ Ci @ ei - ei @ Ci @ (al * (th - th0) * M1)
    return psi


@pytest.mark.parametrize("i", [0, 1, 2])
def test_coupling_term_from_the_free_energy(i):
    """D - Diss = theta psi_{theta eps} : (eps - eps^n)/dt + theta psi_{theta z} . (z - z^n)/dt
    with the mixed derivatives of psi by central differences at (eps, theta, z^{n+1})."""
    eps, th, zn, trn, dt = leaf_state(i)
    zn = np.zeros(79) if zn is None else zn
    # a strain at t^n with the given trace
    eps_n = np.zeros(6)
    eps_n[:3] = trn / 3.0
    o = oracle.leaf(ROW, eps, th, zn, trn, dt)
    z1 = o["znew"]
    ht, he = 1e-3, 1e-6

    def psi_th(e, z):
        return (psi_mech(ROW, e, th + ht, z) - psi_mech(ROW, e, th - ht, z)) / (2 * ht)
    # directional derivatives along the increments
    de, dz = eps - eps_n, z1 - zn
    s = he / max(np.abs(de).max(), 1e-12)
    term_e = (psi_th(eps + s * de, z1) - psi_th(eps - s * de, z1)) / (2 * s)
    s2 = he / max(np.abs(dz).max(), 1e-12)
    zp, zm = z1 + s2 * dz, z1 - s2 * dz
    term_z = (psi_th(eps, zp) - psi_th(eps, zm)) / (2 * s2)
    entropy = th * (term_e + term_z) / dt
    assert abs((o["D"] - o["diss"]) - entropy) <= 1e-5 * max(abs(entropy), 1.0)


@pytest.mark.parametrize("i", [0, 2])
def test_viscoplastic_step_consistency_and_normality(i):
    eps, th, zn, trn, dt = leaf_state(i)
    zn = np.zeros(79) if zn is None else zn
    o = oracle.leaf(ROW, eps, th, zn, trn, dt)
    dp = o["znew"][6] - zn[6]
    assert dp > 0
    x = th - ROW[12]
    G1, G2 = np.exp(-ROW[10] * x), np.exp(-ROW[11] * x)
    sy, eta = G1 * ROW[5], G2 * ROW[9]
    H = G1 * ROW[6] * o["znew"][6] ** ROW[7]
    s = o["sig"] - o["sig"][:3].mean() * M1
    q = SQ32 * np.linalg.norm(s)
    phi = (q - sy - H) / sy
    assert abs(dp - dt * (sy / eta) * phi ** ROW[8]) <= 1e-10 * dp
    devp = o["znew"][:6] - zn[:6]
    np.testing.assert_allclose(devp, SQ32 * dp * s / np.linalg.norm(s), rtol=0, atol=1e-12 * dp)
    assert o["diss"] >= 0.0


def test_rate_independent_limit():
    r = row_with(eta0=1e-9)
    eps, th, zn, trn, dt = leaf_state(0)
    o = oracle.leaf(r, eps, th, None, trn, dt)
    x = th - ROW[12]
    G1 = np.exp(-ROW[10] * x)
    s = o["sig"] - o["sig"][:3].mean() * M1
    q = SQ32 * np.linalg.norm(s)
    yld = G1 * ROW[5] + G1 * ROW[6] * o["znew"][6] ** ROW[7]
    assert abs(q - yld) <= 1e-4 * yld


def test_homogeneous_pa66_tree_is_the_leaf():
    K = 3
    w, n, ph = syn.tree(K)
    mats = syn.materials_pa66()
    t = oracle.Tree(K, w, n, np.ones_like(ph), mats)
    assert t.state_words == 8 + 3 * 7 + 8 * 79 + 1
    eps, th, _, _, dt = leaf_state(0)
    s0 = t.init_state(1, syn.THETA_START)
    so, out, st, it = oracle.eval_batch(t, eps[None], [th], dt, s0)
    assert st[0] == 0
    o = oracle.leaf(mats[1], eps, th, None, 0.0, dt)
    np.testing.assert_allclose(out[0, :6], o["sig"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out[0, 48], o["D"], rtol=1e-12)
    np.testing.assert_allclose(so[0, 8 + 21:8 + 21 + 79], o["znew"], rtol=1e-12, atol=1e-18)
