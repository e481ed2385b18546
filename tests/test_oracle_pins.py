"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formulas: each check compares the
oracle with an independent characterisation (closed-form laminate of the
paper's eq. (laminate) with the projector P(n), Levin's exact two-phase
relation, finite differences, thermodynamic derivation from the free energy,
the kinematic meaning of the jump vectors, invariants of homogeneous and
free-expansion states, Hill-Mandel, and a second dense linear-algebra path).
"""
import numpy as np
import pytest

import oracle
from paper_2109_14403_gb300 import synthetic as syn

SQ2 = np.sqrt(2.0)
PAIRS = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
WM = np.array([1, 1, 1, SQ2, SQ2, SQ2])


# ---------------------------------------------------------------- helpers
def t4_to_mandel(T):
    M = np.zeros((6, 6))
    for I, (i, j) in enumerate(PAIRS):
        for J, (k, l) in enumerate(PAIRS):
            M[I, J] = WM[I] * WM[J] * T[i, j, k, l]
    return M


def t2_to_mandel(s):
    return np.array([WM[I] * s[i, j] for I, (i, j) in enumerate(PAIRS)])


def mandel_to_t2(v):
    s = np.zeros((3, 3))
    for I, (i, j) in enumerate(PAIRS):
        s[i, j] = s[j, i] = v[I] / WM[I]
    return s


def iso_stiffness_tensor(E, nu):
    """Sec. 4: C = 3K P1 + 2G P2 with the projectors written in index form."""
    K = E / (3 * (1 - 2 * nu))
    G = E / (2 * (1 + nu))
    d = np.eye(3)
    P1 = np.einsum("mn,op->mnop", d, d) / 3
    P2 = 0.5 * (np.einsum("mo,pn->mnop", d, d) + np.einsum("mp,on->mnop", d, d)) - P1
    return t4_to_mandel(3 * K * P1 + 2 * G * P2), K


def projector_P(n):
    """Eq. (P(n)) in Cartesian components."""
    d = np.eye(3)
    P = 0.5 * (np.einsum("m,no,p->mnop", n, d, n) + np.einsum("n,mo,p->mnop", n, d, n)
               + np.einsum("m,np,o->mnop", n, d, n) + np.einsum("n,mp,o->mnop", n, d, n)) \
        - np.einsum("m,n,o,p->mnop", n, n, n, n)
    return t4_to_mandel(P)


def milton_laminate(C1, C2, n, c1, lam):
    """Solve eq. (laminate) for the effective stiffness of one laminate."""
    P = projector_P(n)
    I6 = np.eye(6)
    Y = lambda C: np.linalg.inv(P + lam * np.linalg.inv(C - lam * I6))
    Yb = c1 * Y(C1) + (1 - c1) * Y(C2)
    return lam * I6 + lam * np.linalg.inv(np.linalg.inv(Yb) - P)


def dmn_linear(K, w, normals, Cphase):
    """DMN^L: stiffness propagation from the leaves to the root (eq. DMN^L)."""
    lam = 2 * max(np.linalg.eigvalsh(C).max() for C in Cphase)
    Cl = list(Cphase)          # level K+1
    wl = list(w)
    for k in range(K, 0, -1):
        Cn, wn = [], []
        for i in range(1, 2 ** (k - 1) + 1):
            a, b = 2 * i - 2, 2 * i - 1
            p = 2 ** K - 2 ** k + i - 1
            c1 = wl[a] / (wl[a] + wl[b])
            Cn.append(milton_laminate(Cl[a], Cl[b], normals[p], c1, lam))
            wn.append(wl[a] + wl[b])
        Cl, wl = Cn, wn
    return Cl[0]


def elastic_mats(alpha_equal=None):
    m = syn.materials().copy()
    m[1, 5] = 1e12  # yield never reached: linear thermoelastic matrix
    if alpha_equal is not None:
        m[:, 3] = alpha_equal
    return m


def make_tree(K, mats, seed=None, phase=None):
    w, n, ph = syn.tree(K, seed)
    if phase is not None:
        ph = phase
    return oracle.Tree(K, w, n, ph, mats), w, n


# ---------------------------------------------------------------- kinematics
@pytest.mark.parametrize("K", [1, 3, 5])
def test_kinematics_mean_strain_and_jump(K, mats):
    """Every node's weighted mean strain equals its parent's (so the leaf mean is
    eps_bar) and the jump across node p is sym(a_p (x) n_p)."""
    t, w, n = make_tree(K, mats)
    rng = np.random.default_rng(3)
    eb = rng.normal(size=6)
    a = rng.normal(size=3 * t.nnode)
    eps = oracle.leaf_strains(t, eb, a)
    np.testing.assert_allclose(w @ eps, eb, rtol=0, atol=1e-13)
    for k in range(1, K + 1):
        span = 2 ** (K + 1 - k)
        for i in range(1, 2 ** (k - 1) + 1):
            p = 2 ** K - 2 ** k + i - 1
            lo = (i - 1) * span
            L = slice(lo, lo + span // 2)
            R = slice(lo + span // 2, lo + span)
            mL = w[L] @ eps[L] / w[L].sum()
            mR = w[R] @ eps[R] / w[R].sum()
            ap = a[3 * p:3 * p + 3]
            jump = t2_to_mandel(0.5 * (np.outer(ap, n[p]) + np.outer(n[p], ap)))
            np.testing.assert_allclose(mL - mR, jump, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- phase laws
def test_thermoelastic_law_matches_paper_form(mats):
    C, _ = iso_stiffness_tensor(72000.0, 0.22)
    rng = np.random.default_rng(0)
    eps = rng.normal(0, 1e-3, 6)
    th = 330.0
    r = oracle.leaf(mats[0], eps, th)
    m = np.array([1, 1, 1, 0, 0, 0.0])
    np.testing.assert_allclose(r["sig"], C @ (eps - 5e-6 * (th - 293) * m), rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(r["C"], C, rtol=1e-13, atol=1e-9)
    assert r["diss"] == 0.0


def _plastic_case():
    rng = np.random.default_rng(11)
    eps = rng.normal(0, 2e-2, 6)
    zn = np.zeros(7)
    ep0 = rng.normal(0, 5e-4, 6)
    ep0[:3] -= ep0[:3].mean()            # plastic strain is deviatoric
    zn[:6] = ep0
    zn[6] = 0.01
    return eps, zn


def test_j2_return_mapping_characterisation(mats):
    """Closed-form radial return is the unique state that (i) satisfies the
    elastic law with the new plastic strain, (ii) sits on the hardened yield
    surface, (iii) has a plastic increment normal to the deviatoric stress with
    |d eps_p| = sqrt(3/2) dp."""
    eps, zn = _plastic_case()
    th = 320.0
    r = oracle.leaf(mats[1], eps, th, zn)
    C, _ = iso_stiffness_tensor(2500.0, 0.38)
    m = np.array([1, 1, 1, 0, 0, 0.0])
    ep, p = r["znew"][:6], r["znew"][6]
    dp = p - zn[6]
    assert dp > 0
    np.testing.assert_allclose(r["sig"], C @ (eps - ep - 8e-5 * (th - 293) * m), rtol=1e-12,
                               atol=1e-10)
    s = mandel_to_t2(r["sig"])
    sdev = s - np.trace(s) / 3 * np.eye(3)
    qeq = np.sqrt(1.5 * np.sum(sdev * sdev))
    sy = 50.0 - 0.3 * (th - 293)
    assert qeq == pytest.approx(sy + 300.0 * p, rel=1e-12)
    dep = mandel_to_t2(ep - zn[:6])
    np.testing.assert_allclose(dep, 1.5 * dp * sdev / qeq, rtol=0, atol=1e-14)
    assert abs(np.trace(dep)) < 1e-15


def test_j2_elastic_step_keeps_state(mats):
    zn = np.zeros(7)
    zn[6] = 0.02
    r = oracle.leaf(mats[1], np.full(6, 1e-5), 300.0, zn)
    np.testing.assert_array_equal(r["znew"], zn)
    assert r["diss"] == 0.0


@pytest.mark.parametrize("which", ["fiber", "matrix"])
def test_leaf_derivatives_finite_difference(which, mats):
    eps, zn = _plastic_case()
    row = mats[0] if which == "fiber" else mats[1]
    th, trn, dt = 320.0, 1e-3, 0.5
    r = oracle.leaf(row, eps, th, zn, trn, dt)
    h = 1e-8
    for c in range(6):
        e1, e2 = eps.copy(), eps.copy()
        e1[c] += h
        e2[c] -= h
        a, b = oracle.leaf(row, e1, th, zn, trn, dt), oracle.leaf(row, e2, th, zn, trn, dt)
        np.testing.assert_allclose((a["sig"] - b["sig"]) / (2 * h), r["C"][:, c], rtol=1e-6,
                                   atol=1e-6 * np.abs(r["C"]).max())
        assert (a["D"] - b["D"]) / (2 * h) == pytest.approx(r["d"][c], rel=1e-6, abs=1e-6)
    ht = 1e-4
    a, b = oracle.leaf(row, eps, th + ht, zn, trn, dt), oracle.leaf(row, eps, th - ht, zn, trn, dt)
    np.testing.assert_allclose((a["sig"] - b["sig"]) / (2 * ht), r["tau"], rtol=1e-6, atol=1e-8)
    assert (a["D"] - b["D"]) / (2 * ht) == pytest.approx(r["g"], rel=1e-6, abs=1e-9)


def test_coupling_term_from_free_energy(mats):
    """D = theta psi_{,theta eps} : eps_dot + theta psi_{,theta z} . z_dot - psi_{,z} . z_dot
    (Sec. 2 coupling term, Sec. 4) with the partials of the free energy
    psi = 1/2 (eps-ep):C(eps-ep) - (eps-ep):C[alpha(theta-theta0)] + H p^2/2 taken
    by finite differences; Diss = -psi_{,z} . z_dot."""
    eps, zn = _plastic_case()
    th, dt = 320.0, 0.5
    epsn = eps - np.random.default_rng(5).normal(0, 1e-3, 6)
    trn = epsn[:3].sum()
    r = oracle.leaf(mats[1], eps, th, zn, trn, dt)
    C, _ = iso_stiffness_tensor(2500.0, 0.38)
    m = np.array([1, 1, 1, 0, 0, 0.0])
    Hh, al = 300.0, 8e-5

    def psi(e, T, z):
        ee = e - z[:6]
        return 0.5 * ee @ C @ ee - ee @ C @ (al * (T - 293.0) * m) + 0.5 * Hh * z[6] ** 2

    z1 = r["znew"]
    hz, hT = 1e-6, 1e-3

    def dpsi_dz(T):
        g = np.zeros(7)
        for c in range(7):
            zp, zm = z1.copy(), z1.copy()
            zp[c] += hz
            zm[c] -= hz
            g[c] = (psi(eps, T, zp) - psi(eps, T, zm)) / (2 * hz)
        return g

    def dpsi_de(T):
        g = np.zeros(6)
        for c in range(6):
            ep_, em_ = eps.copy(), eps.copy()
            ep_[c] += hz
            em_[c] -= hz
            g[c] = (psi(ep_, T, z1) - psi(em_, T, z1)) / (2 * hz)
        return g

    d2_te = (dpsi_de(th + hT) - dpsi_de(th - hT)) / (2 * hT)
    d2_tz = (dpsi_dz(th + hT) - dpsi_dz(th - hT)) / (2 * hT)
    zdot = (z1 - zn) / dt
    edot = (eps - epsn) / dt
    D = th * d2_te @ edot + th * d2_tz @ zdot - dpsi_dz(th) @ zdot
    diss = -dpsi_dz(th) @ zdot
    assert r["D"] == pytest.approx(D, rel=1e-6)
    assert r["diss"] == pytest.approx(diss, rel=1e-6)
    assert r["diss"] > 0


# ---------------------------------------------------------------- laminates
def test_k1_equals_milton_laminate():
    m = elastic_mats()
    t, w, n = make_tree(1, m)
    s = t.init_state(1, 293.0)
    _, out, st, _ = oracle.eval_batch(t, np.full((1, 6), 1e-4), [293.0], 1.0, s)
    assert st[0] == 0
    C1, _ = iso_stiffness_tensor(72000.0, 0.22)
    C2, _ = iso_stiffness_tensor(2500.0, 0.38)
    lam = 2 * max(np.linalg.eigvalsh(C1).max(), np.linalg.eigvalsh(C2).max())
    Cm = milton_laminate(C1, C2, n[0], w[0], lam)
    np.testing.assert_allclose(oracle.split_out(out[0])["C"], Cm, rtol=1e-11, atol=1e-8)


@pytest.mark.parametrize("K", [2, 4, 6])
def test_linear_dmn_equals_stiffness_propagation(K):
    m = elastic_mats()
    t, w, n = make_tree(K, m)
    s = t.init_state(1, 293.0)
    _, out, st, _ = oracle.eval_batch(t, np.full((1, 6), 1e-4), [300.0], 1.0, s)
    assert st[0] == 0
    C1, _ = iso_stiffness_tensor(72000.0, 0.22)
    C2, _ = iso_stiffness_tensor(2500.0, 0.38)
    Cl = [C1 if j % 2 == 0 else C2 for j in range(2 ** K)]
    ref = dmn_linear(K, w, n, Cl)
    np.testing.assert_allclose(oracle.split_out(out[0])["C"], ref, rtol=1e-10,
                               atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("K", [1, 3, 5])
def test_levin_thermal_stress(K):
    """Two-phase linear thermoelastic composite: the effective thermal stress
    coefficient obeys Levin's exact relation
    beta_bar = beta1 + (C_bar - C1)(C2 - C1)^{-1}(beta2 - beta1)."""
    m = elastic_mats()
    t, w, n = make_tree(K, m)
    s = t.init_state(1, 293.0)
    _, out, st, _ = oracle.eval_batch(t, np.zeros((1, 6)), [310.0], 1.0, s)
    o = oracle.split_out(out[0])
    C1, K1 = iso_stiffness_tensor(72000.0, 0.22)
    C2, K2 = iso_stiffness_tensor(2500.0, 0.38)
    mm = np.array([1, 1, 1, 0, 0, 0.0])
    b1, b2 = 3 * K1 * 5e-6 * mm, 3 * K2 * 8e-5 * mm
    beta = b1 + (o["C"] - C1) @ np.linalg.solve(C2 - C1, b2 - b1)
    np.testing.assert_allclose(-o["C_theta"], beta, rtol=1e-9, atol=1e-9 * np.abs(beta).max())
    # same statement for the stress itself at eps_bar = 0
    np.testing.assert_allclose(o["sig"], -beta * (310.0 - 293.0), rtol=1e-9, atol=1e-8)


# ---------------------------------------------------------------- invariants
def test_homogeneous_phases_give_phase_response(mats):
    K = 4
    t, w, n = make_tree(K, mats, phase=np.ones(2 ** K, np.uint8))
    s = t.init_state(1, 293.0)
    eps, zn = _plastic_case()
    sout, out, st, _ = oracle.eval_batch(t, eps[None], [320.0], 1.0, s)
    o = oracle.split_out(out[0])
    r = oracle.leaf(mats[1], eps, 320.0, np.zeros(7), 0.0, 1.0)
    assert np.abs(sout[0, 8:8 + 3 * t.nnode]).max() < 1e-12
    np.testing.assert_allclose(o["sig"], r["sig"], rtol=1e-11, atol=1e-9)
    np.testing.assert_allclose(o["C"], r["C"], rtol=1e-9, atol=1e-7)
    np.testing.assert_allclose(o["C_theta"], r["tau"], rtol=1e-9, atol=1e-9)
    assert o["D"] == pytest.approx(r["D"], rel=1e-10)
    assert o["diss"] == pytest.approx(r["diss"], rel=1e-10)
    np.testing.assert_allclose(o["D_eps"], r["d"], rtol=1e-9, atol=1e-9)


def test_free_thermal_expansion_is_stress_free(mats):
    m = syn.materials().copy()
    m[:, 3] = 8e-5
    K = 5
    t, w, n = make_tree(K, m)
    s = t.init_state(1, 293.0)
    th = 340.0
    deps = 8e-5 * (th - 293.0) * np.array([[1, 1, 1, 0, 0, 0.0]])
    sout, out, st, _ = oracle.eval_batch(t, deps, [th], 1.0, s)
    o = oracle.split_out(out[0])
    assert np.abs(o["sig"]).max() < 1e-9
    assert o["diss"] == 0.0


def test_hill_mandel_and_equilibrium(mats):
    K = 4
    t, w, n = make_tree(K, mats)
    s = t.init_state(1, 293.0)
    eps, _ = _plastic_case()
    sout, out, st, _ = oracle.eval_batch(t, eps[None], [320.0], 1.0, s)
    assert st[0] == 0
    o = oracle.split_out(out[0])
    eb = sout[0, :6]
    a = sout[0, 8:8 + 3 * t.nnode]
    le = oracle.leaf_strains(t, eb, a)
    sig = np.zeros((2 ** K, 6))
    zo = 8 + 3 * t.nnode
    for j in range(2 ** K):
        if j % 2 == 1:
            sig[j] = oracle.leaf(mats[1], le[j], 320.0, s[0, zo:zo + 7])["sig"]
            zo += 7
        else:
            sig[j] = oracle.leaf(mats[0], le[j], 320.0)["sig"]
    np.testing.assert_allclose(w @ sig, o["sig"], rtol=1e-12, atol=1e-10)
    rng = np.random.default_rng(1)
    sn = np.linalg.norm(o["sig"])
    for _ in range(5):
        da = rng.normal(size=3 * t.nnode)
        deb = rng.normal(size=6)
        de = oracle.leaf_strains(t, deb, da)
        lhs = np.sum(w[:, None] * sig * de)
        assert lhs == pytest.approx(o["sig"] @ deb, abs=1e-9 * sn * np.abs(de).max())


def test_gough_joule_sign():
    m = elastic_mats()
    t, w, n = make_tree(3, m)
    s = t.init_state(2, 293.0)
    mm = np.array([1, 1, 1, 0, 0, 0.0])
    _, out, st, _ = oracle.eval_batch(t, np.stack([1e-4 * mm, -1e-4 * mm]), [293.0, 293.0], 1.0, s)
    D = oracle.split_out(out)["D"]
    assert D[0] < 0 < D[1]


def test_dissipation_nonnegative(mats):
    t, w, n = make_tree(4, mats)
    deps, th = syn.ramp_k4(n_points=16, n_incr=8)
    s = t.init_state(16, 293.0)
    for k in range(8):
        s, out, st, _ = oracle.eval_batch(t, deps[k], th[k], 1.0, s)
        assert (st == 0).all()
        assert (oracle.split_out(out)["diss"] >= 0).all()


# ---------------------------------------------------------------- tangents (FD)
@pytest.mark.parametrize("K", [2, 3])
def test_effective_tangents_finite_difference(K, mats):
    t, w, n = make_tree(K, mats)
    s = t.init_state(1, 293.0)
    # one plastic increment so the state is non-trivial, then a probe increment
    s, _, _, _ = oracle.eval_batch(t, np.array([[4e-3, -1e-3, -1e-3, 1e-3, 0, 5e-4]]), [305.0], 1.0,
                                   s, tol=1e-14)
    deps = np.array([[2e-3, 5e-4, -1e-3, 2e-4, -3e-4, 1e-3]])
    th = 312.0
    kw = dict(tol=1e-14, dt=0.5) if False else dict(tol=1e-14)
    _, out, st, _ = oracle.eval_batch(t, deps, [th], 0.5, s, **kw)
    o = oracle.split_out(out[0])
    assert o["diss"] > 0
    h = 1e-7
    for c in range(6):
        dp, dm = deps.copy(), deps.copy()
        dp[0, c] += h
        dm[0, c] -= h
        op = oracle.split_out(oracle.eval_batch(t, dp, [th], 0.5, s, **kw)[1][0])
        om = oracle.split_out(oracle.eval_batch(t, dm, [th], 0.5, s, **kw)[1][0])
        np.testing.assert_allclose((op["sig"] - om["sig"]) / (2 * h), o["C"][:, c], rtol=1e-5,
                                   atol=1e-5 * np.abs(o["C"]).max())
        assert (op["D"] - om["D"]) / (2 * h) == pytest.approx(o["D_eps"][c], rel=1e-5,
                                                              abs=1e-5 * np.abs(o["D_eps"]).max())
    ht = 1e-4
    op = oracle.split_out(oracle.eval_batch(t, deps, [th + ht], 0.5, s, **kw)[1][0])
    om = oracle.split_out(oracle.eval_batch(t, deps, [th - ht], 0.5, s, **kw)[1][0])
    np.testing.assert_allclose((op["sig"] - om["sig"]) / (2 * ht), o["C_theta"], rtol=1e-5,
                               atol=1e-5 * np.abs(o["C_theta"]).max())
    assert (op["D"] - om["D"]) / (2 * ht) == pytest.approx(o["D_theta"], rel=1e-5)


# ---------------------------------------------------------------- linear algebra / Newton
@pytest.mark.parametrize("K", [2, 4, 6])
def test_dense_and_sparse_paths_agree(K, mats):
    t, w, n = make_tree(K, mats)
    deps, th = syn.single_increment(6, scale=3e-3)
    s = t.init_state(6, 293.0)
    so1, o1, st1, it1 = oracle.eval_batch(t, deps, th, 1.0, s)
    so2, o2, st2, it2 = oracle.eval_batch(t, deps, th, 1.0, s, dense=True)
    np.testing.assert_array_equal(st1, st2)
    np.testing.assert_allclose(o1, o2, rtol=1e-11, atol=1e-11 * np.abs(o1).max())
    np.testing.assert_allclose(so1, so2, rtol=1e-10, atol=1e-14)


def test_newton_is_exact_for_linear_phases():
    m = elastic_mats()
    t, w, n = make_tree(5, m)
    s = t.init_state(1, 293.0)
    *_, st, it, hist = oracle.eval_point_trace(t, np.array([1e-3, 0, 0, 2e-4, 0, 0]), 320.0, 1.0,
                                               s[0])
    assert st == 0 and it == 1
    assert hist[1] < 1e-14


def test_newton_residual_decreases_and_converges_superlinearly(mats):
    t, w, n = make_tree(6, mats)
    s = t.init_state(1, 293.0)
    *_, st, it, hist = oracle.eval_point_trace(t, np.array([4e-3, -2e-3, 1e-3, 1e-3, -5e-4, 2e-3]),
                                               330.0, 1.0, s[0], tol=1e-13)
    assert st == 0
    assert np.all(np.diff(hist) < 0)
    assert hist[-1] / hist[-2] < 1e-2


def _path_case(law):
    """(K, materials, deps[n_incr, n, 6], theta[n_incr, n], dt, internal words)."""
    if law == "j2":      # the K = 4 configuration's ramp on the K = 8 tree
        deps, theta = syn.ramp_k4(n_points=2, n_incr=6, seed=5)
        return 8, syn.materials(), deps, theta, 1.0, 7
    if law == "perzyna":  # the large configuration: K = 9, strain rates N(0, 1e-2)/s
        deps, theta = syn.large_path(n_points=2, n_incr=4, seed=5)
        return 9, syn.materials_viscoplastic(), 10.0 * deps, theta, syn.LARGE_DT, 13
    deps, theta = syn.ramp_k4(n_points=2, n_incr=6, seed=5)   # PA66 matrix
    return 4, syn.materials_pa66(), 3.0 * deps, theta, 0.05, 79


@pytest.mark.parametrize("law", ["j2", "perzyna", "pa66"])
def test_plastic_path_by_composition(law):
    """A full inelastic load path, pinned increment by increment through parts
    that are pinned on their own: every leaf strain from the kinematic
    operator, every leaf response from the leaf law (characterised by the leaf
    pins), and the oracle's converged jumps checked for equilibrium (virtual
    work of the leaf stresses vanishes for every admissible jump variation).
    The stored internal variables, the macro stress, coupling term and
    dissipation must then be those of the leaves; the tangent at the end of the
    path matches central differences of the whole solve."""
    K, mats, deps, theta, dt, nz = _path_case(law)
    t, w, n = make_tree(K, mats)
    N = t.nnode
    nP, n_incr = deps.shape[1], deps.shape[0]
    s = t.init_state(nP, syn.THETA_START)
    rng = np.random.default_rng(8)
    plastic_seen = 0
    for k in range(n_incr):
        sout, out, st, _ = oracle.eval_batch(t, deps[k], theta[k], dt, s, tol=1e-13)
        assert np.all(st == 0)
        for q in range(nP):
            o = oracle.split_out(out[q])
            np.testing.assert_allclose(sout[q, :6], s[q, :6] + deps[k, q], rtol=0, atol=1e-15)
            assert sout[q, 6] == theta[k, q]
            le = oracle.leaf_strains(t, sout[q, :6], sout[q, 8:8 + 3 * N])
            le_old = oracle.leaf_strains(t, s[q, :6], s[q, 8:8 + 3 * N])
            sig = np.zeros((1 << K, 6))
            D = np.zeros(1 << K)
            diss = np.zeros(1 << K)
            zo = 8 + 3 * N
            for j in range(1 << K):
                trn = le_old[j, :3].sum()
                if t.phase[j] == 1:
                    r = oracle.leaf(mats[1], le[j], theta[k, q], s[q, zo:zo + nz], trn, dt)
                    np.testing.assert_allclose(sout[q, zo:zo + nz], r["znew"][:nz], rtol=1e-11,
                                               atol=1e-15)
                    plastic_seen += int(r["znew"][6] > s[q, zo + 6])
                    zo += nz
                else:
                    r = oracle.leaf(mats[0], le[j], theta[k, q], None, trn, dt)
                sig[j], D[j], diss[j] = r["sig"], r["D"], r["diss"]
            sn = np.linalg.norm(o["sig"])
            np.testing.assert_allclose(w @ sig, o["sig"], rtol=0, atol=1e-11 * sn)
            assert w @ D == pytest.approx(o["D"], rel=1e-10, abs=1e-12)
            assert w @ diss == pytest.approx(o["diss"], rel=1e-10, abs=1e-14)
            for _ in range(3):   # equilibrium: admissible variations at fixed macro strain
                de = oracle.leaf_strains(t, np.zeros(6), rng.normal(size=3 * N))
                assert abs(np.sum(w[:, None] * sig * de)) < 1e-10 * sn * np.abs(de).max()
        s = sout
    assert plastic_seen > 0
    # consistent tangent at the last state against central differences of the solve
    d1 = deps[-1, :1]
    th = theta[-1, 0] + 1.0
    _, out, st, _ = oracle.eval_batch(t, d1, [th], dt, s[:1], tol=1e-14)
    assert st[0] == 0
    C = oracle.split_out(out[0])["C"]
    h = 1e-7
    for c in range(6):
        dp, dm = d1.copy(), d1.copy()
        dp[0, c] += h
        dm[0, c] -= h
        sp = oracle.eval_batch(t, dp, [th], dt, s[:1], tol=1e-14)[1][0, :6]
        sm = oracle.eval_batch(t, dm, [th], dt, s[:1], tol=1e-14)[1][0, :6]
        np.testing.assert_allclose((sp - sm) / (2 * h), C[:, c], rtol=1e-5, atol=1e-5 * np.abs(C).max())


# ---------------------------------------------------------------- Perzyna matrix
# kind 2: J2 viscoplasticity with the overstress rate law of Sec. 4 and
# temperature-dependent moduli E(theta) = E (1 + dE_dT (theta - theta0))
def _perzyna(m=5.0, t_visc=1e3, dE=-0.002, sy0=50.0):
    row = np.array(syn.MATRIX_PERZYNA, dtype=np.float64)
    row[5], row[8], row[9], row[10] = sy0, m, t_visc, dE
    return row


def _perzyna_case():
    eps, z7 = _plastic_case()
    zn = np.zeros(13)
    zn[:7] = z7
    zn[7:] = eps - np.random.default_rng(3).normal(0, 2e-3, 6)  # leaf strain at t^n
    return eps, zn


def _trial(row, eps, th, zn):
    """Independent elastic predictor: moduli at theta, q_trial, f_trial."""
    r = 1 + row[10] * (th - row[4])
    C, Kb = iso_stiffness_tensor(row[1] * r, row[2])
    G = row[1] * r / (2 * (1 + row[2]))
    m = np.array([1, 1, 1, 0, 0, 0.0])
    ee = eps - row[3] * (th - row[4]) * m - zn[:6]
    sig = C @ ee
    dev = sig - sig[:3].mean() * m
    q = np.sqrt(1.5) * np.linalg.norm(dev)
    sy = row[5] + row[6] * (th - row[4])
    return sig, q, q - sy - row[7] * zn[6], G, sy, C


@pytest.mark.parametrize("state", ["elastic", "viscoplastic"])
def test_perzyna_derivatives_finite_difference(state):
    """dsigma/deps, dsigma/dtheta, dD/deps and dD/dtheta of the Perzyna leaf
    against central differences of its stress and coupling term."""
    row = _perzyna(sy0=1e6 if state == "elastic" else 50.0, t_visc=2.0)
    eps, zn = _perzyna_case()
    th, dt = 320.0, 0.5
    r = oracle.leaf(row, eps, th, zn, 0.0, dt)
    assert (r["znew"][6] > zn[6]) == (state == "viscoplastic")
    h = 1e-8
    for c in range(6):
        e1, e2 = eps.copy(), eps.copy()
        e1[c] += h
        e2[c] -= h
        a, b = oracle.leaf(row, e1, th, zn, 0.0, dt), oracle.leaf(row, e2, th, zn, 0.0, dt)
        np.testing.assert_allclose((a["sig"] - b["sig"]) / (2 * h), r["C"][:, c], rtol=1e-6,
                                   atol=1e-6 * np.abs(r["C"]).max())
        assert (a["D"] - b["D"]) / (2 * h) == pytest.approx(r["d"][c], rel=1e-6, abs=1e-6)
    ht = 1e-4
    a, b = oracle.leaf(row, eps, th + ht, zn, 0.0, dt), oracle.leaf(row, eps, th - ht, zn, 0.0, dt)
    np.testing.assert_allclose((a["sig"] - b["sig"]) / (2 * ht), r["tau"], rtol=1e-6, atol=1e-8)
    assert (a["D"] - b["D"]) / (2 * ht) == pytest.approx(r["g"], rel=1e-6, abs=1e-9)


def test_perzyna_linear_rate_closed_form():
    """m = 1: the implicit Euler step dp = c phi(dp) is linear in dp, so
    dp = c f / (sigma_Y + c (3G + H)), c = dt / t_visc."""
    row = _perzyna(m=1.0, t_visc=3.0)
    eps, zn = _perzyna_case()
    th, dt = 330.0, 0.7
    _, q, f, G, sy, _ = _trial(row, eps, th, zn)
    assert f > 0
    c = dt / row[9]
    dp = c * f / (sy + c * (3 * G + row[7]))
    r = oracle.leaf(row, eps, th, zn, 0.0, dt)
    assert r["znew"][6] - zn[6] == pytest.approx(dp, rel=1e-12)
    # and the returned stress has the radial-return form with that dp
    sig_tr, *_ = _trial(row, eps, th, zn)
    m = np.array([1, 1, 1, 0, 0, 0.0])
    dev = sig_tr - sig_tr[:3].mean() * m
    np.testing.assert_allclose(r["sig"], sig_tr - 3 * G * dp / q * dev, rtol=1e-12, atol=1e-9)


def test_perzyna_limits():
    """Fast limit (t_visc -> 0): the rate-independent J2 leaf; slow limit
    (t_visc -> infinity): the elastic predictor.  Moduli held constant.  The
    overstress vanishes like (dt/t_visc)^(-1/m), so the fast limit is taken
    with m = 1 (relative gap sigma_Y / (c (3G + H)) ~ 4e-14)."""
    eps, zn = _perzyna_case()
    th, dt = 320.0, 0.5
    fast = oracle.leaf(_perzyna(m=1.0, t_visc=1e-12, dE=0.0), eps, th, zn, 0.0, dt)
    j2 = oracle.leaf(syn.MATRIX, eps, th, zn[:7], zn[7:10].sum(), dt)
    np.testing.assert_allclose(fast["sig"], j2["sig"], rtol=1e-7, atol=1e-6)
    np.testing.assert_allclose(fast["znew"][:7], j2["znew"], rtol=1e-7, atol=1e-10)
    np.testing.assert_allclose(fast["C"], j2["C"], rtol=1e-5, atol=1e-3)
    assert fast["D"] == pytest.approx(j2["D"], rel=1e-6)
    assert fast["diss"] == pytest.approx(j2["diss"], rel=1e-6)
    slow = oracle.leaf(_perzyna(t_visc=1e20, dE=0.0), eps, th, zn, 0.0, dt)
    sig_tr, *_ = _trial(_perzyna(dE=0.0), eps, th, zn)
    np.testing.assert_allclose(slow["sig"], sig_tr, rtol=1e-9, atol=1e-9)
    assert slow["diss"] < 1e-12


def test_perzyna_moduli_follow_temperature():
    """Below yield the Perzyna leaf is the thermoelastic law with the stiffness
    of E (1 + dE_dT (theta - theta0)) (Sec. 4 projector form, index notation)."""
    row = _perzyna(sy0=1e6, dE=-0.002)
    eps, zn = _perzyna_case()
    for th in (293.0, 350.0, 393.0):
        r = oracle.leaf(row, eps, th, zn, 0.0, 0.01)
        sig, *_ = _trial(row, eps, th, zn)
        np.testing.assert_allclose(r["sig"], sig, rtol=1e-12, atol=1e-10)
        C, _ = iso_stiffness_tensor(2500.0 * (1 - 0.002 * (th - 293.0)), 0.38)
        np.testing.assert_allclose(r["C"], C, rtol=1e-12, atol=1e-9)


def test_perzyna_coupling_term_from_free_energy():
    """The thermal part of D, theta psi_{,theta eps} : eps_dot + theta
    psi_{,theta z} . z_dot, taken by finite differences of the free energy
    psi = 1/2 (eps-ep):C(theta)(eps-ep) - (eps-ep):C(theta)[alpha (theta-theta0)]
    + H p^2/2 with C(theta) = r(theta) C; the remaining, dissipative part is the
    paper's sigma_Y p_dot (Sec. 4), equal to Diss."""
    row = _perzyna(t_visc=2.0, dE=-0.002)
    eps, zn = _perzyna_case()
    th, dt = 320.0, 0.5
    r = oracle.leaf(row, eps, th, zn, 0.0, dt)
    assert r["diss"] > 0
    m = np.array([1, 1, 1, 0, 0, 0.0])

    def psi(e, T, z):
        C, _ = iso_stiffness_tensor(2500.0 * (1 - 0.002 * (T - 293.0)), 0.38)
        ee = e - z[:6]
        return 0.5 * ee @ C @ ee - ee @ C @ (8e-5 * (T - 293.0) * m) + 0.5 * 300.0 * z[6] ** 2

    z1 = r["znew"][:7]
    # psi is quadratic in eps and z and its gradient quadratic in theta, so
    # central differences are exact up to rounding: take wide steps
    hz, hT = 1e-4, 1e-2

    def grad(T, wrt):
        g = np.zeros(6 if wrt == "e" else 7)
        for c in range(g.size):
            if wrt == "e":
                a_, b_ = eps.copy(), eps.copy()
                a_[c] += hz
                b_[c] -= hz
                g[c] = (psi(a_, T, z1) - psi(b_, T, z1)) / (2 * hz)
            else:
                a_, b_ = z1.copy(), z1.copy()
                a_[c] += hz
                b_[c] -= hz
                g[c] = (psi(eps, T, a_) - psi(eps, T, b_)) / (2 * hz)
        return g

    d2_te = (grad(th + hT, "e") - grad(th - hT, "e")) / (2 * hT)
    d2_tz = (grad(th + hT, "z") - grad(th - hT, "z")) / (2 * hT)
    edot = (eps - zn[7:]) / dt
    zdot = (z1 - zn[:7]) / dt
    thermal = th * d2_te @ edot + th * d2_tz @ zdot
    assert r["D"] - r["diss"] == pytest.approx(thermal, rel=1e-6, abs=1e-9)


def test_perzyna_homogeneous_tree_gives_phase_response():
    """All leaves Perzyna: zero jumps, and the DMN returns the leaf law."""
    K = 3
    mats = syn.materials_viscoplastic()
    t, w, n = make_tree(K, mats, phase=np.ones(2 ** K, np.uint8))
    s = t.init_state(1, 293.0)
    eps, _ = _plastic_case()
    sout, out, st, _ = oracle.eval_batch(t, eps[None], [320.0], 0.5, s)
    assert st[0] == 0
    o = oracle.split_out(out[0])
    r = oracle.leaf(mats[1], eps, 320.0, np.zeros(13), 0.0, 0.5)
    assert np.abs(sout[0, 8:8 + 3 * t.nnode]).max() < 1e-12
    np.testing.assert_allclose(o["sig"], r["sig"], rtol=1e-11, atol=1e-9)
    np.testing.assert_allclose(o["C"], r["C"], rtol=1e-9, atol=1e-7)
    np.testing.assert_allclose(o["C_theta"], r["tau"], rtol=1e-9, atol=1e-9)
    assert o["D"] == pytest.approx(r["D"], rel=1e-10)
    np.testing.assert_allclose(o["D_eps"], r["d"], rtol=1e-9, atol=1e-9)
    assert o["D_theta"] == pytest.approx(r["g"], rel=1e-9, abs=1e-12)
    # state: every leaf's z = the leaf law's, including its strain
    z = sout[0, 8 + 3 * t.nnode:8 + 3 * t.nnode + 13]
    np.testing.assert_allclose(z, r["znew"], rtol=1e-12, atol=1e-15)
