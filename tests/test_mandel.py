"""Mandel <-> Voigt (ABAQUS order, engineering shear) conversions of the host
module paper_2109_14403_gb300.mandel, checked against definitions fixed
independently of it: the double contraction, the tangent acting on a strain,
the isotropic tangent in Lame form, and a pure shear written out by hand."""
import numpy as np
import pytest

from paper_2109_14403_gb300 import mandel

torch = pytest.importorskip("torch")


def _sym(rng):
    a = rng.normal(size=(3, 3))
    return a + a.T


def _mandel_of(t):
    r = np.sqrt(2.0)
    return np.array([t[0, 0], t[1, 1], t[2, 2], r * t[1, 2], r * t[0, 2], r * t[0, 1]])


def test_pure_shear_by_hand():
    tau = 3.0
    s_m = np.array([0, 0, 0, 0, 0, np.sqrt(2.0) * tau])  # sigma_12 = tau
    np.testing.assert_allclose(mandel.stress_to_voigt(s_m), [0, 0, 0, tau, 0, 0], atol=1e-15)
    g = 0.02  # engineering shear gamma_23 = 2 eps_23
    e_m = mandel.strain_to_mandel(np.array([0, 0, 0, 0, 0, g]))
    np.testing.assert_allclose(e_m, [0, 0, 0, np.sqrt(2.0) * g / 2, 0, 0], atol=1e-15)


def test_round_trips_and_double_contraction():
    rng = np.random.default_rng(1)
    for _ in range(20):
        s, e = _sym(rng), _sym(rng)
        s_m, e_m = _mandel_of(s), _mandel_of(e)
        s_v, e_v = mandel.stress_to_voigt(s_m), mandel.strain_to_voigt(e_m)
        np.testing.assert_allclose(mandel.stress_to_mandel(s_v), s_m, rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(mandel.strain_to_mandel(e_v), e_m, rtol=1e-14, atol=1e-14)
        # s : e as the full double contraction, in both notations
        full = np.sum(s * e)
        assert abs(s_m @ e_m - full) < 1e-12 * (1 + abs(full))
        assert abs(s_v @ e_v - full) < 1e-12 * (1 + abs(full))
        # engineering shear: gamma_12 = 2 eps_12 in Voigt slot 3
        assert abs(e_v[3] - 2 * e[0, 1]) < 1e-14 and abs(e_v[5] - 2 * e[1, 2]) < 1e-14


def test_tangent_acts_on_voigt_strains():
    rng = np.random.default_rng(2)
    a = rng.normal(size=(6, 6))
    c_m = a @ a.T
    c_v = mandel.tangent_to_voigt(c_m)
    np.testing.assert_allclose(c_v, c_v.T, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(mandel.tangent_to_mandel(c_v), c_m, rtol=1e-14, atol=1e-13)
    for _ in range(10):
        e_m = rng.normal(size=6)
        lhs = mandel.stress_to_voigt(c_m @ e_m)
        rhs = c_v @ mandel.strain_to_voigt(e_m)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-13, atol=1e-13)


def test_isotropic_tangent_in_lame_form():
    E, nu = 2500.0, 0.38
    lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    K = lam + 2 * mu / 3
    P1 = np.zeros((6, 6))
    P1[:3, :3] = 1.0 / 3.0
    P2 = np.eye(6) - P1
    c_m = 3 * K * P1 + 2 * mu * P2  # Mandel: the projector form
    ref = np.zeros((6, 6))
    ref[:3, :3] = lam
    ref[np.arange(3), np.arange(3)] += 2 * mu
    ref[3, 3] = ref[4, 4] = ref[5, 5] = mu  # engineering shear
    np.testing.assert_allclose(mandel.tangent_to_voigt(c_m), ref, rtol=1e-13, atol=1e-10)


def test_strain_gradient():
    rng = np.random.default_rng(3)
    g_m = rng.normal(size=6)
    g_v = mandel.strain_gradient_to_voigt(g_m)
    for _ in range(10):
        e_v = rng.normal(size=6)
        assert abs(g_v @ e_v - g_m @ mandel.strain_to_mandel(e_v)) < 1e-13


def test_torch_batches_match_numpy():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(5, 6))
    c = rng.normal(size=(5, 6, 6))
    for f in (mandel.stress_to_voigt, mandel.strain_to_mandel, mandel.strain_gradient_to_voigt):
        np.testing.assert_allclose(f(torch.tensor(x)).numpy(), f(x), rtol=1e-15)
    np.testing.assert_allclose(mandel.tangent_to_voigt(torch.tensor(c)).numpy(), mandel.tangent_to_voigt(c),
                               rtol=1e-15)
