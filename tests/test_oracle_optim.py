"""Pins of the FP64 AMSGrad step (oracle/optim.py): a two-step example worked
by hand in which one parameter takes the running-maximum branch, the closed
form of a first step from zero moments, and the closed form with b1 = b2 = 0
(the step divides by the largest |g| seen so far)."""
import os

import numpy as np

from oracle import optim

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "amsgrad_two_steps.txt")


def test_two_steps_worked_by_hand():
    rows = np.loadtxt(GOLDEN)
    w, m, v, vm = np.array([0.0, 1.0]), np.zeros(2), np.zeros(2), np.zeros(2)
    for t, g in ((1, [1.0, 0.5]), (2, [0.01, -2.0])):
        w, m, v, vm = optim.amsgrad_step(w, g, m, v, vm, t, 0.1, 0.9, 0.999, 0.01)
        ref = rows[t - 1]
        np.testing.assert_allclose(w, ref[1:3], rtol=1e-14, atol=0)
        np.testing.assert_allclose(m, ref[3:5], rtol=1e-14, atol=0)
        np.testing.assert_allclose(v, ref[5:7], rtol=1e-14, atol=0)
        np.testing.assert_allclose(vm, ref[7:9], rtol=1e-14, atol=0)
    # the branch was taken: vmax of A kept the first step's value, above v
    assert vm[0] > v[0]


def test_first_step_is_lr_g_over_abs_g_plus_eps():
    rng = np.random.default_rng(0)
    w0, g = rng.normal(size=50), rng.normal(size=50) * 10.0 ** rng.uniform(-9, 1, 50)
    z = np.zeros(50)
    lr, eps = 3e-3, 1e-8
    w, m, v, vm = optim.amsgrad_step(w0, g, z, z, z, 1, lr, 0.9, 0.999, eps)
    # bias correction makes m_hat = g and vmax_hat = g^2 after one step
    np.testing.assert_allclose(w, w0 - lr * g / (np.abs(g) + eps), rtol=1e-13, atol=1e-18)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(vm, v, rtol=0)


def test_no_moment_memory_divides_by_the_largest_gradient_so_far():
    rng = np.random.default_rng(1)
    G = rng.normal(size=(6, 20)) * np.array([1.0, 3.0, 0.1, 0.2, 5.0, 0.01])[:, None]
    w = np.zeros(20)
    m = v = vm = np.zeros(20)
    big = np.zeros(20)
    ref = np.zeros(20)
    for t, g in enumerate(G, start=1):
        w, m, v, vm = optim.amsgrad_step(w, g, m, v, vm, t, 0.5, 0.0, 0.0, 1e-3)
        big = np.maximum(big, np.abs(g))
        ref = ref - 0.5 * g / (big + 1e-3)
    np.testing.assert_allclose(w, ref, rtol=1e-13, atol=1e-15)
