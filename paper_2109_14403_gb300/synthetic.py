"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the method: it only draws random trees and
load paths and lists material parameters.  Both the CUDA path and the CPU oracle
consume what it returns.

Workloads (the paper's own trained DMN and FFT data are not available, so these
stand in for its strain-controlled virtual experiments, Sec. 5.4):
  * tree: leaf weights ~ Dirichlet(1) over 2^K leaves, lamination directions
    uniform on the unit sphere, phases alternating as in Sec. 3.3 (leaf j,
    0-based, takes material row j mod 2: even leaves the fiber, odd leaves
    the matrix), seed 1234 + K;
  * fiber: isotropic linear thermoelastic E = 72 GPa, nu = 0.22, alpha = 5e-6/K;
  * matrix: J2 elastoplastic, linear isotropic hardening 300 MPa,
    E = 2.5 GPa, nu = 0.38, alpha = 8e-5/K, yield 50 MPa at 293 K falling
    0.3 MPa/K;
  * K=4 ramp: 64 points, 20 increments of 0.1 % in the 11 component plus
    N(0, 1e-4) on all six Mandel components, temperature 293 -> 353 K;
  * K=8 random walk: 65,536 points, 50 increments with N(0, 2e-4) on every
    Mandel component and temperature steps U(0, 1) K from 293 K;
  * uneven batch: points spread evenly (shuffled) over three DMNs of depth 6,
    7 and 8 with independent seeds; strain increments with a direction
    uniform on the unit sphere of R^6 and a magnitude s0 * LogNormal(0, 1),
    so Newton iteration counts vary from point to point; temperature steps as
    above;
  * viscoplastic matrix (large configuration): the matrix above with a
    Perzyna overstress rate law, rate exponent 5, viscous time 1e3 s, and
    moduli falling 0.2 %/K; K = 9 tree (seed 1234 + 9); 100 increments of
    dt = 0.01 s with strain rates N(0, 1e-2)/s per Mandel component and the
    temperature ramped 293 -> 393 K (1 K per increment);
  * stress-controlled cyclic loading (Sec. 5.4, cyclic validation): uniaxial
    sinusoidal stress sigma_ampl sin(2 pi t / T_c) in the 11 or the 22
    direction, all other stress components 0, adiabatic; T_c = 0.1 s (10 Hz),
    20 increments per cycle, amplitudes 20, 40, 60 and 80 MPa; each point
    draws its amplitude and direction; volumetric heat capacities 2.1 MPa/K
    (E-glass) and 1.9 MPa/K (PA66), the paper's material tables, averaged
    with the leaf weights; the matrix is the Perzyna matrix with the PA66
    rate law's exponent m = 2 and viscous time eta_0 / sigma_Y0 = 74/15.5 s
    and, as the PA66's, moduli that do not depend on the temperature.
Units: MPa, K, s.  Symmetric tensors are Mandel 6-vectors.
"""
from __future__ import annotations

import numpy as np

# material table rows: kind, E, nu, alpha, theta0, sy0, dsy_dT, H
#   (+ for kind 2: rate exponent m, viscous time t_visc (s), dE_dT (1/K), 0)
KIND_THERMOELASTIC = 0
KIND_J2_LINEAR = 1
KIND_J2_PERZYNA = 2
FIBER = (KIND_THERMOELASTIC, 72000.0, 0.22, 5e-6, 293.0, 0.0, 0.0, 0.0)
MATRIX = (KIND_J2_LINEAR, 2500.0, 0.38, 8e-5, 293.0, 50.0, -0.3, 300.0)
MATRIX_PERZYNA = (KIND_J2_PERZYNA, 2500.0, 0.38, 8e-5, 293.0, 50.0, -0.3, 300.0, 5.0, 1e3, -0.002, 0.0)
THETA_START = 293.0
KIND_PA66 = 3
# PA66 matrix (Sec. 4, after Krairi et al.; the paper's material table): E_inf, nu,
# alpha0, theta0 (the paper's reference temperature of its validation runs), sigma_Y0,
# hardening k and exponent n, rate exponent m, eta0, beta1, beta2, theta_ref, WLF C1,
# C2, then the 12 Maxwell moduli E_i (MPa) and relaxation times tau_i (s)
PA66_E_MAXWELL = (265.0, 262.0, 248.0, 231.0, 211.0, 190.0, 170.0, 92.0, 78.0, 65.0, 54.0, 48.0)
PA66_LOG10_TAU = (-4.22, -3.42, -2.63, -1.84, -1.05, -0.26, 0.53, 1.32, 2.12, 2.91, 3.70, 4.49)
MATRIX_PA66 = ((KIND_PA66, 1500.0, 0.42, 70e-6, 293.15, 15.5, 103.0, 0.32, 2.0, 74.0, 0.011, 0.07,
                298.15, 26.21, 446.31, 0.0) + PA66_E_MAXWELL + tuple(10.0 ** t for t in PA66_LOG10_TAU))
# volumetric heat capacity c_0 (MPa/K = 1e6 J m^-3 K^-1) of the rows of
# materials(): E-glass fiber and PA66 matrix (Sec. 4, material tables)
HEAT_CAPACITY = (2.1, 1.9)
CYCLE_PERIOD = 0.1
CYCLE_STEPS = 20
CYCLE_AMPLITUDES = (20.0, 40.0, 60.0, 80.0)
# dmn_eval_mixed mask: all six stress components prescribed, adiabatic
MASK_STRESS_ADIABATIC = 0x7F
LARGE_K = 9
LARGE_DT = 0.01


def materials():
    return np.array([FIBER, MATRIX], dtype=np.float64)


def materials_viscoplastic():
    """Fiber and the Perzyna matrix as 12-column rows."""
    fib = np.zeros(12)
    fib[:8] = FIBER
    return np.array([fib, MATRIX_PERZYNA], dtype=np.float64)


def materials_pa66():
    """E-glass fiber and the PA66 matrix as 40-column rows."""
    fib = np.zeros(40)
    fib[:8] = FIBER
    return np.array([fib, MATRIX_PA66], dtype=np.float64)


def materials_cyclic():
    """Fiber and the matrix of the cyclic workload as 12-column rows."""
    m = materials_viscoplastic()
    m[1, 8], m[1, 9], m[1, 10] = 2.0, 74.0 / 15.5, 0.0
    return m


def large_path(n_points=1048576, n_incr=100, seed=42, dtype=np.float64):
    """Strain-rate path of the large configuration: deps = rate * dt with rates
    N(0, 1e-2)/s, theta = 293 + k K at increment k (1-based).
    Returns (deps[n_incr, n, 6], theta[n_incr, n])."""
    rng = np.random.default_rng(seed)
    deps = (rng.standard_normal((n_incr, n_points, 6)) * (1e-2 * LARGE_DT)).astype(dtype)
    theta = (THETA_START + np.arange(1, n_incr + 1, dtype=np.float64)[:, None]
             * np.ones((1, n_points))).astype(dtype)
    return deps, theta


def tree(K: int, seed: int | None = None):
    """Random DMN parameters: (w, normals in paper order, phase map)."""
    rng = np.random.default_rng(1234 + K if seed is None else seed)
    g = rng.gamma(1.0, 1.0, size=1 << K)
    w = g / g.sum()
    v = rng.standard_normal(((1 << K) - 1, 3))
    normals = v / np.linalg.norm(v, axis=1, keepdims=True)
    phase = (np.arange(1 << K) % 2).astype(np.uint8)  # odd leaves: row 1 (the matrix)
    return w, normals, phase


def ramp_k4(n_points=64, n_incr=20, seed=42):
    """Uniaxial 2 % ramp with noise; returns (deps[n_incr, n, 6], theta[n_incr, n])."""
    rng = np.random.default_rng(seed)
    deps = rng.normal(0.0, 1e-4, size=(n_incr, n_points, 6))
    deps[:, :, 0] += 1e-3
    theta = THETA_START + 3.0 * np.arange(1, n_incr + 1)[:, None] * np.ones((1, n_points))
    return deps, theta


def random_walk_k8(n_points=65536, n_incr=50, seed=42):
    """Random-walk strain path; returns (deps[n_incr, n, 6], theta[n_incr, n])."""
    rng = np.random.default_rng(seed)
    deps = rng.normal(0.0, 2e-4, size=(n_incr, n_points, 6))
    dth = rng.uniform(0.0, 1.0, size=(n_incr, n_points))
    theta = THETA_START + np.cumsum(dth, axis=0)
    return deps, theta


def single_increment(n_points, seed=7, scale=2e-4, theta=300.0):
    """One increment of N(0, scale) strain on every component at a fixed temperature."""
    rng = np.random.default_rng(seed)
    deps = rng.normal(0.0, scale, size=(n_points, 6))
    th = np.full(n_points, theta)
    return deps, th


UNEVEN_DEPTHS = (6, 7, 8)


def uneven_batch(n_points=262144, n_incr=50, s0=1e-3, seed=42):
    """Returns (tree_id[n], deps[n_incr, n, 6], theta[n_incr, n]); tree_id
    indexes UNEVEN_DEPTHS, trees come from tree(K, seed=2000 + K)."""
    rng = np.random.default_rng(seed)
    tree_id = rng.permutation(np.arange(n_points) % len(UNEVEN_DEPTHS)).astype(np.int32)
    d = rng.standard_normal((n_incr, n_points, 6))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    mag = s0 * rng.lognormal(0.0, 1.0, size=(n_incr, n_points, 1))
    dth = rng.uniform(0.0, 1.0, size=(n_incr, n_points))
    theta = THETA_START + np.cumsum(dth, axis=0)
    return tree_id, d * mag, theta


def uneven_trees():
    return [tree(K, seed=2000 + K) for K in UNEVEN_DEPTHS]


def effective_heat_capacity(w, phase, c_by_material=HEAT_CAPACITY):
    """Leaf-weighted mean of the phases' heat capacities (MPa/K)."""
    return float(np.sum(np.asarray(w) * np.asarray(c_by_material)[np.asarray(phase)]))


def cyclic_stress(n_points, n_cycles=1, seed=42, steps_per_cycle=CYCLE_STEPS, period=CYCLE_PERIOD,
                  amplitudes=CYCLE_AMPLITUDES):
    """Stress-controlled adiabatic cyclic loading.  Returns (mask[n] uint8,
    target[n_incr, n, 6] prescribed Mandel stresses, dt, amplitude[n],
    direction[n] in {0, 1} = 11 or 22)."""
    rng = np.random.default_rng(seed)
    amp = np.asarray(amplitudes, np.float64)[rng.integers(0, len(amplitudes), n_points)]
    direction = rng.integers(0, 2, n_points)
    dt = period / steps_per_cycle
    t = dt * np.arange(1, n_cycles * steps_per_cycle + 1)
    target = np.zeros((t.size, n_points, 6))
    target[:, np.arange(n_points), direction] = np.sin(2.0 * np.pi * t / period)[:, None] * amp
    mask = np.full(n_points, MASK_STRESS_ADIABATIC, np.uint8)
    return mask, target, dt, amp, direction



def iso_mandel(E, nu):
    """Isotropic stiffness 3K P1 + 2G P2 as 6x6 Mandel matrices (E, nu arrays)."""
    E, nu = np.asarray(E, np.float64), np.asarray(nu, np.float64)
    K, G = E / (3 * (1 - 2 * nu)), E / (2 * (1 + nu))
    P1 = np.zeros((6, 6))
    P1[:3, :3] = 1.0 / 3.0
    P2 = np.eye(6) - P1
    return 3 * K[..., None, None] * P1 + 2 * G[..., None, None] * P2


def stiffness_pairs(n_samples, seed=7, log10_contrast=2.0):
    """Phase stiffness pairs for offline training (stand-in for the paper's
    sampled 8-D set, Sec. 5.1): C_1 isotropic with E_1 = 1, C_2 isotropic with
    E_2 = 10^U(-c, c), both nu ~ U(0.1, 0.45); C_2 loses a random rank-one
    part, C_2 - t m m^T / (m^T C_2^-1 m) with unit m and t ~ U(0, 0.5), which
    keeps it positive definite (the largest rank-one reduction along m that
    does is t = 1), so it is anisotropic with a smallest eigenvalue at least
    half the isotropic one along m.  Returns C1s, C2s [n, 6, 6]."""
    rng = np.random.default_rng(seed)
    C1 = iso_mandel(np.ones(n_samples), rng.uniform(0.1, 0.45, n_samples))
    C2 = iso_mandel(10.0 ** rng.uniform(-log10_contrast, log10_contrast, n_samples),
                    rng.uniform(0.1, 0.45, n_samples))
    m = rng.standard_normal((n_samples, 6))
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    t = rng.uniform(0.0, 0.5, n_samples)
    mCim = np.einsum("si,si->s", m, np.linalg.solve(C2, m[:, :, None])[:, :, 0])
    C2 = C2 - (t / mCim)[:, None, None] * np.einsum("si,sj->sij", m, m)
    return C1, C2


def linear_params(K, seed=None):
    """Random DMN^L parameters: normals [(2^K-1), 3] (not normalised) and
    unconstrained weights v [2^K] (positive, summing to about 1)."""
    rng = np.random.default_rng(4321 + K if seed is None else seed)
    normals = rng.standard_normal(((1 << K) - 1, 3))
    v = rng.uniform(0.5, 1.5, 1 << K)
    return normals, v / v.sum()
