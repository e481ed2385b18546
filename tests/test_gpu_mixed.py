"""Mixed strain / stress control with adiabatic heating on the GPU
(``dmn_eval_mixed`` through the C ABI) against closed forms and against the
oracle's outer Newton (``oracle.eval_mixed``).

Tolerances.  Both sides stop their outer Newton when every prescribed stress
is within tol_outer = 1e-11 (relative to max(|sigma_bar|, 1 MPa)) of its target
and the heat balance within tol_outer c/dt; the inner solves differ as in the
strain-driven parity tests (stress 1e-10 FP64, 1e-8 mixed).  A stress error
delta maps to a strain error of about delta / E_t with a tangent modulus E_t
that drops to about H = 300 MPa where the matrix flows, i.e. up to
(2.5e3/300) delta relative: strains are compared at 1e-7 (FP64) and 1e-6
(mixed) of their largest magnitude per point, the temperature change at the
same fraction of max(|theta - theta^n|, 1e-3 K), with a factor of 20 for a
20-increment path.
"""
import numpy as np
import pytest

import oracle
from paper_2109_14403_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TH0 = 293.0
ALL_STRESS, ADIABATIC = 0x3F, 0x40
TOL_OUTER = 1e-11
RTOL = {"fp64": 1e-7, "mixed": 1e-6}


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _t(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=_dev())


def gpu_step(d, mask, target, deps0, theta0, dt, c, s, **kw):
    deps = _t(deps0)
    th = _t(theta0)
    so, out, st, it, outer = d.eval_mixed(_t(mask, torch.uint8), _t(target), deps, th, dt, c, s,
                                          tol_outer=TOL_OUTER, **kw)
    return deps, th, so, out, st, outer


def make(K, mats, prec, homogeneous=False, seed=None):
    from paper_2109_14403_gb300 import DMN
    w, n, ph = syn.tree(K, seed)
    if homogeneous:
        ph = np.zeros_like(ph)
    d = DMN(K, w, n, ph, mats, tol=1e-12, precision=prec)
    return d, oracle.Tree(K, w, n, ph, mats), syn.effective_heat_capacity(w, ph) if not homogeneous else None


def check_against(prec, de_g, th_g, out_g, de_o, th_o, out_o, thn, mask, target, scale=1.0):
    r = RTOL[prec] * scale
    emax = np.maximum(np.abs(de_o).max(axis=1), 1e-6)
    assert (np.abs(de_g - de_o).max(axis=1) <= r * emax).all()
    dT = np.maximum(np.abs(th_o - thn), 1e-3)
    assert (np.abs(th_g - th_o) <= r * dT).all()
    # the prescribed stresses themselves, and the heat balance, on the GPU side
    for i in range(mask.size):
        smax = max(1.0, np.abs(out_g[i, :6]).max())
        for c in range(6):
            if (mask[i] >> c) & 1:
                assert abs(out_g[i, c] - target[i, c]) <= TOL_OUTER * smax
            else:
                assert de_g[i, c] == target[i, c]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_closed_forms(prec):
    """The CPU pins' closed forms, reproduced through the C ABI."""
    from scipy.optimize import brentq
    dev = _dev()
    rtol = 1e-9 if prec == "fp64" else 1e-7
    # thermoelastic: Hooke at theta = 320 K, and Kelvin's adiabatic cooling
    E, nu, al, c, dt = 70000.0, 0.22, 5e-6, 2.0, 0.01
    d, _, _ = make(4, [[0, E, nu, al, TH0, 0, 0, 0]], prec, homogeneous=True)
    s0 = d.init_state(torch.full((2,), TH0, dtype=torch.float64, device=dev))
    s = 100.0
    tgt = np.zeros((2, 6))
    tgt[:, 0] = s
    de, th, so, out, st, outer = gpu_step(d, np.array([ALL_STRESS, ALL_STRESS | ADIABATIC], np.uint8),
                                          tgt, np.zeros((2, 6)), [320.0, TH0], dt, c, s0)
    de, th, st = de.cpu().numpy(), th.cpu().numpy(), st.cpu().numpy()
    assert (st == 0).all()
    dT = 320.0 - TH0
    np.testing.assert_allclose(de[0, :3], [s / E + al * dT, -nu * s / E + al * dT,
                                           -nu * s / E + al * dT], rtol=rtol)
    K = E / (3 * (1 - 2 * nu))
    A, B, C = 9 * K * al**2, c + 9 * K * al**2 * TH0 + al * s, al * TH0 * s
    dT = (-B + np.sqrt(B * B - 4 * A * C)) / (2 * A)
    assert abs(th[1] - TH0 - dT) <= 1e-6 * abs(dT)
    d.close()
    # J2 with linear hardening, adiabatic
    E, nu, al, sy0, dsy, H = 2500.0, 0.38, 8e-5, 50.0, -0.3, 300.0
    d, _, _ = make(3, [[1, E, nu, al, TH0, sy0, dsy, H]], prec, homogeneous=True)
    s0 = d.init_state(torch.full((1,), TH0, dtype=torch.float64, device=dev))
    s, c, dt = 80.0, 1.5, 1.0
    tgt = np.zeros((1, 6))
    tgt[0, 0] = s
    de, th, so, out, st, outer = gpu_step(d, np.array([ALL_STRESS | ADIABATIC], np.uint8), tgt,
                                          np.zeros((1, 6)), [TH0], dt, c, s0, max_outer=50)
    de, th = de.cpu().numpy(), th.cpu().numpy()
    assert st.cpu().numpy()[0] == 0
    Kb = E / (3 * (1 - 2 * nu))

    def heat(x):
        th_ = TH0 + x
        sy = sy0 + dsy * x
        return c * x + al * th_ * s + 9 * Kb * al**2 * th_ * x - sy * (s - sy) / H
    dT = brentq(heat, -50.0, 50.0, xtol=1e-14)
    p = (s - (sy0 + dsy * dT)) / H
    assert abs(th[0] - TH0 - dT) <= 1e-6 * abs(dT)
    np.testing.assert_allclose(de[0, :3], [s / E + p + al * dT, -nu * s / E - p / 2 + al * dT,
                                           -nu * s / E - p / 2 + al * dT], rtol=rtol * 10)
    d.close()


MASKS = np.array([0x7F, 0x3F, 0x06, 0x46, 0x40, 0x7E, 0x00, 0x41], np.uint8)


def random_case(m, seed):
    rng = np.random.default_rng(seed)
    mask = MASKS[np.arange(m) % MASKS.size]
    target = rng.normal(0, 40.0, (m, 6))
    strain = ((mask[:, None] >> np.arange(6)) & 1) == 0
    target[strain] = rng.normal(0, 3e-3, strain.sum())
    theta = TH0 + rng.uniform(0, 20, m)
    return mask, target, theta


@pytest.mark.parametrize("K", [3, 5, 8])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_composite_parity(K, prec):
    """Random masks (uniaxial, biaxial, lateral-free, pure strain, adiabatic
    or not) on a two-phase tree, against the oracle's outer Newton."""
    dev = _dev()
    d, tree, c = make(K, syn.materials_cyclic(), prec)
    m = 40
    mask, target, theta = random_case(m, 100 + K)
    dt = 0.01
    s0 = d.init_state(torch.full((m,), TH0, dtype=torch.float64, device=dev))
    de, th, so, out, st, outer = gpu_step(d, mask, target, np.zeros((m, 6)), theta, dt, c, s0,
                                          max_outer=40)
    so_o0 = tree.init_state(m, TH0)
    de_o, th_o, so_o, out_o, st_o, outer_o = oracle.eval_mixed(
        tree, mask, target, np.zeros((m, 6)), theta, dt, c, so_o0, max_outer=40, tol_outer=TOL_OUTER)
    st = st.cpu().numpy()
    assert ((st & ~4) == 0).all() and (st_o == 0).all()
    check_against(prec, de.cpu().numpy(), th.cpu().numpy(), out.cpu().numpy(), de_o, th_o, out_o,
                  TH0, mask, target)
    assert (outer.cpu().numpy() <= outer_o + 2).all()
    d.close()


@pytest.mark.parametrize("matrix,predict", [("perzyna", False), ("perzyna", True), ("pa66", True)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cyclic_self_heating_path(prec, matrix, predict):
    """One load cycle (20 increments) of the stress-controlled adiabatic
    cyclic workload, GPU and oracle each on their own trajectory (with the
    tangent predictor on both sides, or on neither); the matrix is the
    Perzyna law of the workload or the paper's PA66 law."""
    dev = _dev()
    K = 5
    mats = syn.materials_pa66() if matrix == "pa66" else syn.materials_cyclic()
    d, tree, c = make(K, mats, prec)
    mask, target, dt, amp, direction = syn.cyclic_stress(8 if matrix == "pa66" else 16, 1, seed=3)
    n = mask.size
    s = d.init_state(torch.full((n,), TH0, dtype=torch.float64, device=dev))
    so = tree.init_state(n, TH0)
    deps_g = np.zeros((n, 6))
    th_g = np.full(n, TH0)
    deps_o, th_o = deps_g.copy(), th_g.copy()
    out, out_o = None, None
    evals = 0
    for k in range(target.shape[0]):
        thn_o = so[:, 6].copy()
        pred = predict and out is not None
        de, th, s, out, st, outer = gpu_step(d, mask, target[k], deps_g, th_g, dt, c, s,
                                             out=out if pred else None, predict=pred)
        deps_g, th_g = de.cpu().numpy(), th.cpu().numpy()
        assert ((st.cpu().numpy() & ~4) == 0).all()
        assert (out[:, 56].cpu().numpy() >= 0.0).all()  # dissipation
        evals += int(outer.sum().item())
        deps_o, th_o, so, out_o, st_o, _ = oracle.eval_mixed(tree, mask, target[k], deps_o, th_o, dt,
                                                             c, so, tol_outer=TOL_OUTER,
                                                             out_prev=out_o if pred else None)
        assert (st_o == 0).all()
        check_against(prec, deps_g, th_g, out.cpu().numpy(), deps_o, th_o, out_o, thn_o, mask,
                      target[k], scale=20.0)
        eb = s[:, :6].cpu().numpy()
        emax = np.maximum(np.abs(so[:, :6]).max(axis=1), 1e-6)
        assert (np.abs(eb - so[:, :6]).max(axis=1) <= 20 * RTOL[prec] * emax).all()
    if predict and matrix == "perzyna":  # the predictor leaves about 2.3 evaluations per increment
        assert evals <= 2.6 * n * target.shape[0]
    if matrix == "pa66":  # the Maxwell branches still carry the last half cycle
        d.close()
        return
    # self-heating after one cycle grows with the amplitude
    rise = th_g - TH0
    for a_lo, a_hi in zip(syn.CYCLE_AMPLITUDES[:-1], syn.CYCLE_AMPLITUDES[1:]):
        lo, hi = rise[amp == a_lo], rise[amp == a_hi]
        if lo.size and hi.size:
            assert hi.max() > lo.min()
    d.close()


@pytest.mark.parametrize("prec,matrix", [("mixed", "perzyna"), ("mixed", "pa66")])
def test_cyclic_full_batch_sampled(prec, matrix):
    """65,536 points on a K = 8 tree (the benchmark's cyclic workload, with
    either matrix), three increments; the oracle follows sampled points."""
    dev = _dev()
    mats = syn.materials_pa66() if matrix == "pa66" else syn.materials_cyclic()
    d, tree, c = make(8, mats, prec)
    n = 65536
    mask, target, dt, amp, direction = syn.cyclic_stress(n, 1, seed=42)
    idx = np.linspace(0, n - 1, 8 if matrix == "pa66" else 32).astype(int)
    idx_d = torch.tensor(idx, device=dev)
    s = d.init_state(torch.full((n,), TH0, dtype=torch.float64, device=dev))
    so = tree.init_state(idx.size, TH0)
    de = torch.zeros((n, 6), dtype=torch.float64, device=dev)
    th = torch.full((n,), TH0, dtype=torch.float64, device=dev)
    deps_o, th_o = np.zeros((idx.size, 6)), np.full(idx.size, TH0)
    mask_d = _t(mask, torch.uint8)
    for k in range(3):
        thn_o = so[:, 6].copy()
        s, out, st, it, outer = d.eval_mixed(mask_d, _t(target[k]), de, th, dt, c, s,
                                             tol_outer=TOL_OUTER)
        assert ((st.cpu().numpy() & ~4) == 0).all()
        deps_o, th_o, so, out_o, st_o, _ = oracle.eval_mixed(tree, mask[idx], target[k][idx], deps_o,
                                                             th_o, dt, c, so, tol_outer=TOL_OUTER)
        check_against(prec, de[idx_d].cpu().numpy(), th[idx_d].cpu().numpy(),
                      out[idx_d].cpu().numpy(), deps_o, th_o, out_o, thn_o, mask[idx],
                      target[k][idx], scale=3.0)
    d.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_predictor_is_exact_for_linear_phases(prec):
    """Linear thermoelastic phases, isothermal mixed control: the tangent
    predictor's start already meets the conditions (one evaluation)."""
    dev = _dev()
    mats = [[0, 72000.0, 0.22, 5e-6, TH0, 0, 0, 0], [0, 2500.0, 0.38, 8e-5, TH0, 0, 0, 0]]
    d, tree, c = make(6, mats, prec)
    m = 16
    rng = np.random.default_rng(11)
    s0 = d.init_state(torch.full((m,), TH0, dtype=torch.float64, device=dev))
    s1, o1, st1, _ = d.eval(_t(rng.normal(0, 1e-3, (m, 6))), _t(np.full(m, 300.0)), 1.0, s0)
    mask = MASKS[np.arange(m) % 4]  # 0x7F, 0x3F, 0x06, 0x46
    mask = np.where(mask & ADIABATIC, mask & ALL_STRESS, mask).astype(np.uint8)
    target = rng.normal(0, 30.0, (m, 6))
    strain = ((mask[:, None] >> np.arange(6)) & 1) == 0
    target[strain] = rng.normal(0, 1e-3, strain.sum())
    tol = 1e-9 if prec == "fp64" else 1e-7
    so, out, st, it, outer = d.eval_mixed(_t(mask, torch.uint8), _t(target), _t(np.zeros((m, 6))),
                                          _t(np.full(m, 310.0)), 1.0, 2.0, s1, out=o1.clone(),
                                          predict=True, tol_outer=tol)
    # FP64 tangents make the linear model exact to rounding; the mixed path's
    # come from the FP32 condensation (relative error up to ~1e-5), which
    # leaves one more evaluation
    assert (st.cpu().numpy() == 0).all()
    assert (outer.cpu().numpy() == 1).all() if prec == "fp64" else (outer.cpu().numpy() <= 2).all()
    d.close()


def test_cold_restarts_agree_with_warm():
    """Without the warm-start scratch every evaluation starts from a^n: the
    same solution within the tolerance."""
    dev = _dev()
    d, tree, c = make(5, syn.materials_cyclic(), "fp64")
    m = 24
    mask, target, theta = random_case(m, 7)
    s0 = d.init_state(torch.full((m,), TH0, dtype=torch.float64, device=dev))
    r1 = gpu_step(d, mask, target, np.zeros((m, 6)), theta, 0.01, c, s0, max_outer=40)
    r2 = gpu_step(d, mask, target, np.zeros((m, 6)), theta, 0.01, c, s0, max_outer=40, warm=False)
    a, b = r1[0].cpu().numpy(), r2[0].cpu().numpy()
    assert (np.abs(a - b).max(axis=1) <= 1e-7 * np.maximum(np.abs(b).max(axis=1), 1e-6)).all()
    d.close()


def test_outer_limit_and_argument_errors():
    from paper_2109_14403_gb300 import dmn
    dev = _dev()
    d, tree, c = make(4, syn.materials_cyclic(), "mixed")
    m = 8
    mask, target, theta = random_case(m, 9)
    s0 = d.init_state(torch.full((m,), TH0, dtype=torch.float64, device=dev))
    de, th, so, out, st, outer = gpu_step(d, mask, target, np.zeros((m, 6)), theta, 0.01, c, s0,
                                          max_outer=1)
    st, outer = st.cpu().numpy(), outer.cpu().numpy()
    assert (outer == 1).all()
    controlled = (mask & 0x7F) != 0
    assert ((st & dmn.PT_OUTER_NOT_CONVERGED) != 0)[controlled].all()
    assert ((st & dmn.PT_OUTER_NOT_CONVERGED) == 0)[~controlled].all()
    for kw, msg in [(dict(max_outer=0), "max_outer"), (dict(tol_outer=0.0), "tol_outer")]:
        with pytest.raises(RuntimeError, match=msg):
            d.eval_mixed(_t(mask, torch.uint8), _t(target), _t(np.zeros((m, 6))), _t(theta), 0.01,
                         c, s0, **kw)
    with pytest.raises(RuntimeError, match="c_heat"):
        d.eval_mixed(_t(mask, torch.uint8), _t(target), _t(np.zeros((m, 6))), _t(theta), 0.01, 0.0,
                     s0)
    d.close()
