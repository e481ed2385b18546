"""dmn_eval_noalloc: one load increment without any device allocation.

Some users of the library cannot call cudaMalloc: a material routine called
by a host finite-element code that owns all device memory through its own
pool, a sandboxed or real-time plug-in, or code that cannot keep a dmn_handle
alive between calls.  For them the library exports dmn_eval_noalloc, which
takes the tree and materials from host memory on every call and keeps the
derived tables and its work-queue counter in a fixed device array inside the
library.  These tests call it through the C ABI (ctypes on libdmn.so) and
check that it returns what dmn_eval returns, on two calls in a row, within the
tolerances of the parity tests.  (The test itself allocates its buffers with
PyTorch; the entry point under test allocates nothing.)
"""
import ctypes

import numpy as np
import pytest

from paper_2109_14403_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# relative tolerances of the parity tests (stress, tangents)
TOL = {"fp64": (1e-10, 1e-8), "mixed": (1e-8, 5e-6)}


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(lib, K, w, nrm, ph, mats, opt, deps, theta, dt, s_in):
    """Call the allocation-free entry point; return (state_out, out, status, iters)."""
    from paper_2109_14403_gb300 import dmn
    n = deps.shape[0]
    s_out = torch.empty_like(s_in)
    out = torch.empty((n, 57), dtype=torch.float64, device=deps.device)
    st = torch.empty(n, dtype=torch.int32, device=deps.device)
    it = torch.empty(n, dtype=torch.int32, device=deps.device)
    P = ctypes.c_void_p
    rc = lib.dmn_eval_noalloc(K, w.ctypes.data_as(P), nrm.ctypes.data_as(P), ph.ctypes.data_as(P),
                              ctypes.cast(mats, P), len(mats), ctypes.byref(opt),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), n,
                              _ptr(deps), _ptr(theta), dt, _ptr(s_in), _ptr(s_out), _ptr(out),
                              _ptr(st), _ptr(it))
    assert rc == dmn.DMN_OK, lib.dmn_last_error().decode()
    return s_out, out, st, it


def _rel(a, b, floor):
    return (np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), floor)).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_eval_on_two_calls_in_a_row(prec):
    from paper_2109_14403_gb300 import DMN, dmn
    dev = _dev()
    lib = dmn.load()
    K, n = 8, 301  # the largest depth the fixed array holds; a ragged batch
    w, nrm, ph = syn.tree(K)
    rows = syn.materials()
    mats = dmn.materials_from_rows(rows)
    opt = dmn.dmn_options()
    lib.dmn_default_options(ctypes.byref(opt))
    opt.tol = 1e-12
    opt.precision = dmn.PREC_MIXED if prec == "mixed" else dmn.PREC_FP64
    deps_h, theta_h = syn.random_walk_k8(n_points=n, n_incr=2)
    deps_h *= 8.0  # plastic increments: several Newton iterations
    ref = DMN(K, w, nrm, ph, rows, tol=1e-12, precision=prec)
    opt.solve_variant = ref.solve_variant  # the same kernel on both entry points
    s0 = ref.init_state(torch.full((n,), syn.THETA_START, dtype=torch.float64, device=dev))
    s_ref, s_na = s0, s0.clone()
    ts, tt = TOL[prec]
    for k in range(2):
        deps = torch.tensor(deps_h[k], device=dev)
        theta = torch.tensor(theta_h[k], device=dev)
        s_ref, out_r, st_r, it_r = ref.eval(deps, theta, 1.0, s_ref)
        s_na, out_n, st_n, it_n = _noalloc(lib, K, w, nrm, ph, mats, opt, deps, theta, 1.0, s_na)
        torch.cuda.synchronize()
        o_r, o_n = out_r.cpu().numpy(), out_n.cpu().numpy()
        assert (st_n.cpu().numpy() == 0).all() and (st_r.cpu().numpy() == 0).all()
        assert _rel(o_n[:, :6], o_r[:, :6], 1e-3) < ts
        assert _rel(o_n[:, 6:42], o_r[:, 6:42], 1.0) < tt
        np.testing.assert_allclose(o_n[:, 48], o_r[:, 48], rtol=ts, atol=ts * np.abs(o_r[:, 48]).max())
        np.testing.assert_allclose(s_na.cpu().numpy(), s_ref.cpu().numpy(), rtol=1e-9, atol=1e-14)
        np.testing.assert_array_equal(it_n.cpu().numpy(), it_r.cpu().numpy())
    ref.close()


def test_noalloc_rejects_a_tree_beyond_its_fixed_array():
    from paper_2109_14403_gb300 import dmn
    dev = _dev()
    lib = dmn.load()
    K, n = 9, 4
    w, nrm, ph = syn.tree(K)
    mats = dmn.materials_from_rows(syn.materials())
    opt = dmn.dmn_options()
    lib.dmn_default_options(ctypes.byref(opt))
    sw = 8 + 3 * ((1 << K) - 1) + 7 * (1 << (K - 1))
    s = torch.zeros((n, sw + (sw & 1)), dtype=torch.float64, device=dev)
    s2 = torch.zeros_like(s)
    z6 = torch.zeros((n, 6), dtype=torch.float64, device=dev)
    th = torch.full((n,), 300.0, dtype=torch.float64, device=dev)
    out = torch.empty((n, 57), dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    it = torch.empty(n, dtype=torch.int32, device=dev)
    P = ctypes.c_void_p
    rc = lib.dmn_eval_noalloc(K, w.ctypes.data_as(P), nrm.ctypes.data_as(P), ph.ctypes.data_as(P),
                              ctypes.cast(mats, P), len(mats), ctypes.byref(opt), None, n,
                              _ptr(z6), _ptr(th), 1.0, _ptr(s), _ptr(s2), _ptr(out), _ptr(st),
                              _ptr(it))
    assert rc == dmn.DMN_ERR_ARG
    assert b"outside 1..8" in lib.dmn_last_error()


def test_a_smaller_tree_leaves_a_live_larger_handle_launchable():
    """The compact solve kernel is one instance for every depth up to 8, and
    its shared-memory limit is a process-wide attribute.  Preparing a K = 4
    tree (through this entry point, or through a second handle) must not
    lower the limit below what a live K = 8 handle launches with: the K = 8
    handle's next dmn_eval still runs and gives the same bits."""
    from paper_2109_14403_gb300 import DMN, dmn
    dev = _dev()
    lib = dmn.load()
    K8, n = 8, 64
    w8, nrm8, ph8 = syn.tree(K8)
    rows = syn.materials()
    big = DMN(K8, w8, nrm8, ph8, rows, tol=1e-12, precision="mixed", solve_variant=13)
    deps_h, theta_h = syn.random_walk_k8(n_points=n, n_incr=1)
    deps = torch.tensor(deps_h[0] * 8.0, device=dev)
    theta = torch.tensor(theta_h[0], device=dev)
    s0 = big.init_state(torch.full((n,), syn.THETA_START, dtype=torch.float64, device=dev))
    _, out0, st0, _ = big.eval(deps, theta, 1.0, s0)
    torch.cuda.synchronize()
    assert (st0.cpu().numpy() == 0).all()

    # a K = 4 tree on the same kernel instance, through the allocation-free call
    K4 = 4
    w4, nrm4, ph4 = syn.tree(K4)
    opt = dmn.dmn_options()
    lib.dmn_default_options(ctypes.byref(opt))
    opt.tol, opt.precision, opt.solve_variant = 1e-12, dmn.PREC_MIXED, 13
    small = DMN(K4, w4, nrm4, ph4, rows, tol=1e-12, precision="mixed", solve_variant=13)
    s4 = small.init_state(torch.full((n,), syn.THETA_START, dtype=torch.float64, device=dev))
    mats = dmn.materials_from_rows(rows)
    _noalloc(lib, K4, w4, nrm4, ph4, mats, opt, deps, theta, 1.0, s4)
    _, out1, st1, _ = big.eval(deps, theta, 1.0, s0)
    # ... and through a second handle's own launch
    small.eval(deps, theta, 1.0, s4)
    _, out2, st2, _ = big.eval(deps, theta, 1.0, s0)
    torch.cuda.synchronize()
    for o, s in ((out1, st1), (out2, st2)):
        assert (s.cpu().numpy() == 0).all()
        np.testing.assert_array_equal(o.cpu().numpy(), out0.cpu().numpy())
    small.close()
    big.close()
