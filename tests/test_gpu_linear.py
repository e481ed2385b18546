"""The linear homogenization function DMN^L and the gradient of the
offline-training loss on the GPU (``dmn_linear_*`` through the C ABI) against
the oracle (Milton's laminate formula, automatic differentiation in FP64).

Tolerances.  FP64 kernels: the condensed laminate and Milton's formula agree to
rounding, amplified by the conditioning of the 3x3 jump systems (stiffness
contrast up to 100 here): 1e-10 relative for DMN^L, 1e-8 for J and the
gradients (which add the 1/|C|_p and max-normalised q-norm steps).  FP32
kernels: 2^-24 per operation, K levels deep, times the same conditioning:
2e-4 for DMN^L and J, 5e-3 for the gradients (relative to their largest entry).
"""
import numpy as np
import pytest

import oracle.linear as olin
from paper_2109_14403_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(fwd=1e-10, loss=1e-8, grad=1e-8), "fp32": dict(fwd=2e-4, loss=2e-4, grad=5e-3)}


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=_dev())


@pytest.mark.parametrize("K,n", [(1, 33), (3, 17), (5, 9), (8, 3)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_forward_parity(K, n, prec):
    from paper_2109_14403_gb300.linear import DMNLinear
    normals, v = syn.linear_params(K, seed=K)
    C1, C2 = syn.stiffness_pairs(n, seed=10 + K)
    d = DMNLinear(K, normals, v, device=_dev())
    out = d.forward(_t(C1), _t(C2), precision=prec).cpu().numpy()
    ref = olin.forward(C1, C2, normals, v)
    err = np.linalg.norm((out - ref).reshape(n, -1), axis=1) / np.linalg.norm(ref.reshape(n, -1), axis=1)
    assert err.max() < TOL[prec]["fwd"], err.max()


@pytest.mark.parametrize("K,p,q", [(2, 1.0, 10.0), (3, 1.0, 10.0), (4, 2.0, 2.0)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_loss_and_gradient_parity(K, p, q, prec):
    from paper_2109_14403_gb300.linear import DMNLinear
    normals, v = syn.linear_params(K, seed=20 + K)
    v = v.copy()
    v[1] = -0.03  # a dead leaf
    tn, tv = syn.linear_params(K, seed=40 + K)
    n = 12
    C1, C2 = syn.stiffness_pairs(n, seed=30 + K)
    Ct = olin.forward(C1, C2, tn, tv)
    J, gn, gv = olin.loss_grad(C1, C2, Ct, normals, v, p=p, q=q, penalty=10.0)
    d = DMNLinear(K, normals, v, device=_dev())
    loss = d.loss_grad(_t(C1), _t(C2), _t(Ct), p=p, q=q, penalty=10.0, precision=prec).cpu().numpy()
    g = d.grad.cpu().numpy()
    t = TOL[prec]
    assert abs(loss[0] - J) <= t["loss"] * abs(J)
    gscale = max(np.abs(gn).max(), np.abs(gv).max())
    assert np.abs(g[:3 * d.N].reshape(-1, 3) - gn).max() <= t["grad"] * gscale
    assert np.abs(g[3 * d.N:] - gv).max() <= t["grad"] * gscale
    assert g[3 * d.N + 1] == 0.0


def test_training_reduces_the_loss():
    """A depth-3 DMN^L fitted by AMSGrad to the stiffnesses of another one
    (targets from the oracle): the loss falls by an order of magnitude."""
    from paper_2109_14403_gb300.linear import DMNLinear
    K = 3
    tn, tv = syn.linear_params(K, seed=77)
    C1, C2 = syn.stiffness_pairs(256, seed=78, log10_contrast=1.0)
    Ct = olin.forward(C1, C2, tn, tv)
    normals, v = syn.linear_params(K, seed=79)
    d = DMNLinear(K, normals, v, device=_dev())
    c1, c2, ct = _t(C1), _t(C2), _t(Ct)
    first = float(d.loss_grad(c1, c2, ct, p=1.0, q=2.0, penalty=10.0)[0].item())
    for it in range(400):
        d.loss_grad(c1, c2, ct, p=1.0, q=2.0, penalty=10.0)
        d.amsgrad_step(2e-2, 2e-3)
    last = float(d.loss_grad(c1, c2, ct, p=1.0, q=2.0, penalty=10.0)[0].item())
    assert np.isfinite(last) and last < 0.1 * first, (first, last)


def test_argument_errors():
    from paper_2109_14403_gb300 import dmn
    from paper_2109_14403_gb300.linear import DMNLinear
    d = DMNLinear(2, *syn.linear_params(2), device=_dev())
    C1, C2 = syn.stiffness_pairs(2)
    with pytest.raises(RuntimeError, match="p, q"):
        d.loss_grad(_t(C1), _t(C2), _t(C1), p=0.5)
    L = dmn.load()
    assert L.dmn_linear_forward(None, 9, 1, 1, 1, 1, 1, 1, 0) == 1 and b"K must be" in L.dmn_last_error()
    assert L.dmn_linear_forward(None, 2, 0, None, None, None, None, None, 7) == 1
    assert b"precision" in L.dmn_last_error()
    assert L.dmn_linear_amsgrad(None, 4, 1, 1, 1, 1, 1, 0.1, 0.9, 0.999, 1e-8, 0) == 1


def test_full_batch_forward_sampled_and_directional_gradient():
    """The benchmark's size (K = 8, 65,536 samples): DMN^L of four sampled
    samples against the oracle, and the FP64 gradient against a central
    difference of the FP64 loss along a random direction of all parameters
    (a property that holds at any batch size)."""
    from paper_2109_14403_gb300.linear import DMNLinear
    K, n = 8, 65536
    C1h, C2h = syn.stiffness_pairs(n, seed=7)
    c1, c2 = _t(C1h), _t(C2h)
    teacher = DMNLinear(K, *syn.linear_params(K, seed=101), device=_dev())
    ct = teacher.forward(c1, c2, precision="fp64")
    normals, v = syn.linear_params(K, seed=102)
    d = DMNLinear(K, normals, v, device=_dev())
    out = d.forward(c1, c2, precision="fp32").cpu().numpy()
    idx = [0, 12345, 40000, n - 1]
    ref = olin.forward(C1h[idx], C2h[idx], normals, v)
    err = np.linalg.norm((out[idx] - ref).reshape(4, -1), axis=1) / np.linalg.norm(ref.reshape(4, -1), axis=1)
    assert err.max() < TOL["fp32"]["fwd"]
    d.loss_grad(c1, c2, ct, p=1.0, q=10.0, penalty=1e3, precision="fp64")
    g = d.grad.clone()
    rng = np.random.default_rng(5)
    direction = torch.tensor(rng.standard_normal(d.params.numel()), device=_dev())
    direction[3 * d.N:] *= 1e-2  # weights are O(1/2^K)
    x0 = d.params.clone()
    h = 1e-6
    vals = []
    for sgn in (1.0, -1.0):
        d.params.copy_(x0 + sgn * h * direction)
        vals.append(float(d.loss_grad(c1, c2, ct, p=1.0, q=10.0, penalty=1e3, precision="fp64")[0].item()))
    d.params.copy_(x0)
    fd = (vals[0] - vals[1]) / (2 * h)
    an = float((g * direction).sum().item())
    assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-6), (fd, an)


def test_minibatch_training_with_the_paper_schedule():
    """Mini-batches of 32 with the paper's learning-rate modulation (p = 1,
    q = 10, penalty 1e3 as in its Sec. 5.3): the mean error e_mean of a depth-3
    network fitted to another one falls by a factor of ten, and e_mean on the
    GPU equals the oracle's for the same parameters."""
    from paper_2109_14403_gb300.linear import DMNLinear, mean_error, train
    K = 3
    tn, tv = syn.linear_params(K, seed=77)
    C1, C2 = syn.stiffness_pairs(512, seed=78, log10_contrast=1.0)
    Ct = olin.forward(C1, C2, tn, tv)
    normals, v = syn.linear_params(K, seed=79)
    d = DMNLinear(K, normals, v, device=_dev())
    c1, c2, ct = _t(C1), _t(C2), _t(Ct)
    e0 = mean_error(d, c1, c2, ct)
    o_err = olin.loss(C1, C2, Ct, normals, v, p=1.0, q=1.0, penalty=0.0)[1]
    assert abs(e0 - o_err) <= 1e-9 * o_err
    train(d, c1, c2, ct, epochs=40, batch=32, precision="fp64")
    e1 = mean_error(d, c1, c2, ct)
    assert e1 < 0.1 * e0, (e0, e1)


@pytest.mark.parametrize("K", [3, 8])
def test_trained_parameters_drive_the_online_evaluation(K):
    """Offline to online (the paper's workflow): a DMN^L parameter set used by
    dmn_create gives, for linear elastic phases, an algorithmic tangent of
    Algorithm 1 equal to DMN^L of the same phase stiffnesses."""
    from paper_2109_14403_gb300 import DMN
    from paper_2109_14403_gb300.linear import DMNLinear
    dev = _dev()
    normals, v = syn.linear_params(K, seed=55)
    w = np.maximum(v, 0.0)
    w = w / w.sum()
    mats = syn.materials().copy()
    mats[1, 5] = 1e12  # the matrix never yields
    C1 = syn.iso_mandel(mats[0, 1], mats[0, 2])
    C2 = syn.iso_mandel(mats[1, 1], mats[1, 2])
    lin = DMNLinear(K, normals, w, device=dev)
    ref = lin.forward(_t(C1[None]), _t(C2[None]), precision="fp64").cpu().numpy()[0]
    phase = (np.arange(1 << K) % 2).astype(np.uint8)  # leaf 2i: phase 1, leaf 2i+1: phase 2
    d = DMN(K, w, normals, phase, mats, tol=1e-12, precision="fp64")
    s = d.init_state(torch.full((1,), mats[0, 4], dtype=torch.float64, device=dev))
    _, out, st, _ = d.eval(_t(np.full((1, 6), 1e-5)), _t(np.full(1, mats[0, 4])), 1.0, s)
    C = out.cpu().numpy()[0, 6:42].reshape(6, 6)
    assert st.cpu().numpy()[0] == 0
    assert np.abs(C - ref).max() <= 1e-10 * np.abs(ref).max()
    d.close()


def test_linear_amsgrad_matches_oracle_over_three_steps():
    """dmn_linear_amsgrad (FP64) against the FP64 AMSGrad step, element by
    element, over three steps on seeded parameters and gradients; the third
    step's gradients are small, so most entries keep the running maximum."""
    import ctypes
    from oracle import optim
    from paper_2109_14403_gb300 import dmn
    dev = _dev()
    lib = dmn.load()
    rng = np.random.default_rng(8)
    n = 5_001
    mag = 10.0 ** rng.uniform(-6, 1, n)
    G = [rng.normal(size=n) * mag, rng.normal(size=n) * mag, rng.normal(size=n) * mag * 1e-3]
    w0 = rng.normal(size=n)
    X, Gd = torch.tensor(w0, device=dev), torch.empty(n, dtype=torch.float64, device=dev)
    M, S, SM = (torch.zeros(n, dtype=torch.float64, device=dev) for _ in range(3))
    wr, mr, sr, smr = w0.copy(), np.zeros(n), np.zeros(n), np.zeros(n)
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for t, g in enumerate(G, start=1):
        Gd.copy_(torch.tensor(g))
        rc = lib.dmn_linear_amsgrad(stream, n, P(X), P(Gd), P(M), P(S), P(SM), 2e-3, 0.9, 0.999, 1e-8, t)
        assert rc == dmn.DMN_OK, lib.dmn_last_error().decode()
        wr, mr, sr, smr = optim.amsgrad_step(wr, g, mr, sr, smr, t, 2e-3, 0.9, 0.999, 1e-8)
        torch.cuda.synchronize()
        # FP64 on both sides; the kernel may fuse a multiply-add that numpy
        # rounds twice, so a few ulp per step (w: of its O(1) scale)
        np.testing.assert_allclose(X.cpu().numpy(), wr, rtol=1e-14, atol=1e-15)
        for got, ref in ((M, mr), (S, sr), (SM, smr)):
            np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=1e-13, atol=1e-300)
    assert np.mean(smr > sr) > 0.5
