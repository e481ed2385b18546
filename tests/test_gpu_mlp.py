"""Warm-start network on the GPU: the tcgen05 GEMM, gradients and forward pass
against the FP64 reference in oracle/mlp.py, training, and what the trained
network gains in the Newton solve."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2109_14403_gb300 import synthetic as syn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _bf16_round(a):
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).float().numpy().astype(np.float64)


# N a multiple of 256 takes the persistent wide form (one CTA per SM, tiles
# looped, two TMEM accumulators): one tile, fewer tiles than SMs, and the
# benchmark's shapes (thousands of tiles per CTA loop); other N the tile form
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 192), (128, 256, 64), (512, 768, 896),
                                   (2432, 512, 128), (65536, 512, 896), (65536, 512, 512),
                                   (65536, 768, 512)])
def test_gemm_matches_fp32_reference(M, N, K):
    from paper_2109_14403_gb300.mlp import gemm_bf16_tn
    dev = _dev()
    g = torch.Generator(device="cpu").manual_seed(M + N + K)
    a = torch.randn(M, K, generator=g).to(torch.bfloat16).to(dev)
    b = torch.randn(N, K, generator=g).to(torch.bfloat16).to(dev)
    c = gemm_bf16_tn(a, b)
    # products of bf16 values are exact in FP32; only the order and rounding
    # of the FP32 sums differ: each side is within K 2^-24 sum |a_ik b_jk| of
    # the exact sum for IEEE adds; the bound allows 4 times that (tensor-core
    # accumulation need not round to nearest at every add)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    ref = a.float() @ b.float().T
    mag = a.float().abs() @ b.float().abs().T
    torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.synchronize()
    bound = K * 2.0 ** -22 * mag + 1e-30
    assert ((c - ref).abs() <= bound).all().item(), ((c - ref).abs() / bound).max().item()


def _small_net(dev, seed=3):
    from paper_2109_14403_gb300.mlp import MLP
    net = MLP(K=2, hidden=128, n_hidden=2, max_batch=512, seed=seed)
    rng = np.random.default_rng(seed)
    p = np.zeros(net.n_params, np.float32)
    o = 0
    for li, (din, dout) in enumerate(net.layer_dims()):
        rows = net.n_out if li == len(net.layer_dims()) - 1 else dout
        cols = net.n_in if li == 0 else din
        W = np.zeros((dout, din), np.float32)
        W[:rows, :cols] = rng.normal(0, 1.0 / np.sqrt(cols), (rows, cols))
        b = np.zeros(dout, np.float32)
        b[:rows] = rng.normal(0, 0.1, rows)
        p[o:o + din * dout] = W.ravel()
        o += din * dout
        p[o:o + dout] = b
        o += dout
    net.set_params(p)
    return net, p, rng


def _inputs(net, rng, n, dev):
    x = np.zeros((n, net.n_in_pad), np.float32)
    x[:, :net.n_in] = rng.normal(size=(n, net.n_in))
    t = np.zeros((n, net.n_out_pad), np.float32)
    t[:, :net.n_out] = rng.normal(size=(n, net.n_out))
    xg = torch.tensor(x).to(torch.bfloat16).to(dev)
    return xg, torch.tensor(t, device=dev), _bf16_round(x), t


def _oracle_params(net, p):
    """bf16 weights (as the GPU multiplies them), fp32 biases."""
    q = p.astype(np.float64).copy()
    o = 0
    for din, dout in net.layer_dims():
        q[o:o + din * dout] = _bf16_round(p[o:o + din * dout])
        o += din * dout + dout
    return q


def test_gradients_match_fp64_reference():
    """Every gradient entry of a training step against the FP64 gradient of
    the same bf16 weights and inputs, within 6 standard deviations of what
    the bf16 roundings of activations and back-propagated gradients can do
    to that entry (oracle.mlp.grad_error_sigma; a few per mille of |g| at the
    median), plus an FP32 floor.  The loss to 1e-3."""
    dev = _dev()
    net, p, rng = _small_net(dev)
    n = 200  # ragged: padded to 256 rows inside
    xg, tg, x64, t64 = _inputs(net, rng, n, dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    net.train_step(xg, tg, 0.0, loss)
    torch.cuda.synchronize()
    g = net.grads().astype(np.float64)
    q = _oracle_params(net, p)
    L, gref = omlp.loss_and_grads(q, net.layer_dims(), x64, t64, net.n_out)
    sig = omlp.grad_error_sigma(q, net.layer_dims(), x64, t64, net.n_out)
    assert abs(loss.item() - L) <= 1e-3 * L
    o = 0
    for din, dout in net.layer_dims():
        for size in (din * dout, dout):
            a, b, sg = g[o:o + size], gref[o:o + size], sig[o:o + size]
            floor = 1e-6 * np.abs(b).max() + 1e-12
            assert (np.abs(a - b) <= 6.0 * sg + floor).all(), np.max(np.abs(a - b) / (6.0 * sg + floor))
            o += size
    net.close()


def test_amsgrad_kernel_matches_oracle_over_three_steps():
    """The FP32 optimiser kernel of the training step (dmn_mlp_amsgrad) against
    the FP64 AMSGrad step, element by element, over three steps on seeded
    parameters and gradients whose magnitudes span ten decades; the third
    step's gradients are small where the second's were large, so that many
    entries keep the running maximum (the AMSGrad branch).  Bound: a few FP32
    roundings of each quantity (m, v, vmax to 4 ulp; w to 4 ulp of w plus
    8 ulp of the step)."""
    from oracle import optim
    from paper_2109_14403_gb300.mlp import amsgrad
    dev = _dev()
    rng = np.random.default_rng(7)
    n = 100_003  # not a multiple of the block size
    b1, b2, eps, lr = np.float32(0.9), np.float32(0.999), np.float32(1e-8), np.float32(1e-3)
    w = rng.normal(size=n).astype(np.float32)
    mag = 10.0 ** rng.uniform(-8, 2, n)
    G = [rng.normal(size=n) * mag, rng.normal(size=n) * mag, rng.normal(size=n) * mag * 1e-3]
    G = [g.astype(np.float32) for g in G]
    W, Gd = torch.tensor(w, device=dev), torch.empty(n, dtype=torch.float32, device=dev)
    M, V, VM = (torch.zeros(n, dtype=torch.float32, device=dev) for _ in range(3))
    wr, mr, vr, vmr = w.astype(np.float64), np.zeros(n), np.zeros(n), np.zeros(n)
    ulp = 2.0 ** -23
    b1d, b2d = float(b1), float(b2)
    for t, g in enumerate(G, start=1):
        Gd.copy_(torch.tensor(g))
        amsgrad(W, Gd, M, V, VM, t, lr, b1, b2, eps)
        w_prev, m_prev, v_prev, vm_prev = wr.copy(), mr.copy(), vr.copy(), vmr.copy()
        wr, mr, vr, vmr = optim.amsgrad_step(wr, g, mr, vr, vmr, t, float(lr), b1d, b2d, float(eps))
        torch.cuda.synchronize()
        gd = g.astype(np.float64)
        # bounds relative to the operands: b1 m + (1-b1) g can cancel
        em = 4 * ulp * (b1d * np.abs(m_prev) + (1 - b1d) * np.abs(gd))
        ev = 4 * ulp * (b2d * v_prev + (1 - b2d) * gd * gd)
        got_m, got_v, got_vm = (x.cpu().numpy().astype(np.float64) for x in (M, V, VM))
        assert (np.abs(got_m - mr) <= em + 1e-38).all()
        assert (np.abs(got_v - vr) <= ev + 1e-38).all()
        assert (np.abs(got_vm - vmr) <= np.maximum(ev, 4 * ulp * vm_prev) + 1e-38).all()
        got_w = W.cpu().numpy().astype(np.float64)
        step = np.abs(wr - w_prev)
        bc1, bc2 = 1 - b1d ** t, 1 - b2d ** t
        den = np.sqrt(vmr / bc2) + float(eps)
        # the step carries m's error (through m / bc1), a few roundings of its
        # own and of the square root; w one rounding of the subtraction
        e_step = float(lr) * (em / bc1) / den + 8 * ulp * step
        assert (np.abs(got_w - wr) <= 2 * ulp * np.abs(w_prev) + e_step + 1e-38).all()
        # the comparison follows the GPU's own trajectory from here: both sides
        # continue from the same FP32 values
        wr = got_w
        mr, vr, vmr = (x.cpu().numpy().astype(np.float64) for x in (M, V, VM))
    assert np.mean(vmr > vr) > 0.5  # the running-maximum branch was exercised


def test_train_step_moments_and_update_match_oracle():
    """One training step from a known start: the optimiser state equals the
    FP64 AMSGrad step taken with the FP64 gradient, element by element, to
    the gradient's rounding bound (m = 0.1 g, v = vmax = 0.001 g^2), and every
    parameter whose gradient sign the bound settles moved by the oracle's
    update (lr g / (|g| + eps) after one bias-corrected step)."""
    from oracle import optim
    dev = _dev()
    net, p, rng = _small_net(dev, seed=9)
    n = 256
    xg, tg, x64, t64 = _inputs(net, rng, n, dev)
    lr = 1e-3
    net.train_step(xg, tg, lr)
    torch.cuda.synchronize()
    q = _oracle_params(net, p)
    _, gref = omlp.loss_and_grads(q, net.layer_dims(), x64, t64, net.n_out)
    tol = 6.0 * omlp.grad_error_sigma(q, net.layer_dims(), x64, t64, net.n_out) + 1e-6 * np.abs(gref).max()
    z = np.zeros_like(gref)
    w1, m1, v1, vm1 = optim.amsgrad_step(p.astype(np.float64), gref, z, z, z, 1, lr,
                                         float(np.float32(0.9)), float(np.float32(0.999)), 1e-8)
    m, v, vm = (a.astype(np.float64) for a in net.moments())
    b1f, b2f = float(np.float32(0.9)), float(np.float32(0.999))
    assert (np.abs(m - m1) <= (1 - b1f) * tol + 1e-6 * np.abs(m1)).all()
    vtol = (1 - b2f) * (2 * np.abs(gref) * tol + tol * tol) + 1e-6 * v1
    assert (np.abs(v - v1) <= vtol).all() and (np.abs(vm - vm1) <= vtol).all()
    settled = np.abs(gref) > 2 * tol + 1e-7
    assert settled.sum() > 0.5 * (gref != 0).sum()  # padding entries have g = 0 exactly
    w = net.params().astype(np.float64)
    np.testing.assert_allclose(w[settled], w1[settled], rtol=0, atol=1e-6 * lr + 1e-6 * np.abs(w1[settled]).max())
    # any first step moves a parameter by at most lr; padding does not move
    assert (np.abs(w - p) <= lr * (1 + 1e-5)).all()
    assert (w[gref == 0] == p[gref == 0]).all()
    net.close()


def test_forward_matches_fp64_reference():
    dev = _dev()
    net, p, rng = _small_net(dev, seed=5)
    n = 300
    xg, _, x64, _ = _inputs(net, rng, n, dev)
    y = net.predict(xg).cpu().numpy()  # default normalisation: identity
    hs, _ = omlp.forward(omlp.unpack(_oracle_params(net, p), net.layer_dims()), x64)
    ref = hs[-1][:, :net.n_out]
    assert np.abs(y - ref).max() <= 2e-2 * np.abs(ref).max()
    net.close()


def test_training_reduces_the_loss():
    from paper_2109_14403_gb300.mlp import MLP
    dev = _dev()
    net = MLP(K=2, hidden=128, n_hidden=2, max_batch=1024, seed=1)
    rng = np.random.default_rng(2)
    n = 1024
    x = np.zeros((n, net.n_in_pad), np.float32)
    x[:, :net.n_in] = rng.normal(size=(n, net.n_in))
    R = rng.normal(0, 0.3, (net.n_in, net.n_out))
    t = np.zeros((n, net.n_out_pad), np.float32)
    t[:, :net.n_out] = np.tanh(x[:, :net.n_in] @ R)
    xg = torch.tensor(x).to(torch.bfloat16).to(dev)
    tg = torch.tensor(t, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    net.train_step(xg, tg, 0.0, loss)
    l0 = loss.item()
    for _ in range(300):
        net.train_step(xg, tg, 3e-3, loss)
    torch.cuda.synchronize()
    assert loss.item() < 0.1 * l0
    net.close()


def test_warm_start_gain_on_the_k8_random_walk():
    """Pairs from the plain FP64 solver on the K=8 random walk train the
    network; on later, held-out increments the warm-started mixed solve
    (tol 1e-12, the paper's tolerance) must stay within 2e-8 of the FP64
    solution (tol 1e-13), like the plain mixed solve, and take fewer Newton
    iterations."""
    from paper_2109_14403_gb300 import DMN
    from paper_2109_14403_gb300.mlp import MLP
    dev = _dev()
    K, n, n_train, n_eval = 8, 16384, 10, 3
    w, nrm, ph = syn.tree(K)
    mats = syn.materials()
    deps, theta = syn.random_walk_k8(n_points=n, n_incr=n_train + n_eval, seed=11)
    D = torch.tensor(deps, device=dev)
    T = torch.tensor(theta, device=dev)
    plain = DMN(K, w, nrm, ph, mats, precision="fp64", tol=1e-13)
    net = MLP(K=K, hidden=512, n_hidden=3, max_batch=n, seed=0)
    s_prev = None
    s = plain.init_state(torch.full((n,), 293.0, dtype=torch.float64, device=dev))
    feats, tgts, hist = [], [], []
    for k in range(n_train + n_eval):
        s1, out, st, it = plain.eval(D[k], T[k], 1.0, s)
        if k < n_train:
            feats.append(net.features(D[k], T[k], s, s_prev))
            tgts.append(net.targets(s, s1))
        hist.append((s_prev, s, out.cpu().numpy()[:, :6]))
        s_prev, s = s, s1
    F = torch.cat(feats)
    Tg = torch.cat(tgts)
    net.fit_normalization(F, Tg)
    X = net.normalize_features(F)
    Y = net.normalize_targets(Tg)
    perm = torch.randperm(X.shape[0], device=dev, generator=torch.Generator(device=dev).manual_seed(0))
    X, Y = X[perm].contiguous(), Y[perm].contiguous()
    B = 4096
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    for ep in range(12):
        for i in range(0, X.shape[0] - B + 1, B):
            net.train_step(X[i:i + B], Y[i:i + B], 1e-3 if ep < 8 else 2e-4, loss)
    torch.cuda.synchronize()
    assert loss.item() < 0.01  # normalised MSE
    mixed = DMN(K, w, nrm, ph, mats, precision="mixed", tol=1e-12)
    it_plain, it_warm, fallbacks = [], [], 0
    for k in range(n_train, n_train + n_eval):
        sp, si, ref = hist[k]
        x1 = net.normalize_features(net.features(D[k], T[k], si, sp))
        x2 = net.input(D[k], T[k], si, sp)  # fused path used in the solve loop
        assert torch.equal(x1, x2)
        da = net.predict(x2)
        _, op, stp, itp = mixed.eval(D[k], T[k], 1.0, si)
        _, ow, stw, itw = mixed.eval_warm(D[k], T[k], 1.0, si, da)
        torch.cuda.synchronize()
        assert (stp.cpu() == 0).all() and ((stw.cpu() & 3) == 0).all()
        fallbacks += int(((stw.cpu() & 4) != 0).sum())
        for o in (op, ow):
            g = o.cpu().numpy()[:, :6]
            assert (np.linalg.norm(g - ref, axis=1) / np.linalg.norm(ref, axis=1)).max() < 2e-8
        it_plain.append(itp.cpu().numpy())
        it_warm.append(itw.cpu().numpy())
    ip, iw = np.concatenate(it_plain), np.concatenate(it_warm)
    print(f"\nwarm start: mean Newton iterations {ip.mean():.4f} -> {iw.mean():.4f}, "
          f"points needing >1 iteration {np.mean(ip > 1):.4f} -> {np.mean(iw > 1):.4f}, "
          f"fallback rate {fallbacks / ip.size:.5f}")
    assert iw.mean() < 0.8 * ip.mean()
    assert fallbacks / ip.size < 0.01
    plain.close()
    mixed.close()
    net.close()


def test_warm_start_k9_perzyna():
    """K = 9 with the Perzyna matrix (1541 network inputs, 1533 outputs): the
    network trained on FP64 pairs warm-starts the mixed solve, which stays
    within the stopping-criterion bound of the FP64 solution (tol 1e-13) and
    takes no more Newton iterations than the plain start.  Algorithm 1 stops
    at |r| < tol N |sigma_bar|, N = 511 here, so the stress can be off by about
    tol N (stiffness contrast ~30) = 1.5e-8; the bound allows a factor 4."""
    from paper_2109_14403_gb300 import DMN
    from paper_2109_14403_gb300.mlp import MLP
    dev = _dev()
    K, n, n_train = 9, 8192, 5
    w, nrm, ph = syn.tree(K)
    mats = syn.materials_viscoplastic()
    deps, theta = syn.large_path(n_points=n, n_incr=n_train + 1, seed=12)
    deps *= 30.0  # strain rates large enough for viscoplastic flow
    D = torch.tensor(deps, device=dev)
    T = torch.tensor(theta, device=dev)
    dt = syn.LARGE_DT
    plain = DMN(K, w, nrm, ph, mats, precision="fp64", tol=1e-13)
    net = MLP(K=K, hidden=256, n_hidden=2, max_batch=n, seed=0)
    assert net.n_in == 8 + 3 * 511 and net.n_out == 3 * 511
    s_prev, s = None, plain.init_state(torch.full((n,), 293.0, dtype=torch.float64, device=dev))
    feats, tgts = [], []
    for k in range(n_train):
        s1, _, _, _ = plain.eval(D[k], T[k], dt, s)
        feats.append(net.features(D[k], T[k], s, s_prev))
        tgts.append(net.targets(s, s1))
        s_prev, s = s, s1
    F, Tg = torch.cat(feats), torch.cat(tgts)
    net.fit_normalization(F, Tg)
    X, Y = net.normalize_features(F), net.normalize_targets(Tg)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    for ep in range(20):
        for i in range(0, X.shape[0] - 2048 + 1, 2048):
            net.train_step(X[i:i + 2048], Y[i:i + 2048], 1e-3, loss)
    k = n_train
    _, ref, st_r, _ = plain.eval(D[k], T[k], dt, s)
    mixed = DMN(K, w, nrm, ph, mats, precision="mixed", tol=1e-12)
    da = net.predict(net.input(D[k], T[k], s, s_prev))
    _, op, stp, itp = mixed.eval(D[k], T[k], dt, s)
    _, ow, stw, itw = mixed.eval_warm(D[k], T[k], dt, s, da)
    torch.cuda.synchronize()
    assert (st_r.cpu() == 0).all() and (stp.cpu() == 0).all() and ((stw.cpu() & 3) == 0).all()
    r = ref.cpu().numpy()[:, :6]
    bound = 4 * 1e-12 * 511 * 30
    for o in (op, ow):
        g = o.cpu().numpy()[:, :6]
        assert (np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1)).max() < bound
    ip, iw = itp.cpu().numpy(), itw.cpu().numpy()
    print(f"\nK=9 warm start: mean Newton iterations {ip.mean():.3f} -> {iw.mean():.3f}")
    assert iw.mean() <= ip.mean()
    plain.close()
    mixed.close()
    net.close()


def test_features_match_the_state():
    """The network's raw features against their definition, computed here
    from the same device states: the load step rounded to FP32, and
    a^n - a^{n-1} as the FP32 difference of the two words rounded to FP32
    (round to nearest even, as numpy's astype); without a previous state the
    difference columns are 0."""
    from paper_2109_14403_gb300 import DMN
    from paper_2109_14403_gb300.mlp import MLP
    dev = _dev()
    K, n = 4, 300
    w, nrm, ph = syn.tree(K)
    d = DMN(K, w, nrm, ph, syn.materials(), tol=1e-12)
    deps, theta = syn.ramp_k4(n_points=n, n_incr=3)
    s0 = d.init_state(torch.full((n,), 293.0, dtype=torch.float64, device=dev))
    s1, _, _, _ = d.eval(torch.tensor(deps[0], device=dev), torch.tensor(theta[0], device=dev), 1.0, s0)
    s2, _, _, _ = d.eval(torch.tensor(deps[1], device=dev), torch.tensor(theta[1], device=dev), 1.0, s1)
    net = MLP(K=K, hidden=128, n_hidden=1, max_batch=n, seed=0)
    D, T = torch.tensor(deps[2], device=dev), torch.tensor(theta[2], device=dev)
    f = net.features(D, T, s2, s1).cpu().numpy()
    f0 = net.features(D, T, s2, None).cpu().numpy()
    a, ap = s2.cpu().numpy(), s1.cpu().numpy()
    n3 = 3 * ((1 << K) - 1)
    ref = np.concatenate([np.asarray(deps[2]).astype(np.float32), theta[2][:, None].astype(np.float32),
                          (theta[2] - a[:, 6])[:, None].astype(np.float32),
                          a[:, 8:8 + n3].astype(np.float32) - ap[:, 8:8 + n3].astype(np.float32)], axis=1)
    assert f.shape == (n, net.n_in) == ref.shape
    np.testing.assert_array_equal(f, ref)
    ref[:, 8:] = 0.0
    np.testing.assert_array_equal(f0, ref)
    net.close()
    d.close()
