"""Plain FP64 CPU oracle of the DMN's linear elastic homogenization function and
of its offline-training objective (arXiv 2109.14403, Sec. 3.2).

TEST INFRASTRUCTURE ONLY: the test suite and the CPU-baseline leg of the
benchmark may use this module; the library never does.

  * eq. (laminate): the effective stiffness of one laminate solves
      (P(n) + lam [C - lam I]^-1)^-1 = c1 (P(n) + lam [C_1 - lam I]^-1)^-1
                                      + c2 (P(n) + lam [C_2 - lam I]^-1)^-1
    with the projector P(n) of eq. (P(n)) in Cartesian components, written out
    here in Mandel form; lam = 2 max eigenvalue of the two phase stiffnesses
    (the paper asks for a "sufficiently large" lam);
  * eq. (DMN^L): the input stiffnesses C_1, C_2 enter the bottom laminates
    pairwise (child 1: C_1, child 2: C_2) and the laminate stiffnesses are
    propagated to the root; c1 = W_1 / (W_1 + W_2) with W the sum of the leaf
    weights of a child's subtree (weight propagation of Sec. 3.1);
  * eq. (loss_function): J = (1/N_b) (sum_s e_s^q)^(1/q) + lam_pen (sum w - 1)^2,
    e_s = |C_bar^s - DMN^L(C_1^s, C_2^s)|_p / |C_bar^s|_p over the 36 Mandel
    components;
  * w = <v>_+ (ReLU of the unconstrained weights), and the lamination
    directions normalised before use (P(n) needs unit vectors);
  * gradients d J / d n and d J / d v by automatic differentiation, as the
    paper computes them (PyTorch, FP64, CPU).
Node order as the paper's: bottom level first, root last.
"""
from __future__ import annotations

import numpy as np
import torch

_SQ2 = 2.0 ** 0.5
_PAIRS = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
_WM = [1.0, 1.0, 1.0, _SQ2, _SQ2, _SQ2]


def _projector(n):
    """eq. (P(n)) as a 6x6 Mandel matrix (torch, differentiable in n)."""
    d = torch.eye(3, dtype=n.dtype)
    P4 = 0.5 * (torch.einsum("m,no,p->mnop", n, d, n) + torch.einsum("n,mo,p->mnop", n, d, n)
                + torch.einsum("m,np,o->mnop", n, d, n) + torch.einsum("n,mp,o->mnop", n, d, n)) \
        - torch.einsum("m,n,o,p->mnop", n, n, n, n)
    rows = []
    for I, (i, j) in enumerate(_PAIRS):
        rows.append(torch.stack([_WM[I] * _WM[J] * P4[i, j, k, l] for J, (k, l) in enumerate(_PAIRS)]))
    return torch.stack(rows)


def laminate(C1, C2, n, c1, lam):
    """eq. (laminate) solved for the effective stiffness (torch tensors)."""
    P = _projector(n)
    I6 = torch.eye(6, dtype=C1.dtype)

    def Y(C):
        return torch.linalg.inv(P + lam * torch.linalg.inv(C - lam * I6))
    Yb = c1 * Y(C1) + (1.0 - c1) * Y(C2)
    return lam * I6 + lam * torch.linalg.inv(torch.linalg.inv(Yb) - P)


def _forward_one(C1, C2, normals, w, lam):
    K = int(round(np.log2(w.shape[0])))
    Cl = [C1 if j % 2 == 0 else C2 for j in range(1 << K)]   # level K+1
    Wl = [w[j] for j in range(1 << K)]
    for k in range(K, 0, -1):
        Cn, Wn = [], []
        for i in range(1 << (k - 1)):
            p = (1 << K) - (1 << k) + i
            a, b = 2 * i, 2 * i + 1
            W = Wl[a] + Wl[b]
            c1 = Wl[a] / W
            nh = normals[p] / torch.linalg.norm(normals[p])
            Cn.append(laminate(Cl[a], Cl[b], nh, c1, lam))
            Wn.append(W)
        Cl, Wl = Cn, Wn
    return Cl[0]


def _lam(C1, C2):
    return 2.0 * max(float(np.linalg.eigvalsh(C1).max()), float(np.linalg.eigvalsh(C2).max()))


def forward(C1s, C2s, normals, v):
    """DMN^L for every sample: C1s, C2s [n, 6, 6] -> [n, 6, 6] (numpy, FP64)."""
    C1s = np.asarray(C1s, np.float64).reshape(-1, 6, 6)
    C2s = np.asarray(C2s, np.float64).reshape(-1, 6, 6)
    nt = torch.tensor(np.asarray(normals, np.float64).reshape(-1, 3))
    w = torch.clamp(torch.tensor(np.asarray(v, np.float64)), min=0.0)
    out = np.zeros_like(C1s)
    with torch.no_grad():
        for s in range(C1s.shape[0]):
            out[s] = _forward_one(torch.tensor(C1s[s]), torch.tensor(C2s[s]), nt, w,
                                  _lam(C1s[s], C2s[s])).numpy()
    return out


def _loss_torch(C1s, C2s, Ct, nt, vt, p, q, penalty):
    w = torch.clamp(vt, min=0.0)
    errs = []
    for s in range(C1s.shape[0]):
        D = _forward_one(torch.tensor(C1s[s]), torch.tensor(C2s[s]), nt, w, _lam(C1s[s], C2s[s]))
        T = torch.tensor(Ct[s])
        errs.append(torch.linalg.norm((T - D).reshape(-1), ord=p) / torch.linalg.norm(T.reshape(-1), ord=p))
    e = torch.stack(errs)
    data = torch.sum(e ** q) ** (1.0 / q) / C1s.shape[0]
    pen = penalty * (torch.sum(w) - 1.0) ** 2
    return data + pen, data, pen, e


def loss(C1s, C2s, Ctarget, normals, v, p=1.0, q=10.0, penalty=1e3):
    """eq. (loss_function): returns (J, data term, penalty term, e_s)."""
    C1s = np.asarray(C1s, np.float64).reshape(-1, 6, 6)
    C2s = np.asarray(C2s, np.float64).reshape(-1, 6, 6)
    Ct = np.asarray(Ctarget, np.float64).reshape(-1, 6, 6)
    with torch.no_grad():
        J, d, pe, e = _loss_torch(C1s, C2s, Ct, torch.tensor(np.asarray(normals, np.float64).reshape(-1, 3)),
                                  torch.tensor(np.asarray(v, np.float64)), p, q, penalty)
    return float(J), float(d), float(pe), e.numpy()


def loss_grad(C1s, C2s, Ctarget, normals, v, p=1.0, q=10.0, penalty=1e3):
    """J and its gradients d J / d normals [N, 3], d J / d v [2^K] by automatic
    differentiation."""
    C1s = np.asarray(C1s, np.float64).reshape(-1, 6, 6)
    C2s = np.asarray(C2s, np.float64).reshape(-1, 6, 6)
    Ct = np.asarray(Ctarget, np.float64).reshape(-1, 6, 6)
    nt = torch.tensor(np.asarray(normals, np.float64).reshape(-1, 3), requires_grad=True)
    vt = torch.tensor(np.asarray(v, np.float64), requires_grad=True)
    J, d, pe, e = _loss_torch(C1s, C2s, Ct, nt, vt, p, q, penalty)
    J.backward()
    return float(J.detach()), nt.grad.numpy().copy(), vt.grad.numpy().copy()
