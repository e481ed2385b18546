"""Plain FP64 CPU oracle of the online DMN evaluation (arXiv 2109.14403, Sec. 3.3,
Algorithm 1) plus an FP64 reference of the warm-start MLP.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library under
``paper_2109_14403_gb300`` never does.  The C source (``dmn_oracle.c``) is
compiled with gcc on first use (or by ``build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

OUT_WORDS = 57
PT_OK, PT_NOT_CONVERGED, PT_NONFINITE = 0, 1, 2
# material row: kinds 0-2: kind E nu alpha theta0 sy0 dsy_dT H m t_visc dE_dT 0 (rows of 8
# or 12 are padded); kind 3 (PA66): kind E_inf nu alpha0 theta0 sy0 k n m eta0 beta1 beta2
# theta_ref C1 C2 0, E_1..E_12, tau_1..tau_12
MAT_WORDS = 40
Z_WORDS = {0: 0, 1: 7, 2: 13, 3: 79}  # internal variables per leaf, by material kind
Z_MAX = 79


def mat_rows(mats):
    """Material table as n x 40 rows; shorter rows (kinds 0-2) are padded with 0."""
    m = np.atleast_2d(np.asarray(mats, np.float64))
    if m.shape[1] < MAT_WORDS:
        m = np.hstack([m, np.zeros((m.shape[0], MAT_WORDS - m.shape[1]))])
    return np.ascontiguousarray(m[:, :MAT_WORDS], dtype=np.float64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
            p = ctypes.c_void_p
            lib.oracle_state_words.restype = i64
            lib.oracle_state_words.argtypes = [i, p, p, p, p, i]
            lib.oracle_eval_batch.restype = i
            lib.oracle_eval_batch.argtypes = [i, p, p, p, p, i, d, i, i, d, d, i, i64, p, p, d,
                                              p, p, p, p, p, i]
            lib.oracle_eval_point_trace.restype = i
            lib.oracle_eval_point_trace.argtypes = [i, p, p, p, p, i, d, i, i, d, d, i, p, d, d,
                                                    p, p, p, p, p, p, i]
            lib.oracle_leaf.restype = None
            lib.oracle_leaf.argtypes = [p, p, d, p, d, d, p]
            lib.oracle_leaf_strains.restype = i
            lib.oracle_leaf_strains.argtypes = [i, p, p, p, p, p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Tree:
    """DMN description: depth K, leaf weights (2^K), normals ((2^K-1) x 3 in the
    paper's order: bottom level first, root last), phase map (2^K) and a material
    table (n_mats x 40 rows as in ``mat_rows``)."""

    def __init__(self, K, w, normals, phase, mats):
        self.K = int(K)
        self.w = _c(w, np.float64)
        self.normals = _c(normals, np.float64).reshape(-1, 3)
        self.phase = _c(phase, np.uint8)
        self.mats = mat_rows(mats)
        n = _load().oracle_state_words(self.K, _ptr(self.w), _ptr(self.normals), _ptr(self.phase),
                                       _ptr(self.mats), self.mats.shape[0])
        if n < 0:
            raise ValueError(f"oracle rejected the tree (code {n})")
        self.state_words = int(n)
        self.nnode = (1 << self.K) - 1

    def init_state(self, n_points, theta0):
        s = np.zeros((n_points, self.state_words), np.float64)
        s[:, 6] = theta0
        return s


def eval_batch(tree: Tree, deps, theta, dt, state_in, *, tol=1e-12, maxit=50, maxbacktrack=8,
               gamma=0.5, res_floor=None, dense=False, threads=None):
    """Algorithm 1 at every point.  Returns (state_out, out[n,57], status, iters)."""
    deps = _c(deps, np.float64).reshape(-1, 6)
    n = deps.shape[0]
    theta = _c(np.broadcast_to(np.asarray(theta, np.float64), (n,)), np.float64)
    sin = _c(state_in, np.float64).reshape(n, tree.state_words)
    sout = np.zeros_like(sin)
    out = np.zeros((n, OUT_WORDS), np.float64)
    status = np.zeros(n, np.int32)
    iters = np.zeros(n, np.int32)
    if res_floor is None:
        res_floor = 1e-8 * float(tree.mats[:, 1].max())
    if threads is None:
        threads = os.cpu_count() or 1
    rc = _load().oracle_eval_batch(tree.K, _ptr(tree.w), _ptr(tree.normals), _ptr(tree.phase),
                                   _ptr(tree.mats), tree.mats.shape[0], tol, maxit, maxbacktrack,
                                   gamma, res_floor, int(bool(dense)), n, _ptr(deps), _ptr(theta),
                                   float(dt), _ptr(sin), _ptr(sout), _ptr(out), _ptr(status),
                                   _ptr(iters), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_eval_batch failed (code {rc})")
    return sout, out, status, iters


def eval_point_trace(tree: Tree, deps, theta, dt, state_in, *, tol=1e-12, maxit=50,
                     maxbacktrack=8, gamma=0.5, res_floor=None, dense=False):
    """One point; also returns the residual history of Algorithm 1."""
    deps = _c(deps, np.float64).reshape(6)
    sin = _c(state_in, np.float64).reshape(tree.state_words)
    sout = np.zeros_like(sin)
    out = np.zeros(OUT_WORDS, np.float64)
    st = np.zeros(1, np.int32)
    it = np.zeros(1, np.int32)
    hist = np.full(maxit + 1, np.nan)
    if res_floor is None:
        res_floor = 1e-8 * float(tree.mats[:, 1].max())
    rc = _load().oracle_eval_point_trace(tree.K, _ptr(tree.w), _ptr(tree.normals),
                                         _ptr(tree.phase), _ptr(tree.mats), tree.mats.shape[0],
                                         tol, maxit, maxbacktrack, gamma, res_floor,
                                         int(bool(dense)), _ptr(deps), float(theta), float(dt),
                                         _ptr(sin), _ptr(sout), _ptr(out), _ptr(st), _ptr(it),
                                         _ptr(hist), maxit + 1)
    if rc != 0:
        raise ValueError(f"oracle_eval_point_trace failed (code {rc})")
    return sout, out, int(st[0]), int(it[0]), hist[~np.isnan(hist)]


def leaf(mat_row, eps, theta, zn=None, trn=0.0, dt=1.0):
    """One phase-law evaluation.  Returns a dict with sig, C, tau, D, d, g, diss, znew."""
    m = mat_rows(mat_row).reshape(MAT_WORDS)
    e = _c(eps, np.float64).reshape(6)
    z = np.zeros(Z_MAX, np.float64)
    if zn is not None:
        zn = np.asarray(zn, np.float64).ravel()
        z[:zn.size] = zn
    o = np.zeros(57 + Z_MAX, np.float64)
    _load().oracle_leaf(_ptr(m), _ptr(e), float(theta), _ptr(z), float(trn), float(dt), _ptr(o))
    return {"sig": o[0:6].copy(), "C": o[6:42].reshape(6, 6).copy(), "tau": o[42:48].copy(),
            "D": float(o[48]), "d": o[49:55].copy(), "g": float(o[55]), "diss": float(o[56]),
            "znew": o[57:57 + max(Z_WORDS[int(m[0])], 7)].copy()}


def leaf_strains(tree: Tree, eps_bar, a):
    """eps_j = eps_bar + A a for every leaf j (explicit kinematic operator)."""
    eb = _c(eps_bar, np.float64).reshape(6)
    av = _c(a, np.float64).reshape(3 * tree.nnode)
    out = np.zeros((1 << tree.K, 6), np.float64)
    rc = _load().oracle_leaf_strains(tree.K, _ptr(tree.w), _ptr(tree.normals), _ptr(eb),
                                     _ptr(av), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_leaf_strains failed")
    return out


def split_out(out):
    """Named views of the 57 output words."""
    out = np.asarray(out)
    return {"sig": out[..., 0:6], "C": out[..., 6:42].reshape(out.shape[:-1] + (6, 6)),
            "C_theta": out[..., 42:48], "D": out[..., 48], "D_eps": out[..., 49:55],
            "D_theta": out[..., 55], "diss": out[..., 56]}


def eval_mixed(tree: Tree, mask, target, deps, theta, dt, c_heat, state_in, *, max_outer=20,
               tol_outer=1e-10, tol=1e-12, threads=None, out_prev=None):
    """One increment under mixed control, by a plain outer Newton on eval_batch.

    Per point, bit c (0..5) of ``mask`` prescribes the Mandel stress component
    sigma_bar_c = target_c instead of the strain increment deps_c = target_c;
    bit 6 replaces the prescribed theta^{n+1} by the implicit-Euler form of the
    macroscopic heat equation (Sec. 2, eq. macro_heat) without heat source and
    flux (adiabatic): c_heat (theta^{n+1} - theta^n) / dt = D_bar.  The
    unknowns are solved with the algorithmic tangents d sigma_bar / d eps_bar,
    d sigma_bar / d theta, d D_bar / d eps_bar and d D_bar / d theta (Sec. 3.3)
    and numpy.linalg.solve.  ``deps`` and ``theta`` are starting values; with
    ``out_prev`` (the outputs of the increment that ended in ``state_in``) the
    start is instead the solution of the linearisation at that state,
    sigma_bar ~ sigma_bar^n + C deps + C_theta (theta - theta^n) and
    D_bar ~ D_eps . deps + D_theta (theta - theta^n).
    Returns (deps, theta, state_out, out, status, outer): status 8 = the
    conditions were not met within max_outer evaluations.
    """
    mask = np.asarray(mask, np.uint8).ravel()
    n = mask.size
    target = np.asarray(target, np.float64).reshape(n, 6)
    x_eps = np.array(deps, np.float64).reshape(n, 6)
    x_th = np.array(np.broadcast_to(np.asarray(theta, np.float64), (n,)))
    sin = np.asarray(state_in, np.float64).reshape(n, tree.state_words)
    theta_n = sin[:, 6]
    for c in range(6):
        strain = ((mask >> c) & 1) == 0
        x_eps[strain, c] = target[strain, c]
    if out_prev is not None:
        op = np.asarray(out_prev, np.float64).reshape(n, OUT_WORDS)
        for i in range(n):
            stress = [c for c in range(6) if (mask[i] >> c) & 1]
            adiabatic = bool((mask[i] >> 6) & 1)
            if not stress and not adiabatic:
                continue
            # linear model: unknowns u = (stress components' deps, theta - theta^n)
            C, C_th, D_eps, D_th = op[i, 6:42].reshape(6, 6), op[i, 42:48], op[i, 49:55], op[i, 55]
            known = np.array([0.0 if c in stress else x_eps[i, c] for c in range(6)])
            dth = 0.0 if adiabatic else x_th[i] - theta_n[i]
            rows, rhs = [], []
            for c in stress:
                rows.append([C[c, e] for e in stress] + ([C_th[c]] if adiabatic else []))
                rhs.append(target[i, c] - op[i, c] - C[c] @ known - C_th[c] * dth)
            if adiabatic:
                rows.append([-D_eps[e] for e in stress] + [c_heat / dt - D_th])
                rhs.append(D_eps @ known)
            u = np.linalg.solve(np.array(rows), np.array(rhs))
            for a, c in enumerate(stress):
                x_eps[i, c] = u[a]
            if adiabatic:
                x_th[i] = theta_n[i] + u[-1]
    outer = np.zeros(n, np.int32)
    failed = np.zeros(n, bool)
    open_ = np.ones(n, bool)
    sout = np.zeros_like(sin)
    out = np.zeros((n, OUT_WORDS))
    st = np.zeros(n, np.int32)
    for k in range(max_outer):
        idx = np.nonzero(open_)[0]
        if idx.size == 0:
            break
        so, o, s, _ = eval_batch(tree, x_eps[idx], x_th[idx], dt, sin[idx], tol=tol,
                                 threads=threads)
        sout[idx], out[idx], st[idx] = so, o, s
        for q, i in enumerate(idx):
            sig, C, C_th = o[q, 0:6], o[q, 6:42].reshape(6, 6), o[q, 42:48]
            D, D_eps, D_th = o[q, 48], o[q, 49:55], o[q, 55]
            if s[q] & 3:
                failed[i], open_[i], outer[i] = True, False, k + 1
                continue
            stress = [c for c in range(6) if (mask[i] >> c) & 1]
            adiabatic = bool((mask[i] >> 6) & 1)
            scale = max(1.0, np.abs(sig).max())
            r = [sig[c] - target[i, c] for c in stress]
            done = all(abs(v) <= tol_outer * scale for v in r)
            if adiabatic:
                rh = c_heat * (x_th[i] - theta_n[i]) / dt - D
                r.append(rh)
                done = done and abs(rh) <= tol_outer * c_heat / dt
            if done:
                open_[i], outer[i] = False, k + 1
                continue
            if k + 1 == max_outer:
                failed[i], open_[i], outer[i] = True, False, k + 1
                continue
            J = np.zeros((len(r), len(r)))
            for a, c in enumerate(stress):
                for b, e in enumerate(stress):
                    J[a, b] = C[c, e]
                if adiabatic:
                    J[a, -1] = C_th[c]
            if adiabatic:
                for b, e in enumerate(stress):
                    J[-1, b] = -D_eps[e]
                J[-1, -1] = c_heat / dt - D_th
            step = np.linalg.solve(J, -np.asarray(r))
            for a, c in enumerate(stress):
                x_eps[i, c] += step[a]
            if adiabatic:
                x_th[i] += step[-1]
    st = st | np.where(failed, 8, 0).astype(np.int32)
    return x_eps, x_th, sout, out, st, outer
