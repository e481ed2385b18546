"""Thin ctypes binding of the C ABI in ``include/dmn.h``.

Argument marshalling only: every step of the evaluation runs in the CUDA
library.  PyTorch tensors provide device memory and streams.  If the library
is missing the import fails; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

DMN_OK, DMN_ERR_ARG = 0, 1
PT_OK, PT_NOT_CONVERGED, PT_NONFINITE, PT_FALLBACK_USED = 0, 1, 2, 4
PT_OUTER_NOT_CONVERGED = 8
PT_BOUNDS = 16  # debug library: an index check failed at the point
MIXED_ADIABATIC = 1 << 6  # dmn_eval_mixed mask bit: theta from the heat balance
MIXED_PREDICT = 1  # dmn_eval_mixed flag: start from the previous outputs' linear model
PREC_FP64, PREC_MIXED = 0, 1
OUT_WORDS = 57

_lib = None


class dmn_material(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad_", ctypes.c_int32), ("E", ctypes.c_double),
                ("nu", ctypes.c_double), ("alpha", ctypes.c_double), ("theta0", ctypes.c_double),
                ("sy0", ctypes.c_double), ("dsy_dT", ctypes.c_double), ("H", ctypes.c_double),
                ("m_rate", ctypes.c_double), ("t_visc", ctypes.c_double), ("dE_dT", ctypes.c_double),
                ("k_hard", ctypes.c_double), ("n_hard", ctypes.c_double), ("eta0", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("theta_ref", ctypes.c_double),
                ("wlf_C1", ctypes.c_double), ("wlf_C2", ctypes.c_double),
                ("E_maxwell", ctypes.c_double * 12), ("tau_maxwell", ctypes.c_double * 12)]


class dmn_options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("gamma", ctypes.c_double),
                ("res_floor", ctypes.c_double), ("maxit", ctypes.c_int32),
                ("maxbacktrack", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("solve_variant", ctypes.c_int32)]


# every symbol the header declares, with its signature
_P, _I32, _I64, _D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "dmn_default_options": (None, [_P]),
    "dmn_create": (_I32, [_P, _I32, _P, _P, _P, _P, _I32, _P]),
    "dmn_destroy": (_I32, [_P]),
    "dmn_state_words": (_I64, [_P]),
    "dmn_state_init": (_I32, [_P, _P, _I64, _P, _P]),
    "dmn_eval": (_I32, [_P, _P, _I64, _P, _P, _D, _P, _P, _P, _P, _P]),
    "dmn_last_error": (ctypes.c_char_p, []),
    "dmn_eval_noalloc": (_I32, [_I32, _P, _P, _P, _P, _I32, _P, _P, _I64, _P, _P, _D, _P, _P, _P,
                                _P, _P]),
    "dmn_debug_bounds_log": (_I32, [_P, _P, _P, _P, _I32]),
    # include/dmn_mlp.h
    "dmn_mlp_create": (_I32, [_P, _I32, _I32, _I32, _I64, ctypes.c_uint64]),
    "dmn_mlp_destroy": (_I32, [_P]),
    "dmn_mlp_dims": (_I32, [_P, _P, _P, _P, _P]),
    "dmn_mlp_features": (_I32, [_P, _P, _I64, _P, _P, _P, _P, _I64, _P]),
    "dmn_mlp_input": (_I32, [_P, _P, _I64, _P, _P, _P, _P, _I64, _P]),
    "dmn_mlp_targets": (_I32, [_P, _P, _I64, _P, _P, _I64, _P]),
    "dmn_mlp_fit_normalization": (_I32, [_P, _P, _I64, _P, _P]),
    "dmn_mlp_normalize_features": (_I32, [_P, _P, _I64, _P, _P]),
    "dmn_mlp_normalize_targets": (_I32, [_P, _P, _I64, _P, _P]),
    "dmn_mlp_train_step": (_I32, [_P, _P, _I64, _P, _P, ctypes.c_float, _P]),
    "dmn_mlp_predict": (_I32, [_P, _P, _I64, _P, _P]),
    "dmn_mlp_param_count": (_I64, [_P]),
    "dmn_mlp_get_params": (_I32, [_P, _P]),
    "dmn_mlp_set_params": (_I32, [_P, _P]),
    "dmn_mlp_get_grads": (_I32, [_P, _P]),
    "dmn_mlp_get_moments": (_I32, [_P, _P, _P, _P]),
    "dmn_mlp_amsgrad": (_I32, [_P, _I64, _P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, ctypes.c_float, _I64]),
    "dmn_mlp_get_normalization": (_I32, [_P, _P, _P, _P, _P]),
    "dmn_gemm_bf16_tn": (_I32, [_P, _I32, _I32, _I32, _P, _P, _P]),
    "dmn_eval_warm": (_I32, [_P, _P, _I64, _P, _P, _D, _P, _P, _P, _P, _P, _P]),
    "dmn_eval_mixed": (_I32, [_P, _P, _I64, _P, _P, _P, _P, _D, _D, _I32, _D, _P, _P, _P, _P, _P,
                              _P, _P, _I32]),
    # include/dmn_linear.h
    "dmn_linear_forward": (_I32, [_P, _I32, _I64, _P, _P, _P, _P, _P, _I32]),
    "dmn_linear_loss_grad": (_I32, [_P, _I32, _I64, _P, _P, _P, _P, _P, _D, _D, _D, _P, _P, _P, _P, _I32]),
    "dmn_linear_amsgrad": (_I32, [_P, _I64, _P, _P, _P, _P, _P, _D, _D, _D, _D, _I64]),
}


def _debug() -> bool:
    """DMN_LIBRARY=debug selects the bounds-checking build of the library."""
    return os.environ.get("DMN_LIBRARY", "") == "debug"


def library_path() -> str:
    return _build.LIB_DEBUG if _debug() else _build.LIB


def load(build_if_missing: bool = True):
    """Load ``libdmn.so`` (or, with DMN_LIBRARY=debug, ``libdmn_debug.so``),
    building it with nvcc if it is missing."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise ImportError(f"DMN CUDA library not built: {path}")
            _build.build(debug=_debug())
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(rc, what):
    if rc != DMN_OK:
        msg = _lib.dmn_last_error().decode(errors="replace")
        raise RuntimeError(f"{what} failed with status {rc}: {msg}")


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def materials_from_rows(rows):
    """Material table rows -> ctypes array.  Kinds 0-2: (kind, E, nu, alpha,
    theta0, sy0, dsy_dT, H[, m_rate, t_visc, dE_dT, 0]); rows of 8 leave the
    Perzyna fields 0.  Kind 3 (PA66, 40 columns): (3, E_inf, nu, alpha0, theta0,
    sy0, k, n, m, eta0, beta1, beta2, theta_ref, C1, C2, 0, E_1..E_12,
    tau_1..tau_12).  Shorter rows may be padded with zeros to 40 columns."""
    rows = np.atleast_2d(np.asarray(rows, np.float64))
    if rows.shape[1] not in (8, 11, 12, 40):
        raise ValueError("material rows have 8, 12 or 40 columns")
    arr = (dmn_material * rows.shape[0])()
    for i, r in enumerate(rows):
        arr[i].kind = int(r[0])
        arr[i].E, arr[i].nu, arr[i].alpha, arr[i].theta0 = r[1], r[2], r[3], r[4]
        arr[i].sy0 = r[5]
        if int(r[0]) == 3:
            if rows.shape[1] != 40:
                raise ValueError("PA66 rows have 40 columns")
            arr[i].k_hard, arr[i].n_hard, arr[i].m_rate, arr[i].eta0 = r[6], r[7], r[8], r[9]
            arr[i].beta1, arr[i].beta2, arr[i].theta_ref = r[10], r[11], r[12]
            arr[i].wlf_C1, arr[i].wlf_C2 = r[13], r[14]
            for b in range(12):
                arr[i].E_maxwell[b], arr[i].tau_maxwell[b] = r[16 + b], r[28 + b]
            continue
        arr[i].dsy_dT, arr[i].H = r[6], r[7]
        if rows.shape[1] > 8:
            arr[i].m_rate, arr[i].t_visc, arr[i].dE_dT = r[8], r[9], r[10]
    return arr


class DMN:
    """A DMN handle on the current CUDA device (``dmn_create``)."""

    def __init__(self, K, w, normals, phase, mats, *, tol=1e-10, maxit=50, maxbacktrack=8,
                 gamma=0.5, precision="fp64", res_floor=0.0, solve_variant=None):
        lib = load()
        self.K = int(K)
        w = np.ascontiguousarray(w, np.float64)
        normals = np.ascontiguousarray(normals, np.float64)
        phase = np.ascontiguousarray(phase, np.uint8)
        mt = materials_from_rows(mats)
        opt = dmn_options()
        lib.dmn_default_options(ctypes.byref(opt))
        opt.tol, opt.maxit, opt.maxbacktrack, opt.gamma = tol, maxit, maxbacktrack, gamma
        opt.res_floor = res_floor
        opt.precision = {"fp64": PREC_FP64, "mixed": PREC_MIXED}[precision]
        if solve_variant is None:  # the autotuner's choice, if it ran for this case
            from .autotune import lookup
            solve_variant = lookup(self.K, precision) if self.K <= 8 else 0
        opt.solve_variant = int(solve_variant)
        self.solve_variant = int(solve_variant)
        self.precision = precision
        h = ctypes.c_void_p()
        _check(lib.dmn_create(ctypes.byref(h), self.K, w.ctypes.data_as(_P),
                              normals.ctypes.data_as(_P), phase.ctypes.data_as(_P),
                              ctypes.cast(mt, _P), len(mt), ctypes.byref(opt)), "dmn_create")
        self._h = h
        self.state_words = int(lib.dmn_state_words(h))
        self.nnode = (1 << self.K) - 1

    def close(self):
        if getattr(self, "_h", None):
            _check(_lib.dmn_destroy(self._h), "dmn_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_state(self, theta0, stream=None):
        """Allocate and initialise a state batch for ``theta0`` (CUDA float64, n)."""
        import torch
        n = theta0.numel()
        s = torch.empty((n, self.state_words), dtype=torch.float64, device=theta0.device)
        _check(_lib.dmn_state_init(self._h, _dev(s, torch.float64, None, "state"), n,
                                   _dev(theta0, torch.float64, (n,), "theta0"),
                                   _stream_ptr(stream)), "dmn_state_init")
        return s

    def eval(self, deps, theta, dt, state_in, state_out=None, out=None, status=None, iters=None,
             stream=None):
        """One increment at every point (``dmn_eval``).  Returns (state_out, out, status, iters)."""
        import torch
        n = deps.shape[0]
        dev = deps.device
        if state_out is None:
            state_out = torch.empty_like(state_in)
        if out is None:
            out = torch.empty((n, OUT_WORDS), dtype=torch.float64, device=dev)
        if status is None:
            status = torch.empty(n, dtype=torch.int32, device=dev)
        if iters is None:
            iters = torch.empty(n, dtype=torch.int32, device=dev)
        _check(_lib.dmn_eval(self._h, _stream_ptr(stream), n,
                             _dev(deps, torch.float64, (n, 6), "deps"),
                             _dev(theta, torch.float64, (n,), "theta"), float(dt),
                             _dev(state_in, torch.float64, (n, self.state_words), "state_in"),
                             _dev(state_out, torch.float64, (n, self.state_words), "state_out"),
                             _dev(out, torch.float64, (n, OUT_WORDS), "out"),
                             _dev(status, torch.int32, (n,), "status"),
                             _dev(iters, torch.int32, (n,), "iters")), "dmn_eval")
        return state_out, out, status, iters

    def eval_mixed(self, mask, target, deps, theta, dt, c_heat, state_in, *, max_outer=10,
                   tol_outer=1e-10, warm=True, out=None, predict=False, stream=None):
        """``dmn_eval_mixed``: prescribed stresses (mask bits 0..5) and adiabatic
        temperature (bit 6).  ``deps`` and ``theta`` are updated in place.  With
        ``predict``, ``out`` must hold the outputs of the increment that ended
        in ``state_in``; it is overwritten.  Returns (state_out, out, status,
        iters, outer)."""
        import torch
        n = deps.shape[0]
        dev = deps.device
        state_out = torch.empty_like(state_in)
        if predict and out is None:
            raise ValueError("predict needs the previous increment's out")
        if out is None:
            out = torch.empty((n, OUT_WORDS), dtype=torch.float64, device=dev)
        status = torch.empty(n, dtype=torch.int32, device=dev)
        iters = torch.empty(n, dtype=torch.int32, device=dev)
        outer = torch.empty(n, dtype=torch.int32, device=dev)
        work = torch.empty((n, 3 * self.nnode), dtype=torch.float32, device=dev) if warm else None
        _check(_lib.dmn_eval_mixed(self._h, _stream_ptr(stream), n,
                                   _dev(mask, torch.uint8, (n,), "mask"),
                                   _dev(target, torch.float64, (n, 6), "target"),
                                   _dev(deps, torch.float64, (n, 6), "deps"),
                                   _dev(theta, torch.float64, (n,), "theta"), float(dt),
                                   float(c_heat), int(max_outer), float(tol_outer),
                                   _dev(state_in, torch.float64, (n, self.state_words), "state_in"),
                                   _dev(state_out, torch.float64, (n, self.state_words), "state_out"),
                                   _dev(out, torch.float64, (n, OUT_WORDS), "out"),
                                   _dev(status, torch.int32, (n,), "status"),
                                   _dev(iters, torch.int32, (n,), "iters"),
                                   _dev(outer, torch.int32, (n,), "outer"),
                                   None if work is None else
                                   _dev(work, torch.float32, None, "work"),
                                   MIXED_PREDICT if predict else 0), "dmn_eval_mixed")
        return state_out, out, status, iters, outer

    def eval_warm(self, deps, theta, dt, state_in, da, state_out=None, out=None, status=None,
                  iters=None, stream=None):
        """``dmn_eval_warm``: start from a^n + da (fp32 [n, 3(2^K-1)])."""
        import torch
        n = deps.shape[0]
        dev = deps.device
        if state_out is None:
            state_out = torch.empty_like(state_in)
        if out is None:
            out = torch.empty((n, OUT_WORDS), dtype=torch.float64, device=dev)
        if status is None:
            status = torch.empty(n, dtype=torch.int32, device=dev)
        if iters is None:
            iters = torch.empty(n, dtype=torch.int32, device=dev)
        _check(_lib.dmn_eval_warm(self._h, _stream_ptr(stream), n,
                                  _dev(deps, torch.float64, (n, 6), "deps"),
                                  _dev(theta, torch.float64, (n,), "theta"), float(dt),
                                  _dev(state_in, torch.float64, (n, self.state_words), "state_in"),
                                  _dev(state_out, torch.float64, (n, self.state_words), "state_out"),
                                  _dev(out, torch.float64, (n, OUT_WORDS), "out"),
                                  _dev(status, torch.int32, (n,), "status"),
                                  _dev(iters, torch.int32, (n,), "iters"),
                                  _dev(da, torch.float32, (n, 3 * self.nnode), "da")), "dmn_eval_warm")
        return state_out, out, status, iters


def bounds_log(clear=True):
    """The debug library's index-check log: (count, index, bound, line)."""
    lib = load()
    c, i, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    ln = ctypes.c_int32()
    _check(lib.dmn_debug_bounds_log(ctypes.byref(c), ctypes.byref(i), ctypes.byref(b), ctypes.byref(ln),
                                    1 if clear else 0), "dmn_debug_bounds_log")
    return c.value, i.value, b.value, ln.value
