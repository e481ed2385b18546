"""Thin binding of ``include/dmn_mlp.h``: the learned warm start.

Argument marshalling only; the network's forward and backward passes, the
normalisation and the optimiser run in the CUDA library (tcgen05 GEMMs).
"""
from __future__ import annotations

import ctypes

import numpy as np

from .dmn import _P, _check, _dev, _stream_ptr, load


class MLP:
    def __init__(self, K, hidden=512, n_hidden=3, max_batch=65536, seed=0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.dmn_mlp_create(ctypes.byref(h), int(K), int(hidden), int(n_hidden),
                                  int(max_batch), int(seed)), "dmn_mlp_create")
        self._h = h
        self.K, self.hidden, self.n_hidden, self.max_batch = int(K), int(hidden), int(n_hidden), int(max_batch)
        d = [ctypes.c_int32() for _ in range(4)]
        _check(lib.dmn_mlp_dims(h, *[ctypes.byref(x) for x in d]), "dmn_mlp_dims")
        self.n_in, self.n_in_pad, self.n_out, self.n_out_pad = (x.value for x in d)
        self.n_params = int(lib.dmn_mlp_param_count(h))

    def layer_dims(self):
        """(in_pad, out_pad) of every layer, in the flat parameter order."""
        dims = [(self.n_in_pad, self.hidden)] + [(self.hidden, self.hidden)] * (self.n_hidden - 1)
        return dims + [(self.hidden, self.n_out_pad)]

    def close(self):
        if getattr(self, "_h", None):
            _check(load().dmn_mlp_destroy(self._h), "dmn_mlp_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def features(self, deps, theta, state_in, state_prev=None, out=None, stream=None):
        import torch
        n = deps.shape[0]
        if out is None:
            out = torch.empty((n, self.n_in), dtype=torch.float32, device=deps.device)
        sw = state_in.shape[1]
        prev = ctypes.c_void_p(0) if state_prev is None else _dev(state_prev, torch.float64, (n, sw), "state_prev")
        _check(load().dmn_mlp_features(self._h, _stream_ptr(stream), n,
                                       _dev(deps, torch.float64, (n, 6), "deps"),
                                       _dev(theta, torch.float64, (n,), "theta"),
                                       _dev(state_in, torch.float64, (n, sw), "state_in"), prev, sw,
                                       _dev(out, torch.float32, (n, self.n_in), "feat")), "dmn_mlp_features")
        return out

    def input(self, deps, theta, state_in, state_prev=None, out=None, stream=None):
        """Normalised bf16 network input in one pass (``dmn_mlp_input``)."""
        import torch
        n = deps.shape[0]
        if out is None:
            out = torch.empty((n, self.n_in_pad), dtype=torch.bfloat16, device=deps.device)
        sw = state_in.shape[1]
        prev = ctypes.c_void_p(0) if state_prev is None else _dev(state_prev, torch.float64, (n, sw), "state_prev")
        _check(load().dmn_mlp_input(self._h, _stream_ptr(stream), n,
                                    _dev(deps, torch.float64, (n, 6), "deps"),
                                    _dev(theta, torch.float64, (n,), "theta"),
                                    _dev(state_in, torch.float64, (n, sw), "state_in"), prev, sw,
                                    _dev(out, torch.bfloat16, (n, self.n_in_pad), "x")), "dmn_mlp_input")
        return out

    def targets(self, state_in, state_out, out=None, stream=None):
        import torch
        n, sw = state_in.shape
        if out is None:
            out = torch.empty((n, self.n_out), dtype=torch.float32, device=state_in.device)
        _check(load().dmn_mlp_targets(self._h, _stream_ptr(stream), n,
                                      _dev(state_in, torch.float64, (n, sw), "state_in"),
                                      _dev(state_out, torch.float64, (n, sw), "state_out"), sw,
                                      _dev(out, torch.float32, (n, self.n_out), "tgt")), "dmn_mlp_targets")
        return out

    def fit_normalization(self, feat, tgt, stream=None):
        import torch
        n = feat.shape[0]
        _check(load().dmn_mlp_fit_normalization(self._h, _stream_ptr(stream), n,
                                                _dev(feat, torch.float32, (n, self.n_in), "feat"),
                                                _dev(tgt, torch.float32, (n, self.n_out), "tgt")),
               "dmn_mlp_fit_normalization")

    def normalize_features(self, feat, out=None, stream=None):
        import torch
        n = feat.shape[0]
        if out is None:
            out = torch.empty((n, self.n_in_pad), dtype=torch.bfloat16, device=feat.device)
        _check(load().dmn_mlp_normalize_features(self._h, _stream_ptr(stream), n,
                                                 _dev(feat, torch.float32, (n, self.n_in), "feat"),
                                                 _dev(out, torch.bfloat16, (n, self.n_in_pad), "x")),
               "dmn_mlp_normalize_features")
        return out

    def normalize_targets(self, tgt, out=None, stream=None):
        import torch
        n = tgt.shape[0]
        if out is None:
            out = torch.empty((n, self.n_out_pad), dtype=torch.float32, device=tgt.device)
        _check(load().dmn_mlp_normalize_targets(self._h, _stream_ptr(stream), n,
                                                _dev(tgt, torch.float32, (n, self.n_out), "tgt"),
                                                _dev(out, torch.float32, (n, self.n_out_pad), "t")),
               "dmn_mlp_normalize_targets")
        return out

    def train_step(self, x, t, lr, loss=None, stream=None):
        import torch
        n = x.shape[0]
        lp = ctypes.c_void_p(0) if loss is None else _dev(loss, torch.float32, (1,), "loss")
        _check(load().dmn_mlp_train_step(self._h, _stream_ptr(stream), n,
                                         _dev(x, torch.bfloat16, (n, self.n_in_pad), "x"),
                                         _dev(t, torch.float32, (n, self.n_out_pad), "t"),
                                         float(lr), lp), "dmn_mlp_train_step")

    def predict(self, x, out=None, stream=None):
        import torch
        n = x.shape[0]
        if out is None:
            out = torch.empty((n, self.n_out), dtype=torch.float32, device=x.device)
        _check(load().dmn_mlp_predict(self._h, _stream_ptr(stream), n,
                                      _dev(x, torch.bfloat16, (n, self.n_in_pad), "x"),
                                      _dev(out, torch.float32, (n, self.n_out), "da")), "dmn_mlp_predict")
        return out

    def params(self):
        h = np.empty(self.n_params, np.float32)
        _check(load().dmn_mlp_get_params(self._h, h.ctypes.data_as(_P)), "dmn_mlp_get_params")
        return h

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.n_params
        _check(load().dmn_mlp_set_params(self._h, p.ctypes.data_as(_P)), "dmn_mlp_set_params")

    def grads(self):
        h = np.empty(self.n_params, np.float32)
        _check(load().dmn_mlp_get_grads(self._h, h.ctypes.data_as(_P)), "dmn_mlp_get_grads")
        return h

    def moments(self):
        """(m, v, vmax) of the optimiser after the last train step."""
        m, v, vm = (np.empty(self.n_params, np.float32) for _ in range(3))
        _check(load().dmn_mlp_get_moments(self._h, m.ctypes.data_as(_P), v.ctypes.data_as(_P),
                                          vm.ctypes.data_as(_P)), "dmn_mlp_get_moments")
        return m, v, vm

    def normalization(self):
        fm, fi = np.empty(self.n_in, np.float32), np.empty(self.n_in, np.float32)
        tm, ts = np.empty(self.n_out, np.float32), np.empty(self.n_out, np.float32)
        _check(load().dmn_mlp_get_normalization(self._h, fm.ctypes.data_as(_P), fi.ctypes.data_as(_P),
                                                tm.ctypes.data_as(_P), ts.ctypes.data_as(_P)),
               "dmn_mlp_get_normalization")
        return fm, fi, tm, ts


def amsgrad(w, g, m, v, vmax, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """One FP32 AMSGrad step on CUDA tensors, in place (``dmn_mlp_amsgrad``)."""
    import torch
    n = w.numel()
    ptrs = [_dev(t, torch.float32, (n,), name) for t, name in
            ((w, "w"), (g, "g"), (m, "m"), (v, "v"), (vmax, "vmax"))]
    _check(load().dmn_mlp_amsgrad(_stream_ptr(stream), n, *ptrs, float(lr), float(beta1), float(beta2),
                                  float(eps), int(step)), "dmn_mlp_amsgrad")


def gemm_bf16_tn(a, b, out=None, stream=None):
    """C = A B^T (bf16 in, fp32 out) on the library's tcgen05 GEMM."""
    import torch
    M, K = a.shape
    N = b.shape[0]
    if out is None:
        out = torch.empty((M, N), dtype=torch.float32, device=a.device)
    _check(load().dmn_gemm_bf16_tn(_stream_ptr(stream), M, N, K, _dev(a, torch.bfloat16, (M, K), "a"),
                                   _dev(b, torch.bfloat16, (N, K), "b"),
                                   _dev(out, torch.float32, (M, N), "c")), "dmn_gemm_bf16_tn")
    return out
