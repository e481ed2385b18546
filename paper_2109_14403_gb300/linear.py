"""Python binding of include/dmn_linear.h: the linear homogenization function
DMN^L of a batch of stiffness samples, the gradient of the offline-training
loss and an AMSGrad step (arXiv 2109.14403, Sec. 3.2).  Argument marshalling
only; every step runs in the library's kernels."""
from __future__ import annotations

from . import dmn as _dmn

LIN_FP64, LIN_FP32 = 0, 1


def _prec(precision):
    return {"fp64": LIN_FP64, "fp32": LIN_FP32}[precision]


class DMNLinear:
    """Parameters (normals [(2^K-1), 3], unconstrained weights v [2^K]) of a
    depth-K DMN^L on the current CUDA device, kept in one FP64 tensor so that
    one AMSGrad call updates them together."""

    def __init__(self, K, normals, v, device=None):
        import torch
        self._lib = _dmn.load()
        self.K = int(K)
        self.N = (1 << self.K) - 1
        dev = torch.device("cuda") if device is None else device
        n = torch.as_tensor(normals, dtype=torch.float64).reshape(self.N, 3)
        w = torch.as_tensor(v, dtype=torch.float64).reshape(1 << self.K)
        self.params = torch.cat([n.reshape(-1), w]).to(dev).contiguous()
        self.grad = torch.zeros_like(self.params)
        self._m = torch.zeros_like(self.params)
        self._s = torch.zeros_like(self.params)
        self._smax = torch.zeros_like(self.params)
        self.loss = torch.zeros(3, dtype=torch.float64, device=dev)
        self.step_count = 0
        self._work = None

    @property
    def normals(self):
        return self.params[:3 * self.N].view(self.N, 3)

    @property
    def v(self):
        return self.params[3 * self.N:]

    def _ptr(self, t):
        import ctypes
        return ctypes.c_void_p(t.data_ptr())

    def _check_batch(self, *ts):
        import torch
        for t in ts:
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise TypeError("stiffness batches must be contiguous CUDA float64 tensors [n, 6, 6]")
            if t.numel() != 36 * ts[0].shape[0]:
                raise ValueError("stiffness batches must be [n, 6, 6]")

    def forward(self, C1, C2, precision="fp64", out=None, stream=None):
        """DMN^L(C1^s, C2^s) for every sample: [n, 6, 6]."""
        import torch
        self._check_batch(C1, C2)
        n = C1.shape[0]
        if out is None:
            out = torch.empty((n, 6, 6), dtype=torch.float64, device=C1.device)
        _dmn._check(self._lib.dmn_linear_forward(_dmn._stream_ptr(stream), self.K, n, self._ptr(C1),
                                                 self._ptr(C2), self._ptr(self.normals.contiguous()),
                                                 self._ptr(self.v), self._ptr(out), _prec(precision)),
                    "dmn_linear_forward")
        return out

    def loss_grad(self, C1, C2, Ctarget, p=1.0, q=10.0, penalty=1e3, precision="fp64", stream=None):
        """Loss J (eq. loss_function) into self.loss = (J, data, penalty) and
        its gradient into self.grad (normals first, then v)."""
        import torch
        self._check_batch(C1, C2, Ctarget)
        n = C1.shape[0]
        cells = 42 * (self.N + 1) * n  # packed phases, node stiffnesses and adjoints
        need = n + 8 * self.N + 8 + (cells if precision == "fp64" else (cells + 1) // 2)
        if self._work is None or self._work.numel() < need:
            self._work = torch.empty(need, dtype=torch.float64, device=C1.device)
        _dmn._check(self._lib.dmn_linear_loss_grad(
            _dmn._stream_ptr(stream), self.K, n, self._ptr(C1), self._ptr(C2), self._ptr(Ctarget),
            self._ptr(self.params), self._ptr(self.v), float(p), float(q), float(penalty),
            self._ptr(self.loss), self._ptr(self.grad), self._ptr(self.grad[3 * self.N:]),
            self._ptr(self._work), _prec(precision)), "dmn_linear_loss_grad")
        return self.loss

    def amsgrad_step(self, lr_n, lr_v, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        """One AMSGrad step of the normals (rate lr_n) and the weights (lr_v)."""
        self.step_count += 1
        s = _dmn._stream_ptr(stream)
        for lo, hi, lr in ((0, 3 * self.N, lr_n), (3 * self.N, self.params.numel(), lr_v)):
            _dmn._check(self._lib.dmn_linear_amsgrad(
                s, hi - lo, self._ptr(self.params[lo:]), self._ptr(self.grad[lo:]), self._ptr(self._m[lo:]),
                self._ptr(self._s[lo:]), self._ptr(self._smax[lo:]), float(lr), float(beta1), float(beta2),
                float(eps), self.step_count), "dmn_linear_amsgrad")
