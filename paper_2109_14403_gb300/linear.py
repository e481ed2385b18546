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


def lr_schedule(m, alpha_min=1.5e-3, alpha_max=1.5e-2, M=50, gamma=0.999):
    """Learning rate of epoch m: the harmonic modulation with geometric decay
    of the paper's offline training (Sec. 5.3, eq. learning_rate_modulation),
    gamma^m (alpha_min + (alpha_max - alpha_min)(1 + cos(pi m / M)) / 2);
    its defaults are the paper's values."""
    import math
    return gamma ** m * (alpha_min + 0.5 * (alpha_max - alpha_min) * (1.0 + math.cos(math.pi * m / M)))


def mean_error(net, C1, C2, Ctarget, precision="fp64"):
    """e_mean of Sec. 5.3: the mean over the samples of |DMN^L - C_target|_1 /
    |C_target|_1 (36 components), which is the data term of the loss with
    p = q = 1 (one loss launch sequence; the gradient it also computes is
    discarded)."""
    keep = net.grad.clone()
    loss = net.loss_grad(C1, C2, Ctarget, p=1.0, q=1.0, penalty=0.0, precision=precision)
    net.grad.copy_(keep)
    return float(loss[1].item())


def train(net, C1, C2, Ctarget, epochs, batch=32, p=1.0, q=10.0, penalty=1e3, precision="fp32",
          schedule=lr_schedule, seed=0):
    """Mini-batch offline training (Sec. 3.2 and 5.3): every epoch visits the
    samples in a random order in batches of `batch` (a smaller last batch is
    dropped, as in the paper), takes the loss gradient of each batch on the
    GPU and one AMSGrad step with the epoch's learning rate for the normals and
    the weights.  Returns the data term of the loss of the last batch of each
    epoch."""
    import torch
    n = C1.shape[0]
    g = torch.Generator(device=C1.device).manual_seed(seed)
    history = []
    for m in range(epochs):
        lr = schedule(m)
        perm = torch.randperm(n, device=C1.device, generator=g)
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            net.loss_grad(C1[idx].contiguous(), C2[idx].contiguous(), Ctarget[idx].contiguous(), p=p, q=q,
                          penalty=penalty, precision=precision)
            net.amsgrad_step(lr, lr)
        history.append(float(net.loss[1].item()))
    return history
