"""FP64 reference of the AMSGrad optimiser step.

TEST INFRASTRUCTURE ONLY: the tests compare the library's optimiser kernels
(the warm-start network's FP32 master weights, the DMN^L parameters in FP64)
with it.  Plain numpy, FP64.

AMSGrad (Reddi, Kale and Kumar, "On the convergence of Adam and beyond",
ICLR 2018, Algorithm 2) keeps the running maximum of the second-moment
estimate and divides by its square root; with the bias correction of Adam
(Kingma and Ba, ICLR 2015, Algorithm 1), which the paper's own training uses
through PyTorch's AMSGrad option (Sec. 5.3), one step t >= 1 is
    m_t = b1 m_{t-1} + (1 - b1) g_t
    v_t = b2 v_{t-1} + (1 - b2) g_t^2
    vmax_t = max(vmax_{t-1}, v_t)
    w_t = w_{t-1} - lr (m_t / (1 - b1^t)) / (sqrt(vmax_t / (1 - b2^t)) + eps)
with m, v, vmax zero before the first step.
"""
import numpy as np


def amsgrad_step(w, g, m, v, vmax, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One step at iteration t (1-based); returns the new (w, m, v, vmax)."""
    w, g, m, v, vmax = (np.asarray(a, np.float64) for a in (w, g, m, v, vmax))
    if t < 1:
        raise ValueError("t is 1-based")
    m_new = b1 * m + (1.0 - b1) * g
    v_new = b2 * v + (1.0 - b2) * g * g
    vmax_new = np.maximum(vmax, v_new)
    m_hat = m_new / (1.0 - b1 ** t)
    v_hat = vmax_new / (1.0 - b2 ** t)
    return w - lr * m_hat / (np.sqrt(v_hat) + eps), m_new, v_new, vmax_new
