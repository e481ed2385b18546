"""Host-side conversion between the library's Mandel notation and the Voigt
notation with engineering shear that finite-element codes such as ABAQUS use
for a material routine (UMAT: STRESS, DSTRAN, DDSDDE, DDSDDT, RPL, DRPLDE).

Mandel (the library): symmetric tensors as
    (x11, x22, x33, sqrt2 x23, sqrt2 x13, sqrt2 x12),
the same for stresses and strains, so that s . e is the double contraction
and a fourth-order tangent is a symmetric 6 x 6 matrix.
Voigt (ABAQUS order): stresses (s11, s22, s33, s12, s13, s23), strains
(e11, e22, e33, g12, g13, g23) with engineering shear g_ij = 2 e_ij.

With s_m = T_s s_v and e_m = T_e e_v (T_s, T_e the permutation below with the
shear entries scaled by sqrt2 and 1/sqrt2), the tangent is
C_v = T_s^-1 C_m T_e, i.e. C_v[i, j] = f_i f_j C_m[m(i), m(j)] with
f = (1, 1, 1, 1/sqrt2, 1/sqrt2, 1/sqrt2); it stays symmetric.

The functions take numpy arrays or torch tensors whose last axis (or last two,
for a tangent) has length 6.  Nothing here runs on the solve path.
"""
import math

# Mandel component of each Voigt slot (and the reverse: the map is its own
# inverse): 11, 22, 33, then 12 <-> Mandel 5, 13 <-> 4, 23 <-> Mandel 3
PERM = [0, 1, 2, 5, 4, 3]
_S = 1.0 / math.sqrt(2.0)
_F = [1.0, 1.0, 1.0, _S, _S, _S]       # shear scale from Mandel to Voigt stress
_FI = [1.0, 1.0, 1.0, 1 / _S, 1 / _S, 1 / _S]


def _vec(x, scale):
    """x[..., PERM] times the per-slot scale (numpy or torch)."""
    out = x[..., PERM]
    return out * _as(scale, out)


def _as(vals, like):
    try:
        import torch
        if isinstance(like, torch.Tensor):
            return torch.tensor(vals, dtype=like.dtype, device=like.device)
    except ImportError:
        pass
    import numpy as np
    return np.asarray(vals, dtype=like.dtype)


def stress_to_voigt(s_mandel):
    """Stress, or a stress-like vector (d sigma / d theta: DDSDDT), Mandel to Voigt."""
    return _vec(s_mandel, _F)


def stress_to_mandel(s_voigt):
    return _vec(s_voigt, _FI)


def strain_to_mandel(e_voigt):
    """Strain or strain increment with engineering shear (DSTRAN), Voigt to Mandel."""
    return _vec(e_voigt, _F)


def strain_to_voigt(e_mandel):
    return _vec(e_mandel, _FI)


def strain_gradient_to_voigt(g_mandel):
    """Derivative of a scalar by the Mandel strain (d D / d eps) as the derivative
    by the Voigt strain with engineering shear (DRPLDE): g_v = T_e^T g_m."""
    return _vec(g_mandel, _F)


def tangent_to_voigt(c_mandel):
    """d sigma / d eps, 6 x 6 Mandel, as ABAQUS's DDSDDE."""
    c = c_mandel[..., PERM, :][..., :, PERM]
    f = _as(_F, c)
    return c * f[:, None] * f[None, :]


def tangent_to_mandel(c_voigt):
    """Inverse of tangent_to_voigt."""
    c = c_voigt[..., PERM, :][..., :, PERM]
    f = _as(_FI, c)
    return c * f[:, None] * f[None, :]
