/*
 * dmn_linear.h -- C ABI of the DMN's linear elastic homogenization function
 * DMN^L and of the gradient of the offline-training loss, for a batch of
 * stiffness samples on the GPU (Gajek, Schneider, Boehlke, arXiv 2109.14403,
 * Sec. 3.2: eqs. DMN^L, laminate, loss_function; w = <v>_+).
 *
 * Conventions as in dmn.h: Mandel basis, 6x6 stiffnesses row-major (the
 * library reads the symmetric part), lamination directions in the paper's
 * node order (bottom level first, root last; 2^K - 1 of them, normalised
 * inside: P(n) needs unit vectors), unconstrained weights v (2^K; the leaf
 * weights are w = max(v, 0)).  Leaf 2i (0-based) of bottom laminate i takes
 * phase 1 (C1), leaf 2i+1 phase 2 (C2).  A node whose leaves all have zero
 * weight gets volume fractions 1/2 (its parent gives it fraction 0).
 * Every d_* pointer is device memory owned by the caller; calls are stream-
 * ordered and do not synchronise; argument errors are reported before any
 * launch (DMN_ERR_ARG, message by dmn_last_error()).
 */
#ifndef DMN_LINEAR_H_
#define DMN_LINEAR_H_

#include "dmn.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { DMN_LIN_FP64 = 0, DMN_LIN_FP32 = 1 }; /* arithmetic of the laminate kernels */

/*
 * DMN^L(C1^s, C2^s, n, w) for every sample s (eq. DMN^L): the laminates are
 * propagated from the bottom level to the root.  Each laminate is computed in
 * the condensed form C = c1 C_L + c2 C_R - c1 c2 D B (B^T M B)^-1 B^T D with
 * D = C_L - C_R, M = c2 C_L + c1 C_R, B a = sym(a (x) n), the same stiffness as
 * the paper's eq. (laminate) in exact arithmetic.
 *   K          depth, 1..8
 *   n_samples  >= 0
 *   d_C1, d_C2 n_samples x 36 doubles
 *   d_normals  (2^K - 1) x 3 doubles, non-zero
 *   d_v        2^K doubles
 *   d_Cbar     n_samples x 36 doubles, written (symmetric)
 *   precision  DMN_LIN_FP64 or DMN_LIN_FP32 (laminate arithmetic; inputs and
 *              outputs stay FP64)
 */
dmn_status dmn_linear_forward(dmn_stream stream, int32_t K, int64_t n_samples, const double *d_C1,
                              const double *d_C2, const double *d_normals, const double *d_v,
                              double *d_Cbar, int32_t precision);

/*
 * The offline-training loss of eq. (loss_function) over the batch and its
 * gradient with respect to the normals and the unconstrained weights:
 *   J = (1/N) (sum_s e_s^q)^(1/q) + penalty (sum_j w_j - 1)^2,
 *   e_s = |C_target^s - DMN^L(C1^s, C2^s)|_p / |C_target^s|_p  (36 components)
 *   p, q >= 1; penalty >= 0
 *   d_loss     3 doubles: J, its data term, its penalty term
 *   d_grad_n   (2^K - 1) x 3 doubles: dJ / d normals (through the normalisation)
 *   d_grad_v   2^K doubles: dJ / dv (zero where v_j < 0)
 *   d_work     scratch of n_samples + 8 (2^K - 1) + 8 doubles, then the packed
 *              phase stiffnesses, the node stiffnesses and their adjoints:
 *              42 2^K n_samples words of the laminate precision (doubles for
 *              DMN_LIN_FP64, floats for DMN_LIN_FP32), 2.8 GB at K = 8,
 *              65,536 samples, FP32
 * The gradient is exact for the forward computation (reverse mode through
 * every laminate).  Level-synchronous over the batch: K forward launches,
 * errors, batch reduction, seed, K backward launches, the chain through the
 * weights (2K + 7 launches).
 */
dmn_status dmn_linear_loss_grad(dmn_stream stream, int32_t K, int64_t n_samples, const double *d_C1,
                                const double *d_C2, const double *d_Ctarget, const double *d_normals,
                                const double *d_v, double p, double q, double penalty, double *d_loss,
                                double *d_grad_n, double *d_grad_v, double *d_work,
                                int32_t precision);

/*
 * One AMSGrad step (the optimiser the paper trains with) on n_params FP64
 * parameters, bias-corrected: m = b1 m + (1-b1) g, s = b2 s + (1-b2) g^2,
 * smax = max(smax, s), x -= lr (m / (1 - b1^t)) / (sqrt(smax / (1 - b2^t)) + eps).
 * t = step >= 1; m, s, smax start at zero.
 */
dmn_status dmn_linear_amsgrad(dmn_stream stream, int64_t n_params, double *d_params,
                              const double *d_grad, double *d_m, double *d_s, double *d_smax,
                              double lr, double beta1, double beta2, double eps, int64_t step);

#ifdef __cplusplus
}
#endif
#endif /* DMN_LINEAR_H_ */
