/*
 * dmn_mlp.h -- learned warm start for the DMN Newton solve.
 *
 * The paper starts Algorithm 1 from the previous converged jumps, a^{n+1} <-
 * a^n.  This part of the library (no counterpart in the paper) predicts the
 * increment a^{n+1} - a^n with a small multilayer perceptron and starts the
 * same Newton iteration, to the same tolerance, from a^n + prediction; a point
 * whose warm-started iteration fails is re-run from a^n.
 *
 * Network: input [deps (6), theta^{n+1}, theta^{n+1} - theta^n,
 * a^n - a^{n-1} (3(2^K - 1))], normalised per column; n_hidden layers of width
 * `hidden` with SiLU; linear output of 3(2^K - 1) normalised increments.
 * BF16 weights and activations, FP32 accumulation on the tensor cores
 * (tcgen05), FP32 master weights, MSE loss on normalised targets, AMSGrad
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 *
 * Padding: the input width is padded with zero columns to a multiple of 128
 * (n_in_pad), the output width to a multiple of 128 (n_out_pad); batches are
 * padded to a multiple of 128 rows internally.  All pointers are device
 * memory owned by the caller unless named h_*.  Every call is stream-ordered;
 * calls on one dmn_mlp must not overlap (they share its workspace).
 */
#ifndef DMN_MLP_H_
#define DMN_MLP_H_

#include "dmn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmn_mlp_s *dmn_mlp;

/* Create a network for trees of depth K (1..9), hidden width a multiple of 128,
   n_hidden >= 1 hidden layers, batches up to max_batch rows; weights drawn from
   U(-1/sqrt(fan_in), 1/sqrt(fan_in)) with the given seed, biases 0.
   Allocates weights, optimiser state and workspace on the current device. */
dmn_status dmn_mlp_create(dmn_mlp *out, int32_t K, int32_t hidden, int32_t n_hidden,
                          int64_t max_batch, uint64_t seed);
dmn_status dmn_mlp_destroy(dmn_mlp m);

/* Widths: n_in = 8 + 3(2^K-1), n_in_pad, n_out = 3(2^K-1), n_out_pad. */
dmn_status dmn_mlp_dims(dmn_mlp m, int32_t *n_in, int32_t *n_in_pad, int32_t *n_out,
                        int32_t *n_out_pad);

/* Raw features, fp32 [n x n_in], from the increment's inputs and the state at
   t^n; d_state_prev (state at t^{n-1}) may be NULL (no previous increment:
   the a^n - a^{n-1} columns are 0). */
dmn_status dmn_mlp_features(dmn_mlp m, dmn_stream stream, int64_t n, const double *d_deps,
                            const double *d_theta, const double *d_state_in,
                            const double *d_state_prev, int64_t state_words, float *d_feat);

/* The network input in one pass: the features above, normalised and rounded
   to bf16 [n x n_in_pad] (what dmn_mlp_predict takes). */
dmn_status dmn_mlp_input(dmn_mlp m, dmn_stream stream, int64_t n, const double *d_deps,
                         const double *d_theta, const double *d_state_in,
                         const double *d_state_prev, int64_t state_words, void *d_x_bf16);

/* Raw targets, fp32 [n x n_out]: a^{n+1} - a^n from the states before and
   after a converged increment. */
dmn_status dmn_mlp_targets(dmn_mlp m, dmn_stream stream, int64_t n, const double *d_state_in,
                           const double *d_state_out, int64_t state_words, float *d_tgt);

/* Per-column mean and standard deviation of a training set (device
   reduction); columns with zero spread are mapped to 0. */
dmn_status dmn_mlp_fit_normalization(dmn_mlp m, dmn_stream stream, int64_t n, const float *d_feat,
                                     const float *d_tgt);

/* Normalised network input, bf16 [n x n_in_pad] (padding columns 0). */
dmn_status dmn_mlp_normalize_features(dmn_mlp m, dmn_stream stream, int64_t n,
                                      const float *d_feat, void *d_x_bf16);

/* Normalised targets, fp32 [n x n_out_pad] (padding columns 0). */
dmn_status dmn_mlp_normalize_targets(dmn_mlp m, dmn_stream stream, int64_t n, const float *d_tgt,
                                     float *d_t);

/* One AMSGrad step on a batch of n <= max_batch rows: forward, MSE on the
   normalised targets (mean over n x n_out), backward, update.  *d_loss (may be
   NULL) receives the batch loss.  lr = 0 computes gradients only. */
dmn_status dmn_mlp_train_step(dmn_mlp m, dmn_stream stream, int64_t n, const void *d_x_bf16,
                              const float *d_t, float lr, float *d_loss);

/* Forward pass: the de-normalised predicted increment, fp32 [n x n_out]. */
dmn_status dmn_mlp_predict(dmn_mlp m, dmn_stream stream, int64_t n, const void *d_x_bf16,
                           float *d_da);

/* Number of parameters in the flat layout used below: per layer l, W_l
   [out_pad x in_pad] row-major then b_l [out_pad] (padded entries are 0). */
int64_t dmn_mlp_param_count(dmn_mlp m);
/* FP32 master parameters to / from host memory (synchronous). */
dmn_status dmn_mlp_get_params(dmn_mlp m, float *h_params);
dmn_status dmn_mlp_set_params(dmn_mlp m, const float *h_params);
/* Gradients of the last train step, same layout (synchronous). */
dmn_status dmn_mlp_get_grads(dmn_mlp m, float *h_grads);
/* Optimiser state of the last train step, same layout (synchronous): the
   first and second moment estimates and the running maximum of the second
   (each pointer may be NULL). */
dmn_status dmn_mlp_get_moments(dmn_mlp m, float *h_m, float *h_v, float *h_vmax);

/* The optimiser step dmn_mlp_train_step ends with, on caller buffers: one
   AMSGrad step (Reddi, Kale, Kumar 2018, the running maximum of the second
   moment; the optimiser the paper trains its DMN with, Sec. 5.3) with Adam's
   bias correction, in FP32, element-wise over n entries of device arrays:
     m = b1 m + (1-b1) g,  v = b2 v + (1-b2) g^2,  vmax = max(vmax, v),
     w -= lr (m / (1 - b1^t)) / (sqrt(vmax / (1 - b2^t)) + eps),
   t = step >= 1; m, v, vmax start at 0.  The bias corrections are formed in
   FP64 from the FP32 betas and rounded once.  dmn_mlp_train_step uses
   b1 = 0.9, b2 = 0.999, eps = 1e-8.  Stream-ordered; DMN_ERR_ARG for
   step < 1, betas outside [0, 1), eps <= 0 or a NULL pointer. */
dmn_status dmn_mlp_amsgrad(dmn_stream stream, int64_t n, float *d_w, const float *d_g, float *d_m,
                           float *d_v, float *d_vmax, float lr, float beta1, float beta2, float eps,
                           int64_t step);
/* Normalisation statistics (synchronous): feature mean and 1/std [n_in],
   target mean and std [n_out]. */
dmn_status dmn_mlp_get_normalization(dmn_mlp m, float *h_fmean, float *h_finv, float *h_tmean,
                                     float *h_tstd);

/* Building block: C = A B^T with A bf16 [M x K], B bf16 [N x K] (K
   contiguous), C fp32 [M x N]; M, N multiples of 128, K of 64.  Runs the
   tcgen05 GEMM the network uses. */
dmn_status dmn_gemm_bf16_tn(dmn_stream stream, int32_t M, int32_t N, int32_t K, const void *d_a,
                            const void *d_b, float *d_c);

/* dmn_eval started from a^n + d_da (fp32 [n x 3(2^K-1)], e.g. from
   dmn_mlp_predict) instead of a^n; the same Algorithm 1 iteration and
   tolerance follow.  A point whose warm-started iteration does not converge is
   re-run from a^n in the same launch and gets the status bit
   DMN_PT_FALLBACK_USED; its iteration count includes both runs. */
dmn_status dmn_eval_warm(dmn_handle h, dmn_stream stream, int64_t n_points, const double *d_deps,
                         const double *d_theta, double dt, const double *d_state_in,
                         double *d_state_out, double *d_out, int32_t *d_status, int32_t *d_iters,
                         const float *d_da);

#ifdef __cplusplus
}
#endif
#endif /* DMN_MLP_H_ */
