/*
 * dmn.h -- C ABI of the GB300 (sm_103a) library for the online evaluation of a
 * thermomechanical direct deep material network (DMN) at a batch of
 * macroscopic Gauss points.
 *
 * Method: Gajek, Schneider, Boehlke, "An FE-DMN method for the multiscale
 * analysis of thermomechanical composites", arXiv 2109.14403.
 *   - tree, weights, volume fractions, normals ............ Sec. 3.1
 *   - kinematics eps = eps_bar + A a, balance A^T W sigma = 0, Newton
 *     system, effective stress / coupling term / dissipation, the four
 *     algorithmic tangents ................................ Sec. 3.3
 *   - the driver (warm start, Residual, Newton, Backtracking) Algorithm 1
 *   - phase laws (linear thermoelastic; J2 flow) ........... Sec. 4
 *
 * Conventions
 *   - Units MPa, K, s.
 *   - Symmetric tensors are Mandel 6-vectors (11, 22, 33, sqrt2*23, sqrt2*13,
 *     sqrt2*12); a fourth-order tangent is a 6x6 row-major matrix
 *     T[i][j] = d out_i / d in_j in that basis.
 *   - Tree nodes are numbered as the paper orders its lamination directions:
 *     bottom level first, left to right, root last (Sec. 3.1).  Leaf j
 *     (0-based) lies under child 1 of its parent laminate when j is even.
 *   - Kinematic operator A (the paper defers its form to Gajek et al. 2020):
 *     every leaf under child 1 of node p receives +c_{p,2} sym(a_p (x) n_p),
 *     every leaf under child 2 receives -c_{p,1} sym(a_p (x) n_p).  The
 *     converged stress and tangents do not depend on this choice; the scale
 *     of the Algorithm 1 residual does.
 *
 * Ownership: every d_* pointer is device memory owned by the caller.  A
 * handle owns device copies of the tree and material constants and one
 * work-queue counter that dmn_eval resets with a stream-ordered memset before
 * each launch: calls on one handle must therefore not run concurrently on
 * different streams (use one handle per stream).
 * Streams: every call that takes a stream is stream-ordered and does not
 * synchronise the device.  Errors: a non-zero dmn_status; the message of the
 * last error of the calling thread is returned by dmn_last_error().
 * Argument errors are detected before any launch.  Numerical failures are
 * reported per point in the status array, never as a call error.
 */
#ifndef DMN_H_
#define DMN_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dmn_handle_s *dmn_handle;
typedef void *dmn_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  DMN_OK = 0,
  DMN_ERR_ARG = 1,      /* invalid argument (checked before any launch)  */
  DMN_ERR_CUDA = 2,     /* a CUDA runtime call failed                    */
  DMN_ERR_OOM = 3,      /* device allocation failed                      */
  DMN_ERR_STATE = 4,    /* state buffer too small / wrong tree           */
  DMN_ERR_INTERNAL = 5
} dmn_status;

/* per-point status codes written by dmn_eval */
enum {
  DMN_PT_OK = 0,            /* residual < tol                              */
  DMN_PT_NOT_CONVERGED = 1, /* maxit Newton iterations without res < tol   */
  DMN_PT_NONFINITE = 2,     /* a residual or an output was NaN or Inf      */
  DMN_PT_FALLBACK_USED = 4, /* bit: warm start failed, re-run from a^n     */
  DMN_PT_OUTER_NOT_CONVERGED = 8, /* bit (dmn_eval_mixed): the prescribed
                                     stresses / heat balance were not met    */
  DMN_PT_STAGING_TIMEOUT = 32 /* the point's state block did not arrive in
                                 shared memory within the wait limit; the
                                 point is not evaluated and its CTA stops
                                 (the other points are taken by the others) */
};

/* phase laws (Sec. 4) */
enum {
  DMN_MAT_THERMOELASTIC = 0, /* sigma = C[eps - alpha (theta - theta0) I] */
  DMN_MAT_J2_LINEAR = 1,     /* J2 plasticity, linear isotropic hardening  */
  DMN_MAT_J2_PERZYNA = 2     /* J2 viscoplasticity with the overstress rate
                                law of Sec. 4 (p_dot = (1/t_visc)
                                <(q - sigma_Y - H p)/sigma_Y>^m), linear
                                hardening, moduli E (1 + dE_dT (theta -
                                theta0)); internal variables eps_p, p and
                                the leaf strain (13 words)                */,
  DMN_MAT_PA66 = 3           /* the PA66 matrix of Sec. 4 (after Krairi et
                                al.): long-term branch E (here E_inf) and up
                                to 12 Maxwell branches E_maxwell[i],
                                tau_maxwell[i] with a common nu, WLF-shifted
                                viscosities (wlf_C1, wlf_C2, theta_ref),
                                J2 viscoplasticity p_dot = (sigma_Y/eta)
                                <(q - sigma_Y - H)/sigma_Y>^m with sigma_Y =
                                Gamma(beta1) sy0, H = Gamma(beta1) k_hard
                                p^n_hard, eta = Gamma(beta2) eta0, Gamma(b) =
                                exp(-b (theta - theta_ref)); coupling term
                                and dissipation of the PA66 model; implicit
                                Euler; internal variables eps_vp (6), p and
                                the 12 Maxwell strains (79 words); trees
                                with K <= 8                                */
};

typedef struct {
  int32_t kind;   /* DMN_MAT_*                                              */
  int32_t pad_;
  double E;       /* Young's modulus (MPa), > 0                             */
  double nu;      /* Poisson's ratio, (-1, 0.5)                             */
  double alpha;   /* isotropic thermal expansion coefficient (1/K)          */
  double theta0;  /* reference temperature (K), > 0                         */
  double sy0;     /* J2: yield stress at theta0 (MPa), > 0                  */
  double dsy_dT;  /* J2: yield-stress slope (MPa/K); sigma_Y is floored at
                     1e-6 MPa                                               */
  double H;       /* J2: linear isotropic hardening modulus (MPa), >= 0     */
  double m_rate;  /* Perzyna: rate exponent m, an integer in 1..8           */
  double t_visc;  /* Perzyna: viscous time (s), > 0                         */
  double dE_dT;   /* Perzyna: relative modulus slope (1/K); the factor
                     1 + dE_dT (theta - theta0) is floored at 1e-3          */
  /* PA66 (kind 3; also uses E = E_inf, nu, alpha, theta0, sy0 and m_rate) */
  double k_hard, n_hard; /* hardening H = Gamma k_hard p^n_hard: k >= 0,
                            0 < n <= 1                                      */
  double eta0;           /* reference viscosity (MPa s), > 0                */
  double beta1, beta2;   /* thermal softening of sigma_Y and H, of eta (1/K) */
  double theta_ref;      /* reference temperature of Gamma and WLF (K)      */
  double wlf_C1, wlf_C2; /* WLF constants; C2 + theta - theta_ref must stay
                            > 0 (else the point reports a non-finite output) */
  double E_maxwell[12];  /* Maxwell moduli (MPa), >= 0; 0 = unused branch   */
  double tau_maxwell[12]; /* relaxation times at theta_ref (s), > 0 where
                             E_maxwell > 0                                  */
} dmn_material;

enum { DMN_PREC_FP64 = 0, DMN_PREC_MIXED = 1 };

typedef struct {
  double tol;           /* relative residual tolerance of Algorithm 1 (1e-10) */
  double gamma;         /* backtracking factor, step gamma^{i+1} (0.5)        */
  double res_floor;     /* floor of |sigma_bar|_F in the residual's
                           denominator (MPa); <= 0 selects 1e-8 * max E       */
  int32_t maxit;        /* Newton iterations (50), >= 1                       */
  int32_t maxbacktrack; /* backtracking steps per iteration (8), >= 0         */
  int32_t precision;    /* DMN_PREC_FP64: every step in FP64.  DMN_PREC_MIXED:
                           leaf tangents, condensation and the Newton
                           correction in FP32; strains, leaf stresses, the
                           residual, the convergence test and every output
                           accumulation in FP64-class precision (float-float
                           on the FP32 pipe, about 48 significant bits)          */
  int32_t solve_variant; /* kernel variant of the solve, depth K <= 8 (deeper
                           trees always take the default).  0 = library
                           default (owner-mapped kernel; mixed: 3 CTAs/SM);
                           2, 3, 4 = owner-mapped mixed kernel compiled for
                           that many resident CTAs per SM; 11 = compact kernel
                           (upper tree levels on one warp, strains updated by
                           the Newton step), FP64 (mixed: as 12); 12, 13, 14
                           = compact mixed kernel for 2, 3 or 4 CTAs per SM.  The
                           2..4 choice has no effect in FP64.  22, 23, 24 =
                           one warp per Gauss point (lane l condenses the
                           subtree under level-6 node l in registers, levels
                           5..1 by shuffles; four points per CTA, register
                           budget for 2, 3 or 4 CTAs per SM): mixed
                           precision, 6 <= K <= 8, thermoelastic and J2
                           leaves only, else dmn_create returns DMN_ERR_ARG;
                           the handle then also owns a scratch buffer of
                           (2^(K-5) - 1) x 21 floats per lane of every
                           resident warp (about 22 MB at K = 8 on 152 SMs)
                           and dmn_eval_noalloc rejects these variants.  Any
                           other value is DMN_ERR_ARG.  Chosen by the
                           autotuner                                          */
} dmn_options;

/* Fill *opt with the defaults listed above. */
void dmn_default_options(dmn_options *opt);

/*
 * Create a DMN handle (Sec. 3.1 tree; Sec. 4 phase laws).
 *   K          tree depth, 1..10 (2^K leaves, 2^K - 1 laminates).
 *   leaf_w     host, 2^K weights w_{K+1}^i, each > 0, summing to 1 within
 *              1e-12 (Sec. 3.1 constraint; zero weights are rejected).
 *   normals    host, (2^K - 1) x 3 lamination directions in the paper's
 *              order; normalised on create, zero vectors rejected.
 *   phase_map  host, 2^K indices into mats (the paper alternates two phases;
 *              any map is accepted).
 *   mats       host, n_mats materials, 1 <= n_mats <= 16.
 *   opt        host options; NULL selects the defaults.
 * Copies everything to device memory of the current device.
 */
dmn_status dmn_create(dmn_handle *out, int32_t K, const double *leaf_w, const double *normals,
                      const uint8_t *phase_map, const dmn_material *mats, int32_t n_mats,
                      const dmn_options *opt);

dmn_status dmn_destroy(dmn_handle h);

/*
 * Device state of one Gauss point: state_words() doubles, 16-byte aligned.
 *   [0..5]   eps_bar^n  (macro strain, Mandel)
 *   [6]      theta^n    (K)
 *   [7]      reserved (0)
 *   [8 .. 8+3(2^K-1))  jump vectors a^n, node order as above, (x, y, z) each
 *   then, for every leaf j in order whose material has internal variables:
 *            DMN_MAT_J2_LINEAR: eps_p (6), p; DMN_MAT_J2_PERZYNA: eps_p (6), p,
 *            the leaf strain (6); DMN_MAT_PA66: eps_vp (6), p, eps_v,1 .. eps_v,12
 *            (6 each), all Mandel; p is the accumulated plastic strain
 *   padded to an even number of words.
 * A batch is n_points such blocks back to back.
 */
int64_t dmn_state_words(dmn_handle h);

/* Initial state: eps_bar = 0, a = 0, internal variables 0, theta^n =
   d_theta0[i] (device, n_points doubles). */
dmn_status dmn_state_init(dmn_handle h, double *d_state, int64_t n_points, const double *d_theta0,
                          dmn_stream stream);

/*
 * One load increment at every point (Algorithm 1).
 *   d_deps     n x 6 macro strain increments (eps_bar^{n+1} = eps_bar^n + deps)
 *   d_theta    n absolute temperatures theta^{n+1} (K), > 0
 *   dt         time increment (s), > 0: rates in D and Diss are (x^{n+1}-x^n)/dt
 *   d_state_in   n x state_words: z^n, a^n, eps_bar^n, theta^n (read only)
 *   d_state_out  n x state_words: written with the converged state; may not
 *                alias d_state_in (a macro solver re-calls with the same
 *                state_in until its global iteration converges)
 *   d_out      n x 57 doubles, per point:
 *                [0..5]   sigma_bar                     (eq. effective stress)
 *                [6..41]  C_algo = d sigma_bar/d eps_bar (eq. ddsdde), 6x6
 *                [42..47] d sigma_bar / d theta          (eq. ddsddt)
 *                [48]     coupling term D_bar            (eq. effective coupling)
 *                [49..54] d D_bar / d eps_bar            (eq. drplde)
 *                [55]     d D_bar / d theta              (eq. drpldt)
 *                [56]     dissipation                    (eq. effective dissipation)
 *   d_status   n int32 per-point codes (DMN_PT_*)
 *   d_iters    n int32 Newton iterations taken
 * The phase coupling term of a J2 leaf is
 *   D = [-3 K alpha theta tr(eps - eps^n) + sigma_Y(theta) dp] / dt
 * and its dissipation sigma_Y(theta) dp / dt (discrete form of Sec. 4).
 */
dmn_status dmn_eval(dmn_handle h, dmn_stream stream, int64_t n_points, const double *d_deps,
                    const double *d_theta, double dt, const double *d_state_in,
                    double *d_state_out, double *d_out, int32_t *d_status, int32_t *d_iters);

/*
 * One load increment without any device allocation (the paper has no
 * counterpart: this is an interface for callers that cannot allocate).
 * Some callers may not call cudaMalloc at all -- a material routine running
 * inside a host finite-element code whose device memory belongs to another
 * allocator or pool, a sandboxed or real-time plug-in, or code that cannot
 * keep a dmn_handle alive between calls.  This call needs no handle: it takes
 * the tree and materials as dmn_create does (host memory, same rules), derives
 * the node tables on the host every call, copies them into a fixed device
 * array that is part of the library (64 KiB per GPU, held by every GPU that
 * loads the library until the process exits) and then runs the same solve as
 * dmn_eval; the caller's inputs, outputs and state are as in dmn_eval.
 *   Limit: K <= 8; larger trees, and trees with PA66 leaves (which need the
 *   per-leaf history offsets a dmn_handle keeps), are rejected with
 *   DMN_ERR_ARG.
 *   The first call on a device looks up the device address of that array
 *   (with the device current).  The host-to-device copies of the tables are
 *   ordinary stream-ordered copies from host memory.
 *   All calls share the one array (tables and the work-queue counter, which
 *   each launch zeroes first): calls that overlap on the GPU -- on different
 *   streams, or from different threads -- race; order them on one stream.
 * Calls no cudaMalloc, cudaFree or other allocating routine.
 */
dmn_status dmn_eval_noalloc(int32_t K, const double *leaf_w, const double *normals,
                            const uint8_t *phase_map, const dmn_material *mats, int32_t n_mats,
                            const dmn_options *opt, dmn_stream stream, int64_t n_points,
                            const double *d_deps, const double *d_theta, double dt,
                            const double *d_state_in, double *d_state_out, double *d_out,
                            int32_t *d_status, int32_t *d_iters);

/*
 * Index-check log of the debug library (no counterpart in the paper).  The
 * library can be built a second time with bounds checks (libdmn_debug.so,
 * compile flag DMN_BOUNDS_CHECK): every node, leaf, point, state-offset and
 * shared-memory slot index of the solve kernels is checked; an index out of
 * range is counted, replaced by 0 (the access stays inside its array) and
 * gives the point being evaluated the status bit DMN_PT_BOUNDS -- nothing
 * traps.  This call copies the log out (synchronous):
 *   *count  violations since the last clear (summed over the kernels)
 *   *index, *bound, *line  the first one's index, bound and source line
 *           (pointers may be NULL)
 *   clear   nonzero: reset the log afterwards
 * The release library has no checks and returns DMN_ERR_ARG.
 */
enum { DMN_PT_BOUNDS = 16 };
dmn_status dmn_debug_bounds_log(int64_t *count, int64_t *index, int64_t *bound, int32_t *line,
                                int32_t clear);

/* Message of the last failed call on this thread ("" if none). */
const char *dmn_last_error(void);

/*
 * Mixed strain / stress control with optional adiabatic heating: one load
 * increment at every point.  No function of the paper has this form; it
 * closes, around Algorithm 1, the conditions of the paper's validation runs
 * (Sec. 5.4: mixed boundary conditions, stress-free perpendicular to the
 * load; Sec. 5.5: stress-controlled cyclic loading under adiabatic
 * conditions).
 *   d_mask     n uint8 (device): bit c (0..5) set = Mandel stress component c
 *              is prescribed, clear = the strain increment of component c
 *              is; bit 6 set = adiabatic, theta^{n+1} solves
 *              c_heat (theta^{n+1} - theta^n) / dt = D_bar; clear = theta^{n+1}
 *              is prescribed
 *   d_target   n x 6: the prescribed sigma_bar_c (MPa) or deps_c per component
 *   d_deps     n x 6, in: a start for the unknown increments (the prescribed
 *              ones are taken from d_target); out: the increments found
 *   d_theta    n, in: theta^{n+1} if prescribed, else a start; out: found
 *   dt, c_heat time increment (s) and volumetric heat capacity (MPa/K, i.e.
 *              1e-6 J/(m^3 K)), both > 0
 *   max_outer  evaluations at most (>= 1); tol_outer (> 0): a point is done
 *              when every prescribed stress is within tol_outer max(|sigma_bar|,
 *              1 MPa) of its target and the heat balance within
 *              tol_outer c_heat (1 K) / dt
 *   d_state_in, d_state_out, d_out, d_status, d_iters: as dmn_eval, holding
 *              the point's last evaluation; d_status also gets
 *              DMN_PT_OUTER_NOT_CONVERGED
 *   d_outer    n int32: evaluations of the point until it was settled (met
 *              the conditions, or was given up); later evaluations skip it
 *   d_work     NULL, or n x 3(2^K-1) floats of scratch: each evaluation after
 *              the first then starts from the previous one's jumps
 *              (dmn_eval_warm), else from a^n
 *   flags      0 or DMN_MIXED_PREDICT: d_out holds, on entry, the outputs of
 *              the increment that ended in d_state_in; the first evaluation
 *              then starts from the solution of the linear model its stress
 *              and tangents give (sigma^n + C deps + C_theta (theta -
 *              theta^n), D ~ D_eps . deps + D_theta (theta - theta^n)) instead
 *              of the d_deps / d_theta given
 * Outer Newton on x = (unknown strain increments, theta^{n+1} if adiabatic)
 * with the algorithmic tangents d sigma_bar/d eps_bar, d sigma_bar/d theta,
 * d D_bar/d eps_bar and d D_bar/d theta (FP64 LU with partial pivoting, one
 * system of at most 7 unknowns per point).  The stream is synchronised once
 * per evaluation to stop when every point is done.
 */
enum { DMN_MIXED_PREDICT = 1 };
dmn_status dmn_eval_mixed(dmn_handle h, dmn_stream stream, int64_t n_points, const uint8_t *d_mask,
                          const double *d_target, double *d_deps, double *d_theta, double dt,
                          double c_heat, int32_t max_outer, double tol_outer,
                          const double *d_state_in, double *d_state_out, double *d_out,
                          int32_t *d_status, int32_t *d_iters, int32_t *d_outer, float *d_work,
                          int32_t flags);

#ifdef __cplusplus
}
#endif
#endif /* DMN_H_ */
