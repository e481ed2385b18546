// dmn_drive.cu -- device side of dmn_eval_mixed (include/dmn.h): prescribed
// strain components, and the per-point outer Newton update of the unknown
// strain increments and temperature from the algorithmic tangents that
// Algorithm 1 returns (arXiv 2109.14403, eqs. ddsdde, ddsddt, drplde, drpldt).
#include "dmn_internal.h"

namespace dmn {
namespace {

// LU with partial pivoting on an m x m system (m <= 7), in place; false when
// a pivot vanishes
__device__ bool small_solve(double A[7][7], double b[7], int m) {
  for (int k = 0; k < m; ++k) {
    int piv = k;
    double best = fabs(A[k][k]);
    for (int r = k + 1; r < m; ++r)
      if (fabs(A[r][k]) > best) {
        best = fabs(A[r][k]);
        piv = r;
      }
    if (!(best > 0.0)) return false;
    if (piv != k) {
      for (int c = 0; c < m; ++c) {
        const double t = A[k][c];
        A[k][c] = A[piv][c];
        A[piv][c] = t;
      }
      const double t = b[k];
      b[k] = b[piv];
      b[piv] = t;
    }
    for (int r = k + 1; r < m; ++r) {
      const double f = A[r][k] / A[k][k];
      for (int c = k; c < m; ++c) A[r][c] -= f * A[k][c];
      b[r] -= f * b[k];
    }
  }
  for (int k = m - 1; k >= 0; --k) {
    double s = b[k];
    for (int c = k + 1; c < m; ++c) s -= A[k][c] * b[c];
    b[k] = s / A[k][k];
  }
  return true;
}

// Unknowns of a point under mask m: the stress-prescribed components (bits
// 0..5) in order, then theta when adiabatic (bit 6); returns their number.
__device__ int unknowns(unsigned m, int unk[7]) {
  int nu = 0;
  for (int c = 0; c < 6; ++c)
    if ((m >> c) & 1u) unk[nu++] = c;
  if ((m >> 6) & 1u) unk[nu++] = 6;
  return nu;
}

// One Newton step on the unknowns: r holds the residuals (stress rows, then
// the heat balance c (theta - theta^n)/dt - D_bar), o the outputs whose
// tangents form the Jacobian.  Adds the step to deps / theta; false when the
// system is singular (nothing changed).
__device__ bool newton_step(const int unk[7], int nu, const double *o, double c_heat, double dt,
                            const double r[7], double *deps, double *theta) {
  double A[7][7], b[7];
  for (int a = 0; a < nu; ++a) {
    for (int q = 0; q < nu; ++q) {
      const int ra = unk[a], cq = unk[q];
      double v;
      if (ra < 6) v = cq < 6 ? o[6 + 6 * ra + cq] : o[42 + ra];  // d sigma / d eps, d sigma / d theta
      else v = cq < 6 ? -o[49 + cq] : c_heat / dt - o[55];       // heat balance
      A[a][q] = v;
    }
    b[a] = -r[a];
  }
  if (!small_solve(A, b, nu)) return false;
  for (int a = 0; a < nu; ++a)
    if (!isfinite(b[a])) return false;
  for (int a = 0; a < nu; ++a) {
    if (unk[a] < 6) deps[unk[a]] += b[a];
    else *theta += b[a];
  }
  return true;
}

// Prescribed strain components and outer = 0.  With predict, the outputs in
// out are those of the increment that ended in state_in (stress and tangents
// at theta^n); the start is the solution of the linear model they give,
//   sigma ~ sigma^n + C deps + C_theta (theta - theta^n),
//   D ~ D_eps . deps + D_theta (theta - theta^n),
// for the prescribed stresses and the heat balance.
__global__ void k_mixed_prepare(int64_t n, int sw, const uint8_t *mask, const double *target,
                                double *deps, double *theta, double dt, double c_heat,
                                const double *sin, const double *out, int predict, int32_t *outer) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const unsigned m = mask[i];
    double *e = deps + i * 6;
    const double *tg = target + i * 6;
    for (int c = 0; c < 6; ++c)
      if (!((m >> c) & 1u)) e[c] = tg[c];
    outer[i] = 0;
    int unk[7];
    const int nu = unknowns(m, unk);
    if (!predict || nu == 0) continue;
    const double *o = out + i * 57;
    const double thn = sin[i * sw + 6];
    const bool adiabatic = (m >> 6) & 1u;
    double x[6], th = adiabatic ? thn : theta[i];
    for (int c = 0; c < 6; ++c) x[c] = ((m >> c) & 1u) ? 0.0 : tg[c];
    double r[7];
    for (int a = 0; a < nu; ++a) {
      const int c = unk[a];
      double v;
      if (c < 6) {
        v = o[c] - tg[c] + o[42 + c] * (th - thn);
        for (int q = 0; q < 6; ++q) v += o[6 + 6 * c + q] * x[q];
      } else {
        v = (c_heat / dt - o[55]) * (th - thn);
        for (int q = 0; q < 6; ++q) v -= o[49 + q] * x[q];
      }
      r[a] = v;
    }
    if (newton_step(unk, nu, o, c_heat, dt, r, x, &th)) {
      for (int c = 0; c < 6; ++c) e[c] = x[c];
      theta[i] = th;
    }
  }
}

// Residuals of the prescribed stresses and of the heat balance at the last
// evaluation; a point that meets them is done (outer = +evaluations), one that
// cannot go on is given up (outer = -evaluations), any other takes one Newton
// step on (unknown deps components, theta) and is counted in *open.  Also
// writes the next evaluation's warm-start increment (its a - a^n).
__global__ void k_mixed_update(int64_t n, int sw, int n3, const uint8_t *mask, const double *target,
                               double *deps, double *theta, double dt, double c_heat, double tol,
                               const double *sin, const double *sout, const double *out,
                               const int32_t *status, int32_t *outer, int it, int last, float *work,
                               unsigned long long *open) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    if (work)
      for (int j = 0; j < n3; ++j)
        work[i * n3 + j] = float(sout[i * sw + 8 + j] - sin[i * sw + 8 + j]);
    if (outer[i] != 0) continue;  // settled in an earlier evaluation
    const unsigned m = mask[i];
    const double *o = out + i * 57;
    if (status[i] & (DMN_PT_NOT_CONVERGED | DMN_PT_NONFINITE)) {  // Algorithm 1 failed
      outer[i] = -(it + 1);
      continue;
    }
    double smax = 1.0;
    for (int c = 0; c < 6; ++c) smax = fmax(smax, fabs(o[c]));
    int unk[7];
    const int nu = unknowns(m, unk);
    double r[7];
    bool ok = true;
    for (int a = 0; a < nu; ++a) {
      const int c = unk[a];
      if (c < 6) {
        r[a] = o[c] - target[i * 6 + c];
        if (!(fabs(r[a]) <= tol * smax)) ok = false;
      } else {
        r[a] = c_heat * (theta[i] - sin[i * sw + 6]) / dt - o[48];
        if (!(fabs(r[a]) <= tol * c_heat / dt)) ok = false;
      }
    }
    if (ok) {
      outer[i] = it + 1;
      continue;
    }
    if (last) {
      outer[i] = -(it + 1);
      continue;
    }
    if (!newton_step(unk, nu, o, c_heat, dt, r, deps + i * 6, theta + i)) {
      outer[i] = -(it + 1);
      continue;
    }
    atomicAdd(open, 1ull);
  }
}

// the status bit of the given-up points; outer becomes the evaluation count
__global__ void k_mixed_finish(int64_t n, int32_t *status, int32_t *outer) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    if (outer[i] < 0) {
      status[i] |= DMN_PT_OUTER_NOT_CONVERGED;
      outer[i] = -outer[i];
    }
}

int blocks_for(int64_t n) {
  int64_t b = (n + 127) / 128;
  return int(b > 65535 ? 65535 : (b < 1 ? 1 : b));
}

}  // namespace

cudaError_t mixed_prepare(cudaStream_t s, int64_t n, int sw, const uint8_t *mask,
                          const double *target, double *deps, double *theta, double dt,
                          double c_heat, const double *sin, const double *out, bool predict,
                          int32_t *outer) {
  k_mixed_prepare<<<blocks_for(n), 128, 0, s>>>(n, sw, mask, target, deps, theta, dt, c_heat, sin,
                                                out, predict ? 1 : 0, outer);
  return cudaGetLastError();
}

cudaError_t mixed_update(cudaStream_t s, int64_t n, int sw, int n3, const uint8_t *mask,
                         const double *target, double *deps, double *theta, double dt, double c_heat,
                         double tol, const double *sin, const double *sout, const double *out,
                         const int32_t *status, int32_t *outer, int it, bool last, float *work,
                         unsigned long long *open) {
  k_mixed_update<<<blocks_for(n), 128, 0, s>>>(n, sw, n3, mask, target, deps, theta, dt, c_heat, tol,
                                               sin, sout, out, status, outer, it, last ? 1 : 0, work,
                                               open);
  return cudaGetLastError();
}

cudaError_t mixed_finish(cudaStream_t s, int64_t n, int32_t *status, int32_t *outer) {
  k_mixed_finish<<<blocks_for(n), 128, 0, s>>>(n, status, outer);
  return cudaGetLastError();
}

}  // namespace dmn
