// dmn_drive.cu -- device side of dmn_eval_mixed (include/dmn.h): prescribed
// strain components, and the per-point outer Newton update of the unknown
// strain increments and temperature from the algorithmic tangents that
// Algorithm 1 returns (arXiv 2109.14403, eqs. ddsdde, ddsddt, drplde, drpldt).
#include "dmn_internal.h"

namespace dmn {
namespace {

__global__ void k_mixed_prepare(int64_t n, const uint8_t *mask, const double *target, double *deps,
                                int32_t *outer) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const unsigned m = mask[i];
    for (int c = 0; c < 6; ++c)
      if (!((m >> c) & 1u)) deps[i * 6 + c] = target[i * 6 + c];
    outer[i] = 0;
  }
}

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
    int unk[7], nu = 0;
    double r[7];
    bool ok = true;
    for (int c = 0; c < 6; ++c)
      if ((m >> c) & 1u) {
        r[nu] = o[c] - target[i * 6 + c];
        if (!(fabs(r[nu]) <= tol * smax)) ok = false;
        unk[nu++] = c;
      }
    const double thn = sin[i * sw + 6];
    if ((m >> 6) & 1u) {
      r[nu] = c_heat * (theta[i] - thn) / dt - o[48];
      if (!(fabs(r[nu]) <= tol * c_heat / dt)) ok = false;
      unk[nu++] = 6;
    }
    if (ok) {
      outer[i] = it + 1;
      continue;
    }
    if (last) {
      outer[i] = -(it + 1);
      continue;
    }
    double A[7][7], b[7];
    for (int a = 0; a < nu; ++a) {
      for (int q = 0; q < nu; ++q) {
        const int ra = unk[a], cq = unk[q];
        double v;
        if (ra < 6) v = cq < 6 ? o[6 + 6 * ra + cq] : o[42 + ra];      // d sigma / d eps, d sigma / d theta
        else v = cq < 6 ? -o[49 + cq] : c_heat / dt - o[55];           // heat balance
        A[a][q] = v;
      }
      b[a] = -r[a];
    }
    if (!small_solve(A, b, nu)) {
      outer[i] = -(it + 1);
      continue;
    }
    for (int a = 0; a < nu; ++a) {
      if (unk[a] < 6) deps[i * 6 + unk[a]] += b[a];
      else theta[i] += b[a];
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

cudaError_t mixed_prepare(cudaStream_t s, int64_t n, const uint8_t *mask, const double *target,
                          double *deps, int32_t *outer) {
  k_mixed_prepare<<<blocks_for(n), 128, 0, s>>>(n, mask, target, deps, outer);
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
