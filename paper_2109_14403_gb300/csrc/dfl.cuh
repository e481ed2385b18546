// dfl.cuh -- float-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits (relative rounding ~2^-46 per operation).  GB300's
// FP64 pipe issues at 1/61 of the FP32 rate, so the mixed-precision solve
// carries its high-precision quantities (strains, leaf stresses, subtree
// stress sums, residual) in this form.
//
// Building blocks (error-free transformations):
//   two_sum   Knuth, TAOCP vol. 2, 4.2.2: s + e = a + b exactly, any a, b;
//   fast_two  Dekker (1971): the same when |a| >= |b| (or a == 0);
//   two_prod  with a fused multiply-add: p + e = a * b exactly.
// Sums and products below follow Dekker's double-length algorithms (add,
// mul); the square root and the quotient take the CUDA single-precision
// result as a first approximation and apply one Newton correction computed
// in float-float (Karp and Markstein's refinement).
//
// These sequences must not be re-associated: the library is compiled without
// fast-math flags, so the compiler keeps every rounding as written.
#pragma once
#include <cuda_runtime.h>

namespace dmn {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ dfl fast_two(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dfl two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ dfl operator+(dfl x, dfl y) {
  const dfl s = two_sum(x.hi, y.hi);
  return fast_two(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ dfl operator-(dfl x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dfl operator-(dfl x, dfl y) { return x + (-y); }
__device__ __forceinline__ dfl operator*(dfl x, dfl y) {
  dfl p = two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
  return fast_two(p.hi, p.lo);
}
__device__ __forceinline__ dfl operator*(dfl x, float c) {
  dfl p = two_prod(x.hi, c);
  p.lo = fmaf(x.lo, c, p.lo);
  return fast_two(p.hi, p.lo);
}
__device__ __forceinline__ dfl &operator+=(dfl &x, dfl y) { return x = x + y; }
__device__ __forceinline__ dfl &operator-=(dfl &x, dfl y) { return x = x - y; }

// exact split of a double (FP64 conversions: used at loads only)
__device__ __forceinline__ dfl dfl_from(double d) {
  const float h = __double2float_rn(d);
  return {h, __double2float_rn(d - double(h))};
}
__device__ __forceinline__ double dfl_to(dfl x) { return double(x.hi) + double(x.lo); }

// the FP64 conversion as a call, so that it is a branch that only the lanes
// needing it take (not an if-converted sequence every lane issues)
static __device__ __noinline__ dfl dfl_from_call(double d) { return dfl_from(d); }

// The same split by integer operations only (no FP64 pipe): hi keeps the
// leading 24 significand bits of d (truncated), lo the next 29 bits rounded
// to a float; a final fast_two renormalises.  Zero (and double subnormals)
// give zero; magnitudes outside [2^-74, 2^127) take the FP64 conversion.
__device__ __forceinline__ dfl dfl_split(double d) {
  const long long b = __double_as_longlong(d);
  const int E = int((b >> 52) & 0x7ff);
  if (E == 0) return dfl{0.0f, 0.0f};
  if (E < 949 || E >= 1150) return dfl_from_call(d);
  const unsigned sign = unsigned(b >> 32) & 0x80000000u;
  const long long mant = b & ((1ll << 52) - 1);
  const float hi = __uint_as_float(sign | (unsigned(E - 1023 + 127) << 23) | unsigned(mant >> 29));
  const float scale = __uint_as_float(unsigned(E - 1075 + 127) << 23);  // 2^(E-1075)
  float lo = float(int(mant & ((1ll << 29) - 1))) * scale;
  if (sign) lo = -lo;
  return fast_two(hi, lo);
}

__device__ __forceinline__ dfl dfl_sqrt(dfl x) {
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
  const float y = sqrtf(x.hi);
  const dfl y2 = two_prod(y, y);
  const float r = ((x.hi - y2.hi) - y2.lo) + x.lo;  // x - y^2 (leading part exact)
  return fast_two(y, r / (y + y));
}
__device__ __forceinline__ dfl dfl_div(dfl a, dfl b) {
  const float q1 = a.hi / b.hi;
  const dfl r = a - b * q1;
  return fast_two(q1, r.hi / b.hi);
}

// ---------------------------------------------------------------- generic
// The solve is written once for the high-precision type HP = double (every
// step FP64) or HP = dfl (mixed).  These overloads give both the same names.
__device__ __forceinline__ double hp_from(double d, double *) { return d; }
__device__ __forceinline__ dfl hp_from(double d, dfl *) { return dfl_from(d); }
// load-path conversion (integer split for float-float)
__device__ __forceinline__ double hp_load(double d, double *) { return d; }
__device__ __forceinline__ dfl hp_load(double d, dfl *) { return dfl_split(d); }
__device__ __forceinline__ double hp_to(double x) { return x; }
__device__ __forceinline__ double hp_to(dfl x) { return dfl_to(x); }
__device__ __forceinline__ double hp_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ dfl hp_sqrt(dfl x) { return dfl_sqrt(x); }
__device__ __forceinline__ double hp_div(double a, double b) { return a / b; }
__device__ __forceinline__ dfl hp_div(dfl a, dfl b) { return dfl_div(a, b); }
// leading part as a float (for quantities needed only to FP32 accuracy)
__device__ __forceinline__ float hp_f(double x) { return float(x); }
__device__ __forceinline__ float hp_f(dfl x) { return x.hi; }
// value in the condensation precision TF (double for HP = double, float for dfl)
__device__ __forceinline__ double tf_of(double x, double *) { return x; }
__device__ __forceinline__ float tf_of(dfl x, float *) { return x.hi; }
__device__ __forceinline__ double hp_d(double x) { return x; }
__device__ __forceinline__ double hp_d(dfl x) { return double(x.hi); }
// a + d with d in the condensation precision (float-float + float, or double)
__device__ __forceinline__ double hp_add_tf(double a, double d) { return a + d; }
__device__ __forceinline__ dfl hp_add_tf(dfl a, float d) { return a + dfl{d, 0.0f}; }
__device__ __forceinline__ double hp_zero(double *) { return 0.0; }
__device__ __forceinline__ dfl hp_zero(dfl *) { return {0.0f, 0.0f}; }
// x > y exactly (hi dominates lo)
__device__ __forceinline__ bool hp_gt(double x, double y) { return x > y; }
__device__ __forceinline__ bool hp_gt(dfl x, dfl y) {
  return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo);
}
// shuffles
__device__ __forceinline__ float hp_shfl_down(unsigned m, float v, int o, int w) {
  return __shfl_down_sync(m, v, o, w);
}
__device__ __forceinline__ double hp_shfl_down(unsigned m, double v, int o, int w) {
  return __shfl_down_sync(m, v, o, w);
}
__device__ __forceinline__ dfl hp_shfl_down(unsigned m, dfl v, int o, int w) {
  return {__shfl_down_sync(m, v.hi, o, w), __shfl_down_sync(m, v.lo, o, w)};
}
__device__ __forceinline__ float hp_shfl(unsigned m, float v, int src, int w) {
  return __shfl_sync(m, v, src, w);
}
__device__ __forceinline__ double hp_shfl(unsigned m, double v, int src, int w) {
  return __shfl_sync(m, v, src, w);
}
__device__ __forceinline__ dfl hp_shfl(unsigned m, dfl v, int src, int w) {
  return {__shfl_sync(m, v.hi, src, w), __shfl_sync(m, v.lo, src, w)};
}

}  // namespace dmn
