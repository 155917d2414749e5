// Double-float ("df") arithmetic on the FP32 pipes: a real number is carried as an unevaluated
// sum hi + lo of two floats (|lo| <= ulp(hi)/2), giving a ~48-bit significand.  Built from the
// error-free transformations TwoSum (Knuth) and TwoProduct via FMA (Ogita, Rump & Oishi 2005).
// Every operation uses the _rn intrinsics so that the compiler neither contracts nor reorders it.
#pragma once

#include "mgh_common.cuh"

namespace mgh {

struct df { float hi, lo; };

// Complex df value in register form.
struct cdf { df re, im; };

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// acc += x * y for df x, y; the hi part is summed exactly by TwoSum, every rounding error
// (of the product and of the sum) is gathered in acc.lo.  acc is left unnormalised.
__device__ __forceinline__ void df_fma(df& acc, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  float e = __fmaf_rn(xh, yh, -p);
  e = __fmaf_rn(xh, yl, e);
  e = __fmaf_rn(xl, yh, e);
  float s, t;
  two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}

// acc += x * y for df x and a float y (exact input).
__device__ __forceinline__ void df_fma1(df& acc, float xh, float xl, float y) {
  const float p = __fmul_rn(xh, y);
  float e = __fmaf_rn(xh, y, -p);
  e = __fmaf_rn(xl, y, e);
  float s, t;
  two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}

// acc += y (float, exact input)
__device__ __forceinline__ void df_add1(df& acc, float y) {
  float s, t;
  two_sum(acc.hi, y, s, t);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, t);
}

__device__ __forceinline__ df df_norm(df a) {
  df r;
  two_sum(a.hi, a.lo, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__host__ __device__ __forceinline__ df df_from_double(double x) {
  df r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}

// acc += conj(q) * u
__device__ __forceinline__ void cdf_dot_acc(cdf& acc, const cdf& q, const cdf& u) {
  df_fma(acc.re, q.re.hi, q.re.lo, u.re.hi, u.re.lo);
  df_fma(acc.re, q.im.hi, q.im.lo, u.im.hi, u.im.lo);
  df_fma(acc.im, q.re.hi, q.re.lo, u.im.hi, u.im.lo);
  df_fma(acc.im, -q.im.hi, -q.im.lo, u.re.hi, u.re.lo);
}

// u -= c * q  (c given as a complex df coefficient)
__device__ __forceinline__ void cdf_sub_mul(cdf& u, const cdf& c, const cdf& q) {
  df_fma(u.re, -c.re.hi, -c.re.lo, q.re.hi, q.re.lo);
  df_fma(u.re, c.im.hi, c.im.lo, q.im.hi, q.im.lo);
  df_fma(u.im, -c.re.hi, -c.re.lo, q.im.hi, q.im.lo);
  df_fma(u.im, -c.im.hi, -c.im.lo, q.re.hi, q.re.lo);
}

// ||u||^2 contribution in df
__device__ __forceinline__ void cdf_abs2_acc(df& acc, const cdf& u) {
  df_fma(acc, u.re.hi, u.re.lo, u.re.hi, u.re.lo);
  df_fma(acc, u.im.hi, u.im.lo, u.im.hi, u.im.lo);
}

// A complex df field is stored as two planes of float2: hi = (re.hi, im.hi) and lo = (re.lo,
// im.lo), each N points long, so a reader that needs only FP32 accuracy reads the hi plane alone.
__device__ __forceinline__ cdf cdf_load(const float2* __restrict__ hi, const float2* __restrict__ lo, size_t q) {
  const float2 a = hi[q], b = lo[q];
  cdf r;
  r.re.hi = a.x; r.im.hi = a.y; r.re.lo = b.x; r.im.lo = b.y;
  return r;
}

__device__ __forceinline__ void cdf_store(float2* __restrict__ hi, float2* __restrict__ lo, size_t q, cdf v) {
  const df re = df_norm(v.re), im = df_norm(v.im);
  hi[q] = make_float2(re.hi, im.hi);
  lo[q] = make_float2(re.lo, im.lo);
}

__device__ __forceinline__ cdf cdf_zero() {
  cdf r;
  r.re.hi = r.re.lo = r.im.hi = r.im.lo = 0.f;
  return r;
}

__device__ __forceinline__ cdf cdf_from(cd v) {
  cdf r;
  r.re = df_from_double(v.re);
  r.im = df_from_double(v.im);
  return r;
}

__device__ __forceinline__ cd cdf_to_cd(const cdf& v) { return mk<double>(df_to_double(v.re), df_to_double(v.im)); }

}  // namespace mgh
