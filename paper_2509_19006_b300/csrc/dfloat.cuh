// Double-float arithmetic: a value is the unevaluated sum hi + lo of two float32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits computed on the FP32
// pipes. On B300 the float64 pipe issues about 1.7 fused multiply-adds per clock per SM
// against 128 float32 ones, so a double-float multiply-add (about 10-20 float32
// operations) runs several times faster than a float64 one while keeping the
// accuracy the beta = 3 truncation needs (unit roundoff 2^-48 against float64's 2^-53
// and float32's 2^-24); the exponent range is float32's.
//
// Building blocks, each exact in float32 arithmetic with round-to-nearest:
//   TwoSum (Knuth, TAOCP vol. 2):   s + e = a + b for any a, b;
//   FastTwoSum (Dekker, 1971):      s + e = a + b when |a| >= |b| (or a = 0);
//   TwoProd with an FMA:            p + e = a * b.
// Double-word addition and multiplication follow Joldes, Muller & Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic", ACM TOMS
// 44 (2017): AccurateDWPlusDW (relative error <= 3u^2 + 13u^3) and a DWTimesDW with
// FMAs (relative error a few u^2), u = 2^-24. Division and square root take one correction step from the
// float32 quotient or root with an exactly computed residual (the scheme of Karp &
// Markstein, "High-precision division and square root", ACM TOMS 23, 1997). Logarithms,
// exponentials and tanh go through float64: they are needed once per site, not per
// tensor element.
#pragma once
#include <cuda_runtime.h>

namespace tnmc {

struct dfloat;
namespace df {
__device__ __forceinline__ dfloat fma(dfloat x, dfloat y, dfloat z);
}

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ dfloat(float x) : hi(x), lo(0.f) {}
  __host__ __device__ dfloat(int x) : hi(float(x)), lo(0.f) {}
  __host__ __device__ dfloat(double x) {
    hi = float(x);
    lo = float(x - double(hi));
  }
  __host__ __device__ explicit operator double() const { return double(hi) + double(lo); }
  __host__ __device__ explicit operator float() const { return hi + lo; }
  // found by argument-dependent lookup only, so they never hide the float and
  // double overloads of the same names
  friend __device__ __forceinline__ dfloat fabs(dfloat a) { return a.hi < 0.f ? dfloat(-a.hi, -a.lo) : a; }
  friend __device__ __forceinline__ bool isfinite(dfloat a) { return ::isfinite(a.hi); }
  friend __device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) { return df::fma(a, b, c); }
};

namespace df {

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  e = b - (s - a);
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  p = a * b;
  e = __fmaf_rn(a, b, -p);
}

// AccurateDWPlusDW
__device__ __forceinline__ dfloat add(dfloat x, dfloat y) {
  float s, t, e, f;
  two_sum(x.hi, y.hi, s, t);
  two_sum(x.lo, y.lo, e, f);
  t += e;
  fast_two_sum(s, t, s, t);
  t += f;
  fast_two_sum(s, t, s, t);
  return dfloat(s, t);
}
// DWTimesDW (FMA form)
__device__ __forceinline__ dfloat mul(dfloat x, dfloat y) {
  float p, e;
  two_prod(x.hi, y.hi, p, e);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  fast_two_sum(p, e, p, e);
  return dfloat(p, e);
}
// double-word times a float32 number
__device__ __forceinline__ dfloat mul(dfloat x, float y) {
  float p, e;
  two_prod(x.hi, y, p, e);
  e = __fmaf_rn(x.lo, y, e);
  fast_two_sum(p, e, p, e);
  return dfloat(p, e);
}
// x * y + z: the product's exact leading part and its error terms, then an accurate sum
__device__ __forceinline__ dfloat fma(dfloat x, dfloat y, dfloat z) {
  float p, e, s, t, g, h;
  two_prod(x.hi, y.hi, p, e);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  two_sum(p, z.hi, s, t);
  two_sum(e, z.lo, g, h);
  t += g;
  fast_two_sum(s, t, s, t);
  t += h;
  fast_two_sum(s, t, s, t);
  return dfloat(s, t);
}
__device__ __forceinline__ dfloat neg(dfloat x) { return dfloat(-x.hi, -x.lo); }

// one correction of the float32 quotient: q = q1 + (x - q1 y) / y
__device__ __forceinline__ dfloat div(dfloat x, dfloat y) {
  const float q1 = __fdiv_rn(x.hi, y.hi);
  const dfloat r = add(x, neg(mul(y, q1)));
  const float q2 = __fdiv_rn(r.hi, y.hi);
  float s, e;
  fast_two_sum(q1, q2, s, e);
  return dfloat(s, e);
}
// one correction of the float32 root: s = s1 + (x - s1^2) / (2 s1)
__device__ __forceinline__ dfloat sqrt(dfloat x) {
  if (!(x.hi > 0.f)) return dfloat(x.hi == 0.f ? 0.f : __fsqrt_rn(x.hi), 0.f);
  const float s1 = __fsqrt_rn(x.hi);
  float p, e;
  two_prod(s1, s1, p, e);
  const dfloat r = add(x, dfloat(-p, -e));
  const float c = __fdiv_rn(r.hi, 2.f * s1);
  float s, t;
  fast_two_sum(s1, c, s, t);
  return dfloat(s, t);
}

// Compensated accumulation of a dot product (Ogita, Rump & Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26, 2005, Dot2, extended to double-word inputs): the
// running sum is kept as hi + lo WITHOUT renormalising, lo collecting the exact
// rounding errors of the TwoSums and the product error terms; finish() renormalises.
// One step costs 12 float32 operations against 24 for a double-word multiply-add, and
// the result is as accurate (error ~ n u^2 sum |x y|, u = 2^-24).
__device__ __forceinline__ void dot_step(dfloat &acc, dfloat x, dfloat y) {
  float p, e, s, t;
  two_prod(x.hi, y.hi, p, e);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo += t + e;
}
__device__ __forceinline__ dfloat finish(dfloat acc) {
  float s, e;
  two_sum(acc.hi, acc.lo, s, e);   // lo may exceed hi after cancellation: not FastTwoSum
  return dfloat(s, e);
}

// c x - s y (a plane rotation's first output) in one pass: both products' leading parts
// exactly, their cross and error terms in float32, and two TwoSums (the second because
// after cancellation the collected errors can exceed the leading difference): 22
// float32 operations against 34 for two double-word products and a difference.
// The error is ~u^2 (|c x| + |s y|), that of float64's c x - s y scaled to 2^-48.
__device__ __forceinline__ dfloat lin2(dfloat c, dfloat x, dfloat s, dfloat y) {
  float p1, e1, p2, e2, h, l;
  two_prod(c.hi, x.hi, p1, e1);
  two_prod(s.hi, y.hi, p2, e2);
  two_sum(p1, -p2, h, l);
  float cross = __fmaf_rn(c.hi, x.lo, __fmaf_rn(c.lo, x.hi, e1 - e2));
  cross = __fmaf_rn(-s.hi, y.lo, __fmaf_rn(-s.lo, y.hi, cross));
  l += cross;
  two_sum(h, l, h, l);
  return dfloat(h, l);
}
// x - w v (a Householder or Gram-Schmidt update) in one pass
__device__ __forceinline__ dfloat axmy(dfloat x, dfloat w, dfloat v) {
  float p, e, h, l;
  two_prod(w.hi, v.hi, p, e);
  two_sum(x.hi, -p, h, l);
  l += x.lo - __fmaf_rn(w.hi, v.lo, __fmaf_rn(w.lo, v.hi, e));
  two_sum(h, l, h, l);
  return dfloat(h, l);
}

// x times a power of two: exact (both words scale)
__device__ __forceinline__ dfloat scale2(dfloat x, float p2) { return dfloat(x.hi * p2, x.lo * p2); }
// The power of two that brings |x| (> 0) into [1, 2), kept inside float32's normal
// range. Double-float has float32's exponent range, so sums of squares of small
// entries (1e-17 of a matrix's norm occur at beta = 3) would otherwise underflow.
__device__ __forceinline__ float unit_scale(float x) {
  int e = (__float_as_int(x) >> 23) & 0xff;
  e = max(1, min(e, 253));
  return __int_as_float((254 - e) << 23);
}

}  // namespace df

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) { return df::add(a, b); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return df::add(a, df::neg(b)); }
__device__ __forceinline__ dfloat operator-(dfloat a) { return df::neg(a); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) { return df::mul(a, b); }
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) { return df::div(a, b); }
__device__ __forceinline__ dfloat &operator+=(dfloat &a, dfloat b) { return a = df::add(a, b); }
__device__ __forceinline__ dfloat &operator-=(dfloat &a, dfloat b) { return a = df::add(a, df::neg(b)); }
__device__ __forceinline__ dfloat &operator*=(dfloat &a, dfloat b) { return a = df::mul(a, b); }
__device__ __forceinline__ bool operator<(dfloat a, dfloat b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(dfloat a, dfloat b) { return b < a; }
__device__ __forceinline__ bool operator<=(dfloat a, dfloat b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(dfloat a, dfloat b) { return !(a < b); }
__device__ __forceinline__ bool operator==(dfloat a, dfloat b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(dfloat a, dfloat b) { return !(a == b); }

// Warp shuffles of float, double and double-float values.
__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ dfloat shfl_xor(dfloat v, int o) {
  return dfloat(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

}  // namespace tnmc
