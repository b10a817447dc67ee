// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// float32 numbers with |lo| <= ulp(hi)/2 when normalised, about 48 bits of
// significand, computed entirely on the FP32 pipe (GB300's float64 rate is
// 1/64 of its float32 rate).
//
// Built from two error-free transformations:
//   TwoSum (Knuth, The Art of Computer Programming vol. 2, 4.2.2; Moller 1965):
//     s = a + b and e = (a - (s - (s - a))) + (b - (s - a)) give a + b = s + e
//     exactly, for any a, b;
//   FastTwoSum (Dekker 1971), valid when |a| >= |b| (or a = 0):
//     s = a + b, e = b - (s - a);
//   TwoProduct with a fused multiply-add (the FMA form of Dekker's product):
//     p = a b, e = fma(a, b, -p) gives a b = p + e exactly.
// From them: addition adds the high parts exactly, folds in the low parts and
// renormalises (its error is a few 2^-48 of the operands' magnitude, as with
// the "sloppy" double-double addition of Hida, Li and Bailey 2001); the
// product keeps the cross terms hi*lo and drops lo*lo (relative error a few
// 2^-48).  Every operation uses explicitly rounded float intrinsics so that
// the compiler neither contracts nor reassociates them.
#pragma once

#include <cuda_runtime.h>

namespace pycool {

struct dd {
  float hi, lo;
  dd() = default;   // trivial (shared-memory records); dd() value-initialises to zero
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  // nearest double-float to a double (two roundings: hi, then the remainder)
  __host__ __device__ explicit dd(double x) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
  }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = fadd(a, b);
  const float bb = fsub(s, a);
  e = fadd(fsub(a, fsub(s, bb)), fsub(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = fadd(a, b);
  e = fsub(b, fsub(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = fmul(a, b);
  e = ffma(a, b, -p);
}

__device__ __forceinline__ dd dd_norm(float s, float e) {
  dd r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ dd operator+(dd x, dd y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e = fadd(e, fadd(x.lo, y.lo));
  return dd_norm(s, e);
}
__device__ __forceinline__ dd operator-(dd x) { return dd(-x.hi, -x.lo); }
__device__ __forceinline__ dd operator-(dd x, dd y) { return x + (-y); }
__device__ __forceinline__ dd operator+(dd x, float b) {
  float s, e;
  two_sum(x.hi, b, s, e);
  return dd_norm(s, fadd(e, x.lo));
}
__device__ __forceinline__ dd operator*(dd x, dd y) {
  float p, e;
  two_prod(x.hi, y.hi, p, e);
  e = ffma(x.hi, y.lo, e);
  e = ffma(x.lo, y.hi, e);
  return dd_norm(p, e);
}
__device__ __forceinline__ dd operator*(dd x, float b) {
  float p, e;
  two_prod(x.hi, b, p, e);
  e = ffma(x.lo, b, e);
  return dd_norm(p, e);
}
__device__ __forceinline__ dd operator*(float b, dd x) { return x * b; }
// x / y: a float quotient, its residual x - q y formed in double-float, and
// one correction term (relative error a few 2^-46).
__device__ __forceinline__ dd dd_div(dd x, dd y) {
  const float inv = __frcp_rn(y.hi);
  const float q1 = fmul(x.hi, inv);
  const dd r = x - y * q1;
  const float q2 = fmul(r.hi, inv);
  return dd_norm(q1, q2);
}
// x^2 with the cross term counted twice
__device__ __forceinline__ dd dd_sqr(dd x) {
  float p, e;
  two_prod(x.hi, x.hi, p, e);
  e = ffma(fadd(x.hi, x.hi), x.lo, e);
  return dd_norm(p, e);
}
// a b + c in one pass: the product's pieces (TwoProduct and the cross terms)
// go into the sum unnormalised, so only the result is renormalised.
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) {
  float p, e, s, t;
  two_prod(a.hi, b.hi, p, e);
  e = ffma(a.hi, b.lo, e);
  e = ffma(a.lo, b.hi, e);
  two_sum(c.hi, p, s, t);
  t = fadd(t, fadd(c.lo, e));
  return dd_norm(s, t);
}
__device__ __forceinline__ dd dd_fma(float a, dd b, dd c) {
  float p, e, s, t;
  two_prod(a, b.hi, p, e);
  e = ffma(a, b.lo, e);
  two_sum(c.hi, p, s, t);
  t = fadd(t, fadd(c.lo, e));
  return dd_norm(s, t);
}
__device__ __forceinline__ dd madd(dd a, dd b, dd c) { return dd_fma(a, b, c); }

// (a + b) + (c + e) + w x: the high parts added exactly in one chain of
// TwoSums, the low parts and the rounding errors gathered in one float, a
// single renormalisation (the in-plane part of the 7-point Laplacian).
__device__ __forceinline__ dd dd_sum4_axpy(dd a, dd b, dd c, dd e, float w, dd x) {
  float s0, s1, s2, s3, s4, r, t = a.lo, p, pe;
  two_sum(a.hi, b.hi, s1, r);
  t = fadd(t, fadd(r, b.lo));
  two_sum(s1, c.hi, s2, r);
  t = fadd(t, fadd(r, c.lo));
  two_sum(s2, e.hi, s3, r);
  t = fadd(t, fadd(r, e.lo));
  two_prod(w, x.hi, p, pe);
  pe = ffma(w, x.lo, pe);
  two_sum(s3, p, s4, r);
  t = fadd(t, fadd(r, pe));
  s0 = s4;
  return dd_norm(s0, t);
}

__device__ __forceinline__ dd dd_shfl_up(dd v, int d) {
  return dd(__shfl_up_sync(0xffffffffu, v.hi, d), __shfl_up_sync(0xffffffffu, v.lo, d));
}
__device__ __forceinline__ dd dd_shfl_down(dd v, int d) {
  return dd(__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d));
}

// Running sum of double-float terms: the high parts are added exactly
// (TwoSum) into s, their errors and the low parts are gathered in c, and no
// renormalisation happens per term.  Over K terms the gathered part loses
// about K^2 2^-48 of the sum, so the owner empties it into an exact
// double-float total every few terms (fold()).
struct DDAcc {
  float s, c;
  __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
  __device__ __forceinline__ void add(dd x) {
    float t, e;
    two_sum(s, x.hi, t, e);
    c = fadd(c, fadd(e, x.lo));
    s = t;
  }
  // a plain float sum of high parts (for sums whose precision does not matter)
  __device__ __forceinline__ void add_fast(float x) { s = fadd(s, x); }
  // add the product a b (TwoProduct and cross terms, unnormalised)
  __device__ __forceinline__ void add_prod(dd a, dd b) {
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = ffma(a.hi, b.lo, e);
    e = ffma(a.lo, b.hi, e);
    add(dd(p, e));
  }
  __device__ __forceinline__ void add_sqr(dd a) {
    float p, e;
    two_prod(a.hi, a.hi, p, e);
    e = ffma(fadd(a.hi, a.hi), a.lo, e);
    add(dd(p, e));
  }
  // move this running sum into the total t (accurate double-float addition:
  // both parts added with TwoSum), and restart from zero
  __device__ __forceinline__ void fold(dd& t) {
    float s1, e1, s2, e2;
    two_sum(t.hi, s, s1, e1);
    two_sum(t.lo, c, s2, e2);
    e1 = fadd(e1, s2);
    fast_two_sum(s1, e1, s1, e1);
    e1 = fadd(e1, e2);
    fast_two_sum(s1, e1, t.hi, t.lo);
    zero();
  }
};

}  // namespace pycool
