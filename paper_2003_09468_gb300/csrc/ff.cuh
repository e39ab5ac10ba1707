// Double-float ("float-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two fp32 numbers with |lo| below one
// ulp of hi: about 48 significant bits, against 53 for FP64.  The FP64 pipe of
// this GPU issues about two fused multiply-adds per clock per SM, the FP32 pipe
// 128, so a double-float multiply-add of some fifteen FP32 instructions still
// runs several times faster than FP64.  Everything here is built from two
// error-free transformations:
//   TwoSum (Knuth):       s = fl(a + b) and the exact error a + b - s, six additions;
//   TwoProduct (Dekker, in its fused multiply-add form): p = fl(a b) and the exact
//                         error a b - p = fma(a, b, -p).
// The additions and products that feed them use the _rn intrinsics so that the
// compiler never contracts them into a fused multiply-add, which would break the
// exactness of the error terms.
//
// Complex values are packed in a float4 as (re.hi, re.lo, im.hi, im.lo): 16 bytes,
// like an FP64 complex, so one vector access moves one element.
#pragma once

#include <cuda_runtime.h>

namespace ffa {

struct f2 {
  float hi, lo;
};

__device__ __forceinline__ f2 make(float hi, float lo) { return f2{hi, lo}; }
__device__ __forceinline__ f2 neg(f2 x) { return f2{-x.hi, -x.lo}; }

// s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// the same when |a| >= |b| (or a == 0): three additions
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ f2 add(f2 x, f2 y) {
  float s, e, t, g;
  two_sum(x.hi, y.hi, s, e);
  two_sum(x.lo, y.lo, t, g);
  e = __fadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __fadd_rn(e, g);
  fast_two_sum(s, e, s, e);
  return f2{s, e};
}

__device__ __forceinline__ f2 mul(f2 x, f2 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  float s, t;
  fast_two_sum(p, e, s, t);
  return f2{s, t};
}

// a + x y: the product's error terms and a.lo are folded into one correction, the
// leading sum a.hi + fl(x.hi y.hi) is exact through TwoSum
__device__ __forceinline__ f2 fma(f2 a, f2 x, f2 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float pe = fmaf(x.hi, y.hi, -p);
  pe = fmaf(x.hi, y.lo, pe);
  pe = fmaf(x.lo, y.hi, pe);
  float s, e;
  two_sum(a.hi, p, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, pe));
  fast_two_sum(s, e, s, e);
  return f2{s, e};
}

// 1 / d: fp32 reciprocal, then one Newton step r + r (1 - d r) in double-float
__device__ __forceinline__ f2 recip(f2 d) {
  const float r0 = __frcp_rn(d.hi);
  const f2 r = make(r0, 0.f);
  const f2 e = fma(make(1.f, 0.f), neg(d), r);   // 1 - d r0
  return fma(r, r, e);
}

// Split of an FP64 value into hi + lo without the FP64 pipe: hi keeps the leading 24
// bits of the significand (truncated), lo the next 29 bits rounded to 24, so the pair
// carries 48 bits.  Zero, and values outside the fp32 normal range, take a rare
// path; below 2^-74 the low part is dropped (relative precision 2^-24 there).
__device__ __forceinline__ f2 from_double(double x) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  const int eb = static_cast<int>((u >> 52) & 0x7ff);
  if (eb == 0) return f2{0.f, 0.f};
  const int e = eb - 1023;
  if (e < -126 || e > 127) return f2{__double2float_rn(x), 0.f};
  const unsigned sgn = static_cast<unsigned>(u >> 63) << 31;
  const float hi = __uint_as_float(sgn | (static_cast<unsigned>(e + 127) << 23) |
                                   static_cast<unsigned>((u >> 29) & 0x7fffffu));
  float lo = 0.f;
  if (e >= -74) {
    const float scale = __uint_as_float(static_cast<unsigned>(e - 52 + 127) << 23);   // 2^(e-52)
    lo = __fmul_rn(__uint2float_rn(static_cast<unsigned>(u & 0x1fffffffu)), scale);
    if (sgn) lo = -lo;
  }
  return f2{hi, lo};
}
__device__ __forceinline__ double to_double(f2 x) { return (double)x.hi + (double)x.lo; }

// Accumulator for a run of products: value = s + t, kept unnormalised between terms (t
// collects the TwoSum and TwoProduct errors); get() renormalises once at the end.
struct acc {
  float s, t;
};
__device__ __forceinline__ acc acc_from(f2 x) { return acc{x.hi, x.lo}; }
// a += x y
__device__ __forceinline__ void acc_fma(acc& a, f2 x, f2 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  float s, u;
  two_sum(a.s, p, s, u);
  a.s = s;
  a.t = __fadd_rn(a.t, __fadd_rn(u, e));
}
__device__ __forceinline__ f2 acc_get(acc a) {
  float s, e;
  two_sum(a.s, a.t, s, e);   // not fast_two_sum: after cancellation |t| may exceed |s|
  return f2{s, e};
}

// ---------------------------------------------------------------- complex
__device__ __forceinline__ f2 re(float4 v) { return f2{v.x, v.y}; }
__device__ __forceinline__ f2 im(float4 v) { return f2{v.z, v.w}; }
__device__ __forceinline__ float4 pack(f2 r, f2 i) { return make_float4(r.hi, r.lo, i.hi, i.lo); }
__device__ __forceinline__ float4 czero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 cneg(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }
__device__ __forceinline__ float4 cfrom(double2 v) { return pack(from_double(v.x), from_double(v.y)); }

// a + x y
__device__ __forceinline__ float4 cfma(float4 a, float4 x, float4 y) {
  const f2 r = fma(fma(re(a), re(x), re(y)), neg(im(x)), im(y));
  const f2 i = fma(fma(im(a), re(x), im(y)), im(x), re(y));
  return pack(r, i);
}
// a - x y
__device__ __forceinline__ float4 cfms(float4 a, float4 x, float4 y) {
  const f2 r = fma(fma(re(a), neg(re(x)), re(y)), im(x), im(y));
  const f2 i = fma(fma(im(a), neg(re(x)), im(y)), neg(im(x)), re(y));
  return pack(r, i);
}
// complex accumulator (re, im) and a += x y on it
struct cacc {
  acc r, i;
};
__device__ __forceinline__ cacc cacc_from(float4 v) { return cacc{acc_from(re(v)), acc_from(im(v))}; }
__device__ __forceinline__ void cacc_fma(cacc& a, float4 x, float4 y) {
  acc_fma(a.r, re(x), re(y));
  acc_fma(a.r, neg(im(x)), im(y));
  acc_fma(a.i, re(x), im(y));
  acc_fma(a.i, im(x), re(y));
}
// a += conj(x) y
__device__ __forceinline__ void cacc_fma_conj(cacc& a, float4 x, float4 y) {
  acc_fma(a.r, re(x), re(y));
  acc_fma(a.r, im(x), im(y));
  acc_fma(a.i, re(x), im(y));
  acc_fma(a.i, neg(im(x)), re(y));
}
// a -= x y
__device__ __forceinline__ void cacc_fms(cacc& a, float4 x, float4 y) {
  acc_fma(a.r, neg(re(x)), re(y));
  acc_fma(a.r, im(x), im(y));
  acc_fma(a.i, neg(re(x)), im(y));
  acc_fma(a.i, neg(im(x)), re(y));
}
__device__ __forceinline__ float4 cacc_get(cacc a) { return pack(acc_get(a.r), acc_get(a.i)); }

// a + conj(x) y
__device__ __forceinline__ float4 cfma_conj(float4 a, float4 x, float4 y) {
  const f2 r = fma(fma(re(a), re(x), re(y)), im(x), im(y));
  const f2 i = fma(fma(im(a), re(x), im(y)), neg(im(x)), re(y));
  return pack(r, i);
}
__device__ __forceinline__ float4 cmul(float4 x, float4 y) {
  const f2 r = fma(mul(re(x), re(y)), neg(im(x)), im(y));
  const f2 i = fma(mul(re(x), im(y)), im(x), re(y));
  return pack(r, i);
}
// 1 / x = conj(x) / |x|^2
__device__ __forceinline__ float4 crecip(float4 x) {
  const f2 d = fma(mul(re(x), re(x)), im(x), im(x));
  const f2 r = recip(d);
  return pack(mul(re(x), r), neg(mul(im(x), r)));
}

}  // namespace ffa
