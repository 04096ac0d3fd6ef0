// Double-float ("double-word") arithmetic on binary32 pairs.
//
// A value is hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits.  The
// building blocks are the classical error-free transformations: Knuth's
// TwoSum, Dekker's FastTwoSum, and the exact product through one fused
// multiply-add; the double-word sum and product follow the algorithms
// analysed by Joldes, Muller and Popescu (ACM TOMS 44(2), 2017, "Tight and
// rigorous error bounds for basic building blocks of double-word
// arithmetic").  Explicit _rn intrinsics keep the compiler from contracting
// or reassociating the transformations.
//
// Used by the mixed-precision path for the point and camera state and for
// the cost evaluation, which would otherwise need binary64 per observation
// (GB300's binary64 rate is 1/59 of its binary32 rate).
#pragma once

#include <cuda_runtime.h>

namespace bagpu {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_make(float v) { return dfl{v, 0.0f}; }

// exact a + b = s + e
__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfl{s, e};
}

// exact a + b = s + e when |a| >= |b| (or a == 0)
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return dfl{s, e};
}

// exact a * b = p + e
__device__ __forceinline__ dfl two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  return dfl{p, e};
}

// double-word + double-word (accurate version)
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  dfl s = two_sum(a.hi, b.hi);
  const dfl t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}

// double-word + double-word, "sloppy" version (Dekker): the low words are
// added without their own TwoSum.  Relative to max(|a|, |b|) the error stays
// near 2^-44, but it is not relative to the result: only for sums without
// heavy cancellation against the needed absolute accuracy.
__device__ __forceinline__ dfl df_add_fast(dfl a, dfl b) {
  const dfl s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }

// double-word + float
__device__ __forceinline__ dfl df_add_f(dfl a, float b) {
  dfl s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return fast_two_sum(s.hi, s.lo);
}

// double-word * double-word
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  dfl p = two_prod(a.hi, b.hi);
  float t = __fmul_rn(a.lo, b.lo);
  t = __fmaf_rn(a.hi, b.lo, t);
  t = __fmaf_rn(a.lo, b.hi, t);
  p.lo = __fadd_rn(p.lo, t);
  return fast_two_sum(p.hi, p.lo);
}

// double-word * float
__device__ __forceinline__ dfl df_mul_f(dfl a, float b) {
  dfl p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// double-word / double-word: one correction step on the binary32 quotient
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const dfl r = df_sub(a, df_mul_f(b, q1));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return fast_two_sum(q1, q2);
}

// 1 / b (b != 0): the binary32 reciprocal r and one Newton correction
// r + r (1 - b r), with 1 - b.hi r exact (TwoProduct, then Sterbenz).
__device__ __forceinline__ dfl df_recip(dfl b) {
  const float r = __frcp_rn(b.hi);
  const dfl p = two_prod(b.hi, r);
  const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p.hi), p.lo), __fmul_rn(b.lo, r));
  return fast_two_sum(r, __fmul_rn(r, e));
}

// sqrt of a double-word (a > 0): one Newton correction
__device__ __forceinline__ dfl df_sqrt(dfl a) {
  const float s = __fsqrt_rn(a.hi);
  const dfl r = df_sub(a, two_prod(s, s));
  const float c = __fdiv_rn(r.hi, __fmul_rn(2.0f, s));
  return fast_two_sum(s, c);
}

// a - x y, the low-order terms added without their own TwoSum (as in
// df_add_fast): the error stays near 2^-47 of max(|a|, |x y|), which is what
// the backward-error analysis of a Cholesky update asks for.
__device__ __forceinline__ dfl df_fms(dfl a, dfl x, dfl y) {
  dfl p = two_prod(x.hi, y.hi);
  p.lo = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
  dfl s = two_sum(a.hi, -p.hi);
  s.lo = __fadd_rn(s.lo, __fsub_rn(a.lo, p.lo));
  return fast_two_sum(s.hi, s.lo);
}

// Compensated dot product of double-float vectors (Ogita, Rump and Oishi,
// SIAM J. Sci. Comput. 26(6), 2005, "Accurate sum and dot product",
// algorithm Dot2, with the low words' cross terms folded into the error
// term): the result is as accurate as if the sum had been formed in twice
// the working precision and then rounded to a double-float.
struct Dot2 {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(dfl x, dfl y) {
    const dfl p = two_prod(x.hi, y.hi);
    const float e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, p.lo));
    const dfl t = two_sum(s, p.hi);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, e));
  }
  // merge another partial sum (the reduction trees of a dot product)
  __device__ __forceinline__ void merge(float s2, float c2) {
    const dfl t = two_sum(s, s2);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, c2));
  }
  __device__ __forceinline__ dfl get() const { return fast_two_sum(s, c); }
};

// 1 / sqrt(d) for d > 0: the binary32 approximation, one binary32 Newton
// step r + r/2 (1 - d r^2), then one in double-float (error about 2^-48).
__device__ __forceinline__ dfl df_rsqrt(dfl d) {
  float r = d.hi < 0x1p-100f ? rsqrtf(d.hi * 0x1p100f) * 0x1p50f : rsqrtf(d.hi);
  const float t = __fmul_rn(d.hi, r);
  const float e = __fmaf_rn(-t, r, 1.0f);
  r = __fmaf_rn(__fmul_rn(0.5f, r), e, r);
  const dfl p = df_mul(d, two_prod(r, r));  // d r^2, near 1
  const float e2 = __fsub_rn(__fsub_rn(1.0f, p.hi), p.lo);
  return fast_two_sum(r, __fmul_rn(__fmul_rn(0.5f, r), e2));
}

__device__ __forceinline__ float df_to_f(dfl a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ double df_to_d(dfl a) { return (double)a.hi + (double)a.lo; }

// binary64 -> double-word (hi = rounded value, lo = rounded remainder)
__device__ __forceinline__ dfl df_from_d(double v) {
  const float hi = __double2float_rn(v);
  const float lo = __double2float_rn(v - (double)hi);
  return dfl{hi, lo};
}

// v 2^e as a double-word (binary64 v, integer e): the same value as
// df_from_d(ldexp(v, e)), formed with integer operations when v 2^e is a
// normal binary64 number with a binary32-normal low word (|v 2^e| within about
// 2^-73 .. 2^127), which spares the binary64 pipe; the conversion itself
// otherwise.  hi = v 2^e rounded to 24 bits (to nearest, ties to even, on the
// integer significand), lo = the exact remainder rounded to 24 bits.
__device__ __forceinline__ dfl df_from_d_pow2(double v, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if ((b << 1) == 0ull) return dfl{0.0f, 0.0f};  // +-0
  const int ex = (int)((b >> 52) & 0x7ffull), E = ex + e;
  if (ex == 0 || ex == 0x7ff || E < 950 || E > 1150) return df_from_d(ldexp(v, e));
  const unsigned long long m = (b & 0xfffffffffffffull) | 0x10000000000000ull;  // 53-bit significand
  unsigned int q = (unsigned int)(m >> 29);
  const unsigned int rem = (unsigned int)(m & 0x1fffffffull);
  if (rem > 0x10000000u || (rem == 0x10000000u && (q & 1u))) ++q;  // q <= 2^24
  const int r = (int)((long long)m - ((long long)q << 29));         // |r| <= 2^28
  const float ph = __int_as_float((E - 1023 - 23 + 127) << 23);    // 2^(E - 1046), normal for E in range
  const float pl = __int_as_float((E - 1023 - 52 + 127) << 23);    // 2^(E - 1075)
  float hi = __uint2float_rn(q) * ph;  // exact
  float lo = __int2float_rn(r) * pl;   // r rounded to 24 bits, scaled exactly
  if (b >> 63) {
    hi = -hi;
    lo = -lo;
  }
  return dfl{hi, lo};
}

}  // namespace bagpu
