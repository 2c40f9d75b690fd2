// Pair-of-FP32 ("float-float") arithmetic for FP64-accurate sweeps in FP32
// instructions, and exact-enough conversions between FP64 data and pairs
// with integer instructions only.
//
// Why: on GB300 an FP64 instruction issues at ~1/66 of the FP32 rate (about
// 1.6 warp-lanes per clock per SM), so a sweep in native FP64 (5 FP64
// instructions per pentadiagonal unknown) is bound by the FP64 pipe at ~1/4
// of the HBM bandwidth.  A value v is carried instead as an unevaluated sum
// v = h + l of two FP32 numbers with |l| <= ulp(h) (48 significant bits), and
// each recurrence step a*F - b*Y1 - c*Y2 is formed with error-free
// transformations:
//   TwoProduct (FMA form): p = fl(a*b), e = fma(a, b, -p), a*b = p + e exactly;
//   TwoSum (Knuth, six additions): s = fl(a+b), a+b = s + t exactly for any a, b;
//   Fast2Sum (Dekker, three additions): exact when |a| >= |b| (or a == 0),
//     used only to renormalise h + l at the end of a step.
// The product terms a_h*F_l, a_l*F_h etc. and the rounding errors are
// accumulated in plain FP32 (their rounding is ~2^-48 of the terms); a_l*F_l
// (~2^-48) is dropped.  Every step thus carries a relative error of a few
// units of 2^-48 of its largest term.
//
// The FP32 range limits the pairs: an FP64 input is split only when it is
// zero or 2^-72 <= |x| < 2^101 (then h keeps the top 24 significant bits, l
// the next 24, both normal FP32 numbers); anything else reports !ok and the
// caller computes that system in native FP64 instead.
//
// Every function is __host__ __device__ so that the host tests can check the
// conversions bit by bit; on the host the same IEEE single-precision
// operations are used (compile with -ffp-contract=off).
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#include <math.h>
#endif

namespace bs {
namespace df {

struct Pair {
  float h, l;
};

// ------------------------------------------------------------ primitives

DF_HD uint32_t f2u(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
#endif
}
DF_HD float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
DF_HD uint32_t hiword(double d) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__double2hiint(d);
#else
  uint64_t u;
  memcpy(&u, &d, 8);
  return (uint32_t)(u >> 32);
#endif
}
DF_HD uint32_t loword(double d) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__double2loint(d);
#else
  uint64_t u;
  memcpy(&u, &d, 8);
  return (uint32_t)u;
#endif
}
DF_HD double words2d(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t u = ((uint64_t)hi << 32) | lo;
  double d;
  memcpy(&d, &u, 8);
  return d;
#endif
}
// IEEE single operations that the compiler must neither contract into an FMA
// nor reorder (the error-free transformations depend on each rounding).
DF_HD float mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
DF_HD float add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
DF_HD float sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
DF_HD float fma_(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}
// round to nearest (ties to even) to a 32-bit integer; |r| < 2^31
DF_HD int rint_i32(float r) {
#ifdef __CUDA_ARCH__
  return __float2int_rn(r);
#else
  return (int)lrintf(r);
#endif
}

// a + b = s + t exactly (Knuth's TwoSum, no condition on a, b)
DF_HD void two_sum(float a, float b, float& s, float& t) {
  s = add(a, b);
  const float bb = sub(s, a);
  t = add(sub(a, sub(s, bb)), sub(b, bb));
}
// a + b = s + t exactly when |a| >= |b| or a == 0 (Dekker's Fast2Sum)
DF_HD void fast_two_sum(float a, float b, float& s, float& t) {
  s = add(a, b);
  t = sub(b, sub(s, a));
}

// ------------------------------------------------------------ conversions

// Splits an FP64 value x into h + l.  h is x truncated to 24 significant bits
// (exponent rebiased 1023 -> 127, integer operations only), l the FP32
// rounding of the remaining 29 bits, so |x - (h + l)| <= 2^-48 |x|.
// ok: x is zero or 2^-72 <= |x| < 2^101 (both h and l then normal or zero);
// otherwise h, l are meaningless.
DF_HD Pair split(double x, bool& ok) {
  const uint32_t hw = hiword(x), lw = loword(x);
  const uint32_t sign = hw & 0x80000000u;
  const uint32_t ex = (hw >> 20) & 0x7ffu;  // biased FP64 exponent
  // (hw << 3) | (lw >> 29): the low nine exponent bits over the top 23
  // mantissa bits; subtracting 384 << 23 rebiases them (896 = 384 mod 512)
  const uint32_t t = (hw << 3) | (lw >> 29);
  const uint32_t hb = ((t - (384u << 23)) & 0x7fffffffu) | sign;
  // l = (lw mod 2^29) * 2^(ex - 1075), the scale built as an FP32 power of two
  // (normal for ex >= 949) carrying x's sign
  const uint32_t sb = ((ex - 948u) << 23) | sign;
  const float l = mul((float)(lw & 0x1fffffffu), u2f(sb));
  const bool zero = ((hw & 0x7fffffffu) | lw) == 0u;
  ok = (ex - 951u <= 172u) || zero;
  Pair p;
  p.h = zero ? u2f(sign) : u2f(hb);
  p.l = zero ? 0.f : l;
  return p;
}

// split() for the common case, without the zero case: returns false (p
// meaningless) unless 2^-72 <= |x| < 2^101, where it gives exactly split()'s
// pair.  Callers vote over the warp and fall back to split() (zeros, range
// edges) when any lane returns false.
DF_HD bool split_fast(double x, Pair& p) {
  const uint32_t hw = hiword(x), lw = loword(x);
  const uint32_t sign = hw & 0x80000000u;
  const uint32_t t = (hw << 3) | (lw >> 29);
  p.h = u2f(((t - (384u << 23)) & 0x7fffffffu) | sign);
  // 2^(ex - 1075) with x's sign; (hw >> 20) carries the sign bit at bit 11,
  // which the shift by 23 drops
  const uint32_t sb = (((hw >> 20) - 948u) << 23) | sign;
  p.l = mul((float)(lw & 0x1fffffffu), u2f(sb));
  return (hw & 0x7fffffffu) - (951u << 20) < (173u << 20);
}

// Exact FP32 -> FP64 widening of a normal FP32 number with integer
// operations (rebias the exponent by 896, move the mantissa to the top of the
// 52-bit field); zero, subnormals, inf and NaN are not handled.
DF_HD double widen_normal(float f) {
  const uint32_t b = f2u(f);
  return words2d((((b & 0x7fffffffu) >> 3) + (896u << 20)) | (b & 0x80000000u), b << 29);
}

// h + l rounded once to FP64 (one FP64 addition of the two exactly widened
// parts), for |h| >= 2^-70 (combine_ok): a low part that is zero or
// subnormal widens to a value below 2^-125, which the addition rounds away
// next to |h| >= 2^-70.
DF_HD bool combine_ok(float h) { return (f2u(h) & 0x7fffffffu) >= (57u << 23); }
DF_HD double combine_fast(float h, float l) { return widen_normal(h) + widen_normal(l); }

// The FP64 value nearest to h + l (up to one FP64 ulp) for a pair with
// |l| <= ulp(h) and h in the normal range, with integer operations and one
// float-to-integer conversion: the low part, scaled to units of the FP64 ulp
// of h's binade (of the binade below when h is a power of two and l points
// towards zero), is added to the 64-bit pattern of h widened exactly.
// |h| < 2^-126 (zero, when l == 0 too, or subnormal) gives a signed zero; for
// |h| < 2^-75 part of the low part is dropped (a relative error below 2^-24
// of a value that small).
DF_HD double combine(float h, float l) {
  const uint32_t hb = f2u(h), lb = f2u(l);
  const uint32_t ah = hb & 0x7fffffffu;
  const uint32_t opp = (hb ^ lb) >> 31;  // l points towards zero
  const uint32_t eb = (ah - opp) & 0x7f800000u;
  uint32_t sb = (306u << 23) - eb;  // 2^(52 - e), e the unbiased exponent of eb
  sb = (sb > (254u << 23) ? (254u << 23) : sb) | (hb & 0x80000000u);
  const int k = rint_i32(mul(l, u2f(sb)));  // |k| < 2^30, towards |h + l|
  const uint32_t whi = ((ah >> 3) + (896u << 20)) | (hb & 0x80000000u);
  const uint32_t wlo = hb << 29;
  // 64-bit add of the sign-extended k
  const uint32_t lo = wlo + (uint32_t)k;
  const uint32_t carry = lo < wlo ? 1u : 0u;
  const uint32_t hi = whi + (uint32_t)(k >> 31) + carry;
  return ah < 0x00800000u ? words2d(hb & 0x80000000u, 0u) : words2d(hi, lo);
}

// ------------------------------------------------------------ one step

// y = A*F - B1*Y1 - B2*Y2 in pairs (A, B1, B2 coefficients, F, Y1, Y2
// values), renormalised (|l| <= ulp(h)/2).  HAS_A = false: A == 1; BW == 1:
// no B2 term.  The terms of Y2 (the older value) are formed first, so that
// the latest value Y1 enters through one product and one TwoSum.  (Leaving
// out the final Fast2Sum saves three instructions a step but loses accuracy
// where the step's terms cancel: stiff I + 1000 D4 went from 6.6e-14 to
// 2.1e-12.)
template <bool HAS_A, int BW>
DF_HD Pair rec_step(Pair A, Pair F, Pair B1, Pair Y1, Pair B2, Pair Y2) {
  float s, lo;
  if (HAS_A) {
    s = mul(A.h, F.h);
    lo = fma_(A.h, F.h, -s);
    lo = fma_(A.h, F.l, lo);
    lo = fma_(A.l, F.h, lo);
  } else {
    s = F.h;
    lo = F.l;
  }
  if (BW == 2) {
    const float p2 = mul(B2.h, Y2.h);
    const float e2 = fma_(B2.h, Y2.h, -p2);
    float t2;
    two_sum(s, -p2, s, t2);
    lo = sub(lo, e2);
    lo = fma_(-B2.h, Y2.l, lo);
    lo = fma_(-B2.l, Y2.h, lo);
    lo = add(lo, t2);
  }
  const float p1 = mul(B1.h, Y1.h);
  const float e1 = fma_(B1.h, Y1.h, -p1);
  float t1;
  two_sum(s, -p1, s, t1);
  lo = sub(lo, e1);
  lo = fma_(-B1.h, Y1.l, lo);
  lo = fma_(-B1.l, Y1.h, lo);
  lo = add(lo, t1);
  Pair y;
  fast_two_sum(s, lo, y.h, y.l);
  return y;
}

}  // namespace df
}  // namespace bs
