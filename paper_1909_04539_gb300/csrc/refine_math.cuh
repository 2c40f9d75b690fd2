// Per-row arithmetic of the mixed-precision solve (FP32 sweeps, one
// refinement step with an FP64-accurate residual), shared by the standalone
// kernel and the grouped serving kernel so both give bitwise the same result.
#pragma once

#include "sweep_kernels.cuh"

namespace bs {

template <int BW>
struct RefineCoefs {
  const float* lu[5];   // s, l1, l2, u1, u2 of A = L U   (l2, u2 unused when BW == 1)
  const float* ul[5];   // s, l1, l2, u1, u2 of A = U' L'
  const float* ahi[2 * BW + 1];
  const float* alo[2 * BW + 1];
};

template <int BW>
__host__ __device__ constexpr int refine_arrays() {
  return 2 * (1 + 2 * BW) + 2 * (2 * BW + 1);
}

// r = b - sum_k (ahi_k + alo_k) x_k with error-free products and sums.
template <int W>
__device__ __forceinline__ float residual_row(float b, const float (&x)[W], const float (&ahi)[W],
                                              const float (&alo)[W]) {
  float s = b, c = 0.f;
#pragma unroll
  for (int k = 0; k < W; k++) {
    const float p = __fmul_rn(ahi[k], x[k]);
    const float e = fmaf(ahi[k], x[k], -p);  // ahi * x = p + e exactly
    const float t = __fsub_rn(s, p);         // TwoSum(s, -p) = t + err exactly
    const float bv = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bv)), __fsub_rn(-p, bv));
    s = t;
    c = __fadd_rn(c, __fsub_rn(err, e));
    c = fmaf(-alo[k], x[k], c);
  }
  return __fadd_rn(s, c);
}

// pass 1: forward sweep of A = L U on the FP32 input b of row i
template <int BW>
__device__ __forceinline__ float refine_fwd(const RefineCoefs<BW>& cf, int i, float b, float& w1, float& w2) {
  float w = b * cf.lu[0][i];
  if (BW == 2) w = fmaf(-cf.lu[2][i], w2, w);
  w = fmaf(-cf.lu[1][i], w1, w);
  w2 = w1;
  w1 = w;
  return w;
}

// pass 2a: backward sweep of A = L U at row i; xw[0], xw[1] hold X0 of rows
// i+1, i+2 on entry (the caller shifts the window afterwards)
template <int BW>
__device__ __forceinline__ float refine_bwd(const RefineCoefs<BW>& cf, int i, float w, const float* xw) {
  float x0 = w;
  if (BW == 2) x0 = fmaf(-cf.lu[4][i], xw[1], x0);
  x0 = fmaf(-cf.lu[3][i], xw[0], x0);
  return x0;
}

// pass 2b: residual of row q (x holds X0 of rows q-BW .. q+BW) and the first
// sweep of A = U' L' over decreasing rows
template <int BW>
__device__ __forceinline__ float refine_resid_z(const RefineCoefs<BW>& cf, int q, float b, const float (&x)[2 * BW + 1],
                                                float& z1, float& z2) {
  constexpr int W = 2 * BW + 1;
  float ah[W], al[W];
#pragma unroll
  for (int k = 0; k < W; k++) {
    ah[k] = cf.ahi[k][q];
    al[k] = cf.alo[k][q];
  }
  const float r = residual_row<W>(b, x, ah, al);
  float z = r * cf.ul[0][q];
  if (BW == 2) z = fmaf(-cf.ul[2][q], z2, z);
  z = fmaf(-cf.ul[1][q], z1, z);
  z2 = z1;
  z1 = z;
  return z;
}

// Exact FP32 -> FP64 widening with integer operations only: on GB300 the
// conversion instruction runs on the slow FP64 pipe, and a conditional
// conversion for the rare cases is if-converted into every call.  A normal
// number keeps its sign, its exponent is rebiased by 1023 - 127 = 896 and its
// mantissa moves to the top of the 52-bit field: five integer operations.
// Zero keeps its sign; a subnormal is normalised with a leading-zero count;
// inf and NaN map to exponent 2047.  Those cases are rare, so they run behind
// a branch that the warp takes only if one of its active lanes needs it.
__device__ __forceinline__ double widen_exact(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  uint32_t hi = (((b & 0x7fffffffu) >> 3) + (896u << 20)) | (b & 0x80000000u);
  uint32_t lo = b << 29;
  const bool normal = (e - 1u) < 254u;
  if (__any_sync(__activemask(), !normal)) {
    if (!normal) {
      const uint32_t sign = b & 0x80000000u;
      const uint32_t m = b & 0x7fffffu;
      if (e == 0xffu) {  // inf / NaN
        hi = sign | 0x7ff00000u | (m >> 3);
        lo = m << 29;
      } else if (m == 0u) {  // zero
        hi = sign;
        lo = 0u;
      } else {  // subnormal: m * 2^-149 = 1.f * 2^(p - 149), p = index of the top set bit
        const int p = 31 - __clz((int)m);
        const uint32_t shifted = (m << (23 - p)) & 0x7fffffu;  // drop the leading 1
        hi = sign | ((uint32_t)(p + 874) << 20) | (shifted >> 3);
        lo = shifted << 29;
      }
    }
  }
  return __hiloint2double((int)hi, (int)lo);
}

// FP32 value whose exact FP64 widening needs no special case (normal, finite)
__device__ __forceinline__ bool widen_plain(float f) {
  const uint32_t e = (__float_as_uint(f) >> 23) & 0xffu;
  return e - 1u < 254u;
}

// widen_exact of a value with widen_plain(f) (normal and finite): the five
// integer operations of the common case, no test
__device__ __forceinline__ double widen_normal32(float f) {
  const uint32_t b = __float_as_uint(f);
  return __hiloint2double((int)((((b & 0x7fffffffu) >> 3) + (896u << 20)) | (b & 0x80000000u)), (int)(b << 29));
}

// pass 3: second sweep of A = U' L' at row i and the FP64 sum X0 + d
template <int BW>
__device__ __forceinline__ double refine_out(const RefineCoefs<BW>& cf, int i, float x0, float z, float& d1, float& d2) {
  float d = z;
  if (BW == 2) d = fmaf(-cf.ul[4][i], d2, d);
  d = fmaf(-cf.ul[3][i], d1, d);
  d2 = d1;
  d1 = d;
  return widen_exact(x0) + widen_exact(d);
}

}  // namespace bs

namespace bs {

// Coefficient set of the mixed-precision solve from a handle's device arrays:
// lu = FP32 primal plan (C_COUNT * N), ul = FP32 reversed plan, bands split
// into FP32 hi/lo (width * N each).
template <int BW>
__host__ __device__ __forceinline__ RefineCoefs<BW> make_refine_coefs(const float* lu, const float* ul,
                                                                     const float* bhi, const float* blo, int64_t n) {
  RefineCoefs<BW> cf{};
  const int idx[5] = {C_S, C_L1, C_L2, C_U1, C_U2};
  for (int k = 0; k < 5; k++) {
    cf.lu[k] = lu + idx[k] * n;
    cf.ul[k] = ul + idx[k] * n;
  }
  for (int k = 0; k < 2 * BW + 1; k++) {
    cf.ahi[k] = bhi + k * n;
    cf.alo[k] = blo + k * n;
  }
  return cf;
}

}  // namespace bs

// ---------------------------------------------------------------------------
// Factor-wise refinement (two passes): each triangular sweep of A = L U is
// solved in FP32 and corrected once with the residual of that triangular
// recurrence evaluated to FP64 accuracy.  With the primal sweep coefficients
// (s, l1, l2 forward; u1, u2 backward -- the unit upper factor) held as FP64
// values split into FP32 (hi, lo) pairs:
//   rows up  : w_i = s b_i - l1 w_{i-1} - l2 w_{i-2}  (FP32, hi parts);
//              rho_i = s b_i - w_i - l1 w_{i-1} - l2 w_{i-2}  (to FP64 accuracy);
//              delta_i = rho_i - l1 delta_{i-1} - l2 delta_{i-2}  (FP32)
//              -> y = w + delta  (kept as the pair, 8 bytes per row)
//   rows down: x = U^{-1} fl32(y) (FP32);  sigma = y - U x;  eps = U^{-1} sigma
//              -> X = x + eps in FP64
// rho is (I + Lambda)(w* - w), Lambda the strictly lower part of the forward
// recurrence and w* its exact solution, so delta is the FP32 solution of the
// same recurrence without the scaling by s.  X solves L U X = B to ~1e-15
// relative for well-conditioned bands.

namespace bs {

template <int BW>
struct FRefineCoefs {
  const float* hi[5];  // s, l1, l2, u1, u2: high parts (the FP32 sweep coefficients)
  const float* lo[5];  //   ... low parts
};

// chi/clo: the primal sweep coefficients split into FP32 parts (5 * N each).
template <int BW>
__host__ __device__ __forceinline__ FRefineCoefs<BW> make_frefine_coefs(const float* chi, const float* clo,
                                                                       int64_t n) {
  FRefineCoefs<BW> cf{};
  for (int k = 0; k < 5; k++) {
    cf.hi[k] = chi + k * n;
    cf.lo[k] = clo + k * n;
  }
  return cf;
}

// Coefficients of one row as the two passes use them.
template <int BW>
struct FRow1 {  // pass 1: s, l1, l2 (hi) and their low parts
  float s, l1, l2;
  float sl, l1l, l2l;
};
template <int BW>
struct FRow2 {  // pass 2: u1, u2 (hi) and their low parts
  float u1, u2;
  float u1l, u2l;
};

__device__ __forceinline__ float4 f4_zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// The same coefficients packed per row in shared memory (records of R1 and
// R2 float4s), so that a row's set arrives in one or two 128-bit loads
// instead of one load per value.  Pass-1 record: BW = 1: (s, l1, sl, l1l);
// BW = 2: (s, l1, l2, sl), (l1l, l2l, -, -).  Pass-2 record: BW = 1: (u1,
// u1l, -, -); BW = 2: (u1, u2, u1l, u2l).
template <int BW>
struct FRefineRecs {
  static constexpr int R1 = BW == 1 ? 1 : 2;
  static constexpr int R2 = 1;
  const float4* r1;  // N * R1
  const float4* r2;  // N * R2
};

template <int BW>
__device__ __forceinline__ FRow1<BW> frow1(const FRefineCoefs<BW>& cf, int i) {
  FRow1<BW> c;
  c.s = cf.hi[0][i];
  c.l1 = cf.hi[1][i];
  c.l2 = (BW == 2) ? cf.hi[2][i] : 0.f;
  c.sl = cf.lo[0][i];
  c.l1l = cf.lo[1][i];
  c.l2l = (BW == 2) ? cf.lo[2][i] : 0.f;
  return c;
}
template <int BW>
__device__ __forceinline__ FRow2<BW> frow2(const FRefineCoefs<BW>& cf, int i) {
  FRow2<BW> c;
  c.u1 = cf.hi[3][i];
  c.u2 = (BW == 2) ? cf.hi[4][i] : 0.f;
  c.u1l = cf.lo[3][i];
  c.u2l = (BW == 2) ? cf.lo[4][i] : 0.f;
  return c;
}
template <int BW>
__device__ __forceinline__ FRow1<BW> frow1(const FRefineRecs<BW>& rc, int i) {
  FRow1<BW> c;
  const float4* p = rc.r1 + (size_t)i * FRefineRecs<BW>::R1;
  if constexpr (BW == 1) {
    const float4 a = p[0];
    c.s = a.x, c.l1 = a.y, c.l2 = 0.f, c.sl = a.z, c.l1l = a.w, c.l2l = 0.f;
  } else {
    const float4 a = p[0], b = p[1];
    c.s = a.x, c.l1 = a.y, c.l2 = a.z, c.sl = a.w, c.l1l = b.x, c.l2l = b.y;
  }
  return c;
}
template <int BW>
__device__ __forceinline__ FRow2<BW> frow2(const FRefineRecs<BW>& rc, int i) {
  FRow2<BW> c;
  const float4 a = rc.r2[i];
  if constexpr (BW == 1) {
    c.u1 = a.x, c.u2 = 0.f, c.u1l = a.y, c.u2l = 0.f;
  } else {
    c.u1 = a.x, c.u2 = a.y, c.u1l = a.z, c.u2l = a.w;
  }
  return c;
}

// Writes the packed records of rows [i_begin, N) with stride `step` (for a
// CTA-wide staging loop), reading the per-array coefficients of cf.
template <int BW>
__device__ __forceinline__ void pack_frefine_recs(const FRefineCoefs<BW>& cf, int N, int i_begin, int step,
                                                  float4* r1, float4* r2) {
  for (int i = i_begin; i < N; i += step) {
    const FRow1<BW> a = frow1<BW>(cf, i);
    const FRow2<BW> b = frow2<BW>(cf, i);
    float4* p1 = r1 + (size_t)i * FRefineRecs<BW>::R1;
    if constexpr (BW == 1) {
      p1[0] = make_float4(a.s, a.l1, a.sl, a.l1l);
      r2[i] = make_float4(b.u1, b.u1l, 0.f, 0.f);
    } else {
      p1[0] = make_float4(a.s, a.l1, a.l2, a.sl);
      p1[1] = make_float4(a.l1l, a.l2l, 0.f, 0.f);
      r2[i] = make_float4(b.u1, b.u2, b.u1l, b.u2l);
    }
  }
}

// a - b = s + e exactly (Knuth's TwoSum on -b)
__device__ __forceinline__ void two_diff(float a, float b, float& s, float& e) {
  s = __fsub_rn(a, b);
  const float bv = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(-b, bv));
}

// t + c -= (ch + cl) y with the product ch * y split exactly (FMA) and the
// subtraction from t error-free; the low-order terms collect in c
__device__ __forceinline__ void resid_term(float& t, float& c, float ch, float cl, float y) {
  const float q = __fmul_rn(ch, y);
  const float eq = fmaf(ch, y, -q);  // ch * y = q + eq exactly
  float s, e;
  two_diff(t, q, s, e);
  t = s;
  c = __fadd_rn(c, __fsub_rn(e, eq));
  c = fmaf(-cl, y, c);
}

// Rows i0 .. i0+n-1 of the first pass.  b: the FP32 inputs; on exit w, d
// hold the pairs (w, delta) to keep.  (w1, w2), (d1, d2): the two previous
// rows of each recurrence.  Acc: FRefineCoefs or FRefineRecs (the same
// values, so the same result).
//
// The FP32 sweep forms w = ((p - q2) - q1) with p = fl(s b) and
// q_k = fl(l_k w_k) (TwoProducts: l_k w_k = q_k + eq_k exactly) and both
// subtractions error-free (TwoSums: errors e1, e2), so that the residual
//   rho = s b - w - l1 w1 - l2 w2  (FP64 coefficients s = s_hi + s_lo, ..)
//       = cc + e1 + e2 - eq1 - eq2 - l1_lo w1 - l2_lo w2,
// cc = s b - p to FP64 accuracy: every term is already of the size of the
// residual, so plain FP32 sums carry it to ~2^-24 of itself.
template <int BW, int U, typename Acc>
__device__ __forceinline__ void frefine_pass1(const Acc& cf, int i0, int n, const float (&b)[U], float (&w)[U],
                                              float (&d)[U], float& w1, float& w2, float& d1, float& d2) {
  FRow1<BW> c[U];
#pragma unroll
  for (int u = 0; u < U; u++) c[u] = frow1<BW>(cf, (u < n) ? i0 + u : i0);
  // forward sweep of w (the chain) with the rounding errors of its
  // products and differences kept as the residual's terms
  float rho[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    rho[u] = 0.f;
    w[u] = 0.f;
    if (u < n) {
      const float p = __fmul_rn(b[u], c[u].s);
      float r = fmaf(c[u].sl, b[u], fmaf(c[u].s, b[u], -p));  // s b = p + r to FP64 accuracy
      float x = p, e;
      if (BW == 2) {
        const float q2 = __fmul_rn(c[u].l2, w2);
        r = __fsub_rn(r, fmaf(c[u].l2, w2, -q2));
        r = fmaf(-c[u].l2l, w2, r);
        two_diff(p, q2, x, e);
        r = __fadd_rn(r, e);
      }
      const float q1 = __fmul_rn(c[u].l1, w1);
      r = __fsub_rn(r, fmaf(c[u].l1, w1, -q1));
      r = fmaf(-c[u].l1l, w1, r);
      float y;
      two_diff(x, q1, y, e);
      rho[u] = __fadd_rn(r, e);
      w[u] = y;
      w2 = w1;
      w1 = y;
    }
  }
  // forward sweep of the correction
#pragma unroll
  for (int u = 0; u < U; u++) {
    if (u < n) {
      float x = rho[u];
      if (BW == 2) x = fmaf(-c[u].l2, d2, x);
      x = fmaf(-c[u].l1, d1, x);
      d[u] = x;
      d2 = d1;
      d1 = x;
    }
  }
}

// Rows top, top-1, .., top-n+1 of the second pass: (w, dl) the kept pairs;
// returns the FP64 solution in X.  (x1, x2), (e1, e2): the two rows below.
// As in pass 1 the FP32 sweep x = ((w - q2) - q1) + dl, q_k = fl(u_k x_k),
// takes its differences and its sum error-free (errors g1, g2, g3), so that
// the residual of U x = w + dl (U has a unit diagonal) is
//   sigma = g1 + g2 + g3 - eq1 - eq2 - u1_lo x1 - u2_lo x2.
template <int BW, int U, typename Acc>
__device__ __forceinline__ void frefine_pass2(const Acc& cf, int top, int n, const float (&w)[U],
                                              const float (&dl)[U], double (&X)[U], float& x1, float& x2,
                                              float& e1, float& e2) {
  FRow2<BW> c[U];
#pragma unroll
  for (int u = 0; u < U; u++) c[u] = frow2<BW>(cf, (u < n) ? top - u : top);
  float x[U], sig[U];
  // backward sweep of x (the chain) with its residual terms
#pragma unroll
  for (int u = 0; u < U; u++) {
    x[u] = 1.f;
    sig[u] = 0.f;
    if (u < n) {
      float a = w[u], r = 0.f, g;
      if (BW == 2) {
        const float q2 = __fmul_rn(c[u].u2, x2);
        r = fmaf(-c[u].u2l, x2, -fmaf(c[u].u2, x2, -q2));
        two_diff(w[u], q2, a, g);
        r = __fadd_rn(r, g);
      }
      const float q1 = __fmul_rn(c[u].u1, x1);
      r = __fsub_rn(r, fmaf(c[u].u1, x1, -q1));
      r = fmaf(-c[u].u1l, x1, r);
      float a2;
      two_diff(a, q1, a2, g);
      r = __fadd_rn(r, g);
      float v;
      two_diff(a2, -dl[u], v, g);  // a2 + dl
      sig[u] = __fadd_rn(r, g);
      x[u] = v;
      x2 = x1;
      x1 = v;
    }
  }
  // backward sweep of the correction
  float ev[U];
  bool plain = true;
#pragma unroll
  for (int u = 0; u < U; u++) {
    ev[u] = 1.f;
    if (u < n) {
      float v = sig[u];
      if (BW == 2) v = fmaf(-c[u].u2, e2, v);
      v = fmaf(-c[u].u1, e1, v);
      e2 = e1;
      e1 = v;
      ev[u] = v;
    }
    plain = plain && widen_plain(x[u]) && widen_plain(ev[u]);
  }
  // X = x + eps in FP64: the exactly widened parts added once; one vote per
  // block for the rare values (zero, subnormal, inf, NaN) that need the
  // general widening
  if (__any_sync(__activemask(), !plain)) {
#pragma unroll
    for (int u = 0; u < U; u++) X[u] = widen_exact(x[u]) + widen_exact(ev[u]);
  } else {
#pragma unroll
    for (int u = 0; u < U; u++) X[u] = widen_normal32(x[u]) + widen_normal32(ev[u]);
  }
}

// Rows move in blocks of kRfU.
constexpr int kRfU = 4;

// The two passes of the factor-wise refinement for system j (column j of B
// and X, row stride M) through the lane's ring of D slots of 8 bytes (ring:
// its first slot, generic and shared-window addresses; pitch: bytes between
// slots).  Pass 1 streams B up through the ring and leaves (w, delta) in the
// 8-byte slots of X; pass 2 streams the slots down through the ring and
// writes the FP64 solution over them.  Acc: FRefineCoefs or FRefineRecs.
template <int BW, int D, typename Acc>
__device__ __forceinline__ void refine_factor_system(const Acc& cf, int N, const float* B, double* X, int64_t M,
                                                     int64_t j, const unsigned char* ring, uint32_t ring_s,
                                                     uint32_t pitch) {
  static_assert(D % kRfU == 0, "ring depth must be a multiple of the block");
  const float* pb = B + j;
  double* px = X + j;
  float2* ps = reinterpret_cast<float2*>(X) + j;

  // ---- pass 1 (rows up): slot <- (w, delta).  Row addresses advance by
  // pointer increments (no 64-bit multiply per row).  One copy group per
  // block of kRfU rows (a block waits for the group committed D / kRfU
  // groups earlier); FULL blocks -- all kRfU rows exist and each refills its
  // slot -- run without per-row guards.
  {
    float w1 = 0.f, w2 = 0.f, d1 = 0.f, d2 = 0.f;
    const float* pnext = pb;  // next row to request
#pragma unroll 1
    for (int r = 0; r < D; r++) {
      if (r < N) cp_async4(ring_s + r * pitch, pnext);
      pnext += M;
      if ((r + 1) % kRfU == 0) cp_commit();
    }
    float2* prow = ps;  // slot of row i0
    auto pass1 = [&](auto full_tag, int i0) {
      constexpr bool FULL = decltype(full_tag)::value;
      cp_wait<D / kRfU - 1>();
      const int n = FULL ? kRfU : ((N - i0) < kRfU ? (N - i0) : kRfU);
      const int s0 = i0 % D;
      float b[kRfU], w[kRfU], d[kRfU];
#pragma unroll
      for (int u = 0; u < kRfU; u++) b[u] = *reinterpret_cast<const float*>(ring + (size_t)(s0 + u) * pitch);
#pragma unroll
      for (int u = 0; u < kRfU; u++) {
        if (FULL || (u < n && i0 + u + D < N)) cp_async4(ring_s + (s0 + u) * pitch, pnext);
        pnext += M;
      }
      cp_commit();
      frefine_pass1<BW, kRfU>(cf, i0, n, b, w, d, w1, w2, d1, d2);
#pragma unroll
      for (int u = 0; u < kRfU; u++) {
        if (FULL || u < n) *prow = make_float2(w[u], d[u]);
        prow += M;
      }
    };
    int i0 = 0;
#pragma unroll 1
    for (; i0 + kRfU + D <= N; i0 += kRfU) pass1(std::true_type{}, i0);
#pragma unroll 1
    for (; i0 < N; i0 += kRfU) pass1(std::false_type{}, i0);
    cp_wait<0>();
  }
  // ---- pass 2 (rows down): X
  {
    float x1 = 0.f, x2 = 0.f, e1 = 0.f, e2 = 0.f;
    const float2* pback = ps + (int64_t)(N - 1) * M;  // next slot row to request
#pragma unroll 1
    for (int r = 0; r < D; r++) {
      if (N - 1 - r >= 0) cp_async8(ring_s + r * pitch, pback);
      pback -= M;
      if ((r + 1) % kRfU == 0) cp_commit();
    }
    double* pout = px + (int64_t)(N - 1) * M;  // output row `top`
    auto pass2 = [&](auto full_tag, int top) {
      constexpr bool FULL = decltype(full_tag)::value;
      cp_wait<D / kRfU - 1>();
      const int n = FULL ? kRfU : ((top + 1) < kRfU ? (top + 1) : kRfU);
      const int s0 = (N - 1 - top) % D;
      float w[kRfU], dl[kRfU];
      double xo[kRfU];
#pragma unroll
      for (int u = 0; u < kRfU; u++) {
        const float2 v = *reinterpret_cast<const float2*>(ring + (size_t)(s0 + u) * pitch);
        w[u] = v.x;
        dl[u] = v.y;
      }
#pragma unroll
      for (int u = 0; u < kRfU; u++) {
        if (FULL || (u < n && top - u - D >= 0)) cp_async8(ring_s + (s0 + u) * pitch, pback);
        pback -= M;
      }
      cp_commit();
      frefine_pass2<BW, kRfU>(cf, top, n, w, dl, xo, x1, x2, e1, e2);
#pragma unroll
      for (int u = 0; u < kRfU; u++) {
        if (FULL || u < n) *pout = xo[u];
        pout -= M;
      }
    };
    int top = N - 1;
#pragma unroll 1
    for (; top >= D + kRfU - 1; top -= kRfU) pass2(std::true_type{}, top);
#pragma unroll 1
    for (; top >= 0; top -= kRfU) pass2(std::false_type{}, top);
    cp_wait<0>();
  }
}

}  // namespace bs
