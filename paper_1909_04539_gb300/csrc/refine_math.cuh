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

// Exact FP32 -> FP64 widening with integer operations (the FP64 pipe, which
// also executes conversions on GB300, stays free): for normal numbers the
// exponent is rebiased and the mantissa shifted; zero, subnormals, inf and
// NaN take the conversion instruction.
__device__ __forceinline__ double widen_exact(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  const uint32_t lo = b << 29;
  return __hiloint2double((int)hi, (int)lo);
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
