// Mixed-precision solve: FP32 storage and FP32 sweeps, one step of iterative
// refinement with the residual r = B - A X0 evaluated to FP64 accuracy, FP64
// solution.  One thread per system, all in one kernel.
//
//   pass 1 (rows up)  : w = L^{-1} B                       (FP32 sweep of A = L U)
//   pass 2 (rows down): X0 = U^{-1} w                      (FP32)
//                       r  = B - A X0                      (exact to ~2^-48, see below)
//                       z  = U'^{-1} r                     (FP32 sweep of A = U' L')
//   pass 3 (rows up)  : d  = L'^{-1} z,  X = X0 + d        (FP32 sweep, FP64 sum)
//
// The correction solve uses the reversed factorisation A = U' L' (the LU of
// the row- and column-reversed matrix, computed once with the handle) so that
// its first sweep runs over decreasing rows, right behind the backward sweep
// that produces X0: the residual of row q is formed as soon as X0_{q-h} is
// known.  A refinement step therefore costs one extra pass instead of two.
//
// Between the passes each system keeps two FP32 values per row, stored in the
// 8-byte slot of the FP64 output X itself: {w, B} after pass 1, {X0, z} after
// pass 2, and the FP64 solution after pass 3.
//
// Residual accuracy: B and X0 are FP32, each band value a = ahi + alo is the
// FP64 band split into two FP32 numbers.  ahi * X0 is split exactly into a
// rounded product and its FMA-computed error; the large terms B - sum ahi X0
// are accumulated with TwoSum (error-free addition), the small terms (the
// product and sum errors, alo * X0) in plain FP32.  So r carries an absolute
// error of a few FP32 ulps of r itself plus ~2^-48 |A||X0| -- what one step
// of refinement needs to bring the FP32 solution to ~1e-15 relative error for
// well-conditioned bands.
#include <algorithm>

#include "refine_math.cuh"

namespace bs {



// FP32 B (4-byte lane rows in pass 1), 8-byte slots in passes 2 and 3; ring of
// D slots of 8 bytes per lane.  Rows move in blocks of kRU: a block's ring
// reads and coefficient loads are issued before its arithmetic, the chains
// (the sweeps) run row by row, and the block's residuals -- independent of
// each other once X0 is known -- interleave.
constexpr int kRU = 4;

template <int BW, int D, bool SMEM>
__global__ void __launch_bounds__(128)
k_refine(RefineCoefs<BW> cg, int N, const float* B, double* X, int64_t M, int steps) {
  constexpr int W = 2 * BW + 1;
  static_assert(D % kRU == 0, "ring depth must be a multiple of the block");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RefineCoefs<BW> cf = cg;
  size_t coef_bytes = 0;
  if (SMEM) {
    float* sm = reinterpret_cast<float*>(smem_raw);
    int off = 0;
    auto stage = [&](const float*& p) {
      float* dst = sm + off;
      for (int i = threadIdx.x; i < N; i += blockDim.x) dst[i] = p[i];
      p = dst;
      off += N;
    };
    stage(cf.lu[0]);
    stage(cf.lu[1]);
    if (BW == 2) stage(cf.lu[2]);
    stage(cf.lu[3]);
    if (BW == 2) stage(cf.lu[4]);
    stage(cf.ul[0]);
    stage(cf.ul[1]);
    if (BW == 2) stage(cf.ul[2]);
    stage(cf.ul[3]);
    if (BW == 2) stage(cf.ul[4]);
#pragma unroll
    for (int k = 0; k < W; k++) {
      stage(cf.ahi[k]);
      stage(cf.alo[k]);
    }
    coef_bytes = align_up((size_t)off * sizeof(float), 16);
    __syncthreads();
  }
  unsigned char* ring = smem_raw + coef_bytes + (size_t)threadIdx.x * 8;
  const uint32_t ring_s = smem_u32(ring);
  const uint32_t pitch = blockDim.x * 8;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;

  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M; j += stride) {
    const float* pb = B + j;
    double* px = X + j;
    float2* ps = reinterpret_cast<float2*>(X) + j;  // the 8-byte slots, as float pairs

    // ---- pass 1: w = L^{-1} B, slot <- {w, B}
    {
      float w1 = 0.f, w2 = 0.f;
#pragma unroll 1
      for (int r = 0; r < D; r++) {
        if (r < N) cp_async4(ring_s + r * pitch, pb + (int64_t)r * M);
        cp_commit();
      }
#pragma unroll 1
      for (int i0 = 0; i0 < N; i0 += kRU) {
        cp_wait<D - kRU>();
        const int n = (N - i0) < kRU ? (N - i0) : kRU;
        const int s0 = i0 % D;
        float b[kRU];
#pragma unroll
        for (int u = 0; u < kRU; u++) b[u] = *reinterpret_cast<const float*>(ring + (size_t)(s0 + u) * pitch);
#pragma unroll
        for (int u = 0; u < kRU; u++) {
          if (u < n && i0 + u + D < N) cp_async4(ring_s + (s0 + u) * pitch, pb + (int64_t)(i0 + u + D) * M);
          cp_commit();
        }
        float w[kRU];
#pragma unroll
        for (int u = 0; u < kRU; u++)
          if (u < n) w[u] = refine_fwd<BW>(cf, i0 + u, b[u], w1, w2);
#pragma unroll
        for (int u = 0; u < kRU; u++)
          if (u < n) ps[(int64_t)(i0 + u) * M] = make_float2(w[u], b[u]);
      }
      cp_wait<0>();
    }

    // ---- pass 2: X0 = U^{-1} w; r = B - A X0; z = U'^{-1} r; slot <- {X0, z}
    {
      float xw[W + kRU];  // X0 of rows top-kRU+1 .. top+2BW (index q -> row top-kRU+1+q)
      float bw[BW + kRU];
#pragma unroll
      for (int k = 0; k < W + kRU; k++) xw[k] = 0.f;
#pragma unroll
      for (int k = 0; k < BW + kRU; k++) bw[k] = 0.f;
      float z1 = 0.f, z2 = 0.f;
#pragma unroll 1
      for (int r = 0; r < D; r++) {
        const int row = N - 1 - r;
        if (row >= 0) cp_async8(ring_s + r * pitch, ps + (int64_t)row * M);
        cp_commit();
      }
      // blocks of rows top, top-1, .., top-kRU+1 (rows < 0 read as 0)
#pragma unroll 1
      for (int top = N - 1; top >= -BW; top -= kRU) {
        // window shift: rows top+1 .. top+2BW move to the high end
#pragma unroll
        for (int k = W + kRU - 1; k >= kRU; k--) xw[k] = xw[k - kRU];
#pragma unroll
        for (int k = BW + kRU - 1; k >= kRU; k--) bw[k] = bw[k - kRU];
        float wv[kRU];
#pragma unroll
        for (int u = 0; u < kRU; u++) {
          wv[u] = 0.f;
          bw[kRU - 1 - u] = 0.f;
        }
        if (top >= 0) {
          cp_wait<D - kRU>();
          const int s0 = (N - 1 - top) % D;
#pragma unroll
          for (int u = 0; u < kRU; u++) {
            if (top - u >= 0) {
              const float2 wb = *reinterpret_cast<const float2*>(ring + (size_t)(s0 + u) * pitch);
              wv[u] = wb.x;
              bw[kRU - 1 - u] = wb.y;
            }
          }
#pragma unroll
          for (int u = 0; u < kRU; u++) {
            const int i = top - u;
            if (i >= 0 && i - D >= 0) cp_async8(ring_s + (s0 + u) * pitch, ps + (int64_t)(i - D) * M);
            cp_commit();
          }
        }
        // X0 chain, rows top down (row top-u sits at xw[kRU-1-u])
#pragma unroll
        for (int u = 0; u < kRU; u++) {
          const int i = top - u;
          float x0 = 0.f;
          if (i >= 0) {
            const float nx[2] = {xw[kRU - u], xw[kRU - u + 1]};
            x0 = refine_bwd<BW>(cf, i, wv[u], nx);
          }
          xw[kRU - 1 - u] = x0;
        }
        // residuals of rows q = top-u+BW (neighbourhood complete), then the z chain
        float zr[kRU];

#pragma unroll
        for (int u = 0; u < kRU; u++) {
          const int q = top - u + BW;
          zr[u] = 0.f;
          if (q < N && q >= 0) {
            float x[W];
#pragma unroll
            for (int k = 0; k < W; k++) x[k] = xw[kRU - 1 - u + k];
            float ah[W], al[W];
#pragma unroll
            for (int k = 0; k < W; k++) {
              ah[k] = cf.ahi[k][q];
              al[k] = cf.alo[k][q];
            }
            zr[u] = residual_row<W>(bw[kRU - 1 - u + BW], x, ah, al);
          }
        }
#pragma unroll
        for (int u = 0; u < kRU; u++) {
          const int q = top - u + BW;
          if (q < N && q >= 0) {
            if (steps == 0) {
              px[(int64_t)q * M] = (double)xw[kRU - 1 - u + BW];
            } else {
              float z = zr[u] * cf.ul[0][q];
              if (BW == 2) z = fmaf(-cf.ul[2][q], z2, z);
              z = fmaf(-cf.ul[1][q], z1, z);
              z2 = z1;
              z1 = z;
              ps[(int64_t)q * M] = make_float2(xw[kRU - 1 - u + BW], z);
            }

          }
        }

      }
      cp_wait<0>();
    }
    if (steps == 0) continue;

    // ---- pass 3: d = L'^{-1} z; X = X0 + d in FP64
    {
      float d1 = 0.f, d2 = 0.f;
#pragma unroll 1
      for (int r = 0; r < D; r++) {
        if (r < N) cp_async8(ring_s + r * pitch, ps + (int64_t)r * M);
        cp_commit();
      }
#pragma unroll 1
      for (int i0 = 0; i0 < N; i0 += kRU) {
        cp_wait<D - kRU>();
        const int n = (N - i0) < kRU ? (N - i0) : kRU;
        const int s0 = i0 % D;
        float2 xz[kRU];
#pragma unroll
        for (int u = 0; u < kRU; u++) xz[u] = *reinterpret_cast<const float2*>(ring + (size_t)(s0 + u) * pitch);
#pragma unroll
        for (int u = 0; u < kRU; u++) {
          if (u < n && i0 + u + D < N) cp_async8(ring_s + (s0 + u) * pitch, ps + (int64_t)(i0 + u + D) * M);
          cp_commit();
        }
        double xo[kRU];
#pragma unroll
        for (int u = 0; u < kRU; u++)
          if (u < n) xo[u] = refine_out<BW>(cf, i0 + u, xz[u].x, xz[u].y, d1, d2);
#pragma unroll
        for (int u = 0; u < kRU; u++)
          if (u < n) px[(int64_t)(i0 + u) * M] = xo[u];
      }
      cp_wait<0>();
    }
  }
}

// Factor-wise refinement, two passes (refine_factor_system in
// refine_math.cuh, shared with the grouped serving kernel), one system per
// thread, the coefficient records staged in shared memory once per CTA.
// (Two adjacent systems per thread -- 8-byte copies of B, 16-byte slot pairs
// and stores, the records read once for both -- measured slower: penta N =
// 512, M = 65536 0.199 against 0.178 ms, tri N = 1024, M = 2^20 4.82 against
// 4.66; only M = 2^18 gained, 0.649 against 0.659.)
constexpr int kRefineThreadsMax = 512;

template <int BW, int D, bool SMEM>
__global__ void __launch_bounds__(kRefineThreadsMax)
k_refine_factor(FRefineCoefs<BW> cg, int N, const float* B, double* X, int64_t M) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FRefineCoefs<BW> cf = cg;
  // with SMEM, every row's coefficients packed into one record per pass
  FRefineRecs<BW> rc{};
  size_t coef_bytes = 0;
  if (SMEM) {
    float4* r1 = reinterpret_cast<float4*>(smem_raw);
    float4* r2 = r1 + (size_t)N * FRefineRecs<BW>::R1;
    pack_frefine_recs<BW>(cf, N, threadIdx.x, blockDim.x, r1, r2);
    rc.r1 = r1;
    rc.r2 = r2;
    coef_bytes = (size_t)N * (FRefineRecs<BW>::R1 + FRefineRecs<BW>::R2) * sizeof(float4);
    __syncthreads();
  }
  unsigned char* ring = smem_raw + coef_bytes + (size_t)threadIdx.x * 8;
  const uint32_t ring_s = smem_u32(ring);
  const uint32_t pitch = blockDim.x * 8;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;

  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M; j += stride) {
    if constexpr (SMEM)
      refine_factor_system<BW, D>(rc, N, B, X, M, j, ring, ring_s, pitch);
    else
      refine_factor_system<BW, D>(cf, N, B, X, M, j, ring, ring_s, pitch);
  }
}

template <int BW>
static cudaError_t launch_refine_factor_bw(bs_handle h, const float* B, double* X, int64_t M, cudaStream_t st) {
  constexpr int D = 16;
  const int N = (int)h->N;
  const FRefineCoefs<BW> cf = make_frefine_coefs<BW>(h->lu_hi, h->lu_lo, N);
  const DeviceInfo& d = device_info();
  // CTA size from shared memory, registers and the busiest SM's warps
  // (staged_shape), ties to the largest: this kernel runs better in fewer,
  // larger CTAs.  Measured (ms; CTA size fixed): penta N = 512, M = 65536:
  // 128: 0.225, 256: 0.213, 320: 0.260, 384: 0.328 (two waves), 448: 0.207,
  // 512: 0.203; tri N = 1024, M = 2^20: 128: 5.48, 256: 5.07, 320: 4.88,
  // 384: 4.79, 448: 5.42, 512: 5.16.
  auto ks = k_refine_factor<BW, D, true>;
  auto kg = k_refine_factor<BW, D, false>;
  const size_t coef = (size_t)N * (FRefineRecs<BW>::R1 + FRefineRecs<BW>::R2) * sizeof(float4);
  const StagedShape sh = staged_shape(M, coef, (size_t)D * 8, kernel_regs((const void*)ks), kRefineThreadsMax, true,
                                      kRefineThreadsMax);
  if (sh.threads == 0) return cudaErrorInvalidValue;
  const int tpb = sh.threads;
  const bool smem = sh.staged;
  const size_t bytes = (smem ? coef : 0) + (size_t)tpb * D * 8;
  int64_t grid = sh.grid;
  const int64_t budget = option(BS_OPT_INFLIGHT_BYTES);
  if (budget > 0) {
    int64_t cap = budget / ((int64_t)tpb * N * 8);
    if (cap < d.sms) cap = d.sms;
    if (grid > cap) grid = cap;
  }
  auto k = smem ? ks : kg;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k<<<(int)grid, tpb, bytes, st>>>(cf, N, B, X, M);
  return cudaGetLastError();
}

template <int BW>
static cudaError_t launch_refine_bw(bs_handle h, const float* B, double* X, int64_t M, int steps, cudaStream_t st) {
  constexpr int D = 16;
  const int N = (int)h->N;
  const int64_t n = N;
  RefineCoefs<BW> cf{};
  const float* lu = h->plan[0].c32;
  const float* ul = h->plan[2].c32;
  const int idx[5] = {C_S, C_L1, C_L2, C_U1, C_U2};
  for (int k = 0; k < 5; k++) {
    cf.lu[k] = lu + idx[k] * n;
    cf.ul[k] = ul + idx[k] * n;
  }
  for (int k = 0; k < 2 * BW + 1; k++) {
    cf.ahi[k] = h->bands_hi + k * n;
    cf.alo[k] = h->bands_lo + k * n;
  }
  const DeviceInfo& d = device_info();
  int tpb = 128;
  while (tpb > 32 && M < (int64_t)2 * d.sms * tpb) tpb /= 2;
  const size_t coef = align_up((size_t)refine_arrays<BW>() * N * sizeof(float), 16);
  const size_t ring = (size_t)tpb * D * 8;
  const size_t limit = (size_t)(d.smem_optin > 0 ? d.smem_optin : 48 * 1024) - 1024;
  const bool smem = coef + ring <= limit;
  const size_t bytes = (smem ? coef : 0) + ring;
  int per_sm = (int)((228 * 1024) / (bytes + 1024));
  if (per_sm > 2048 / tpb) per_sm = 2048 / tpb;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)d.sms * per_sm;
  // Optional bound on the systems in flight (their 8-byte slots, N per
  // system, between the passes); off by default: the kernel is bound by
  // latency and wants every system in flight.
  const int64_t budget = option(BS_OPT_INFLIGHT_BYTES);
  if (budget > 0) {
    int64_t cap = budget / ((int64_t)tpb * N * 8);
    if (cap < d.sms) cap = d.sms;
    if (grid > cap) grid = cap;
  }
  const int64_t need = (M + tpb - 1) / tpb;
  if (grid > need) grid = need;
  cudaError_t e;
  if (smem) {
    auto k = k_refine<BW, D, true>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k<<<(int)grid, tpb, bytes, st>>>(cf, N, B, X, M, steps);
  } else {
    auto k = k_refine<BW, D, false>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k<<<(int)grid, tpb, bytes, st>>>(cf, N, B, X, M, steps);
  }
  return cudaGetLastError();
}

// X = B widened exactly to FP64 (integer operations, no FP64 pipe).
__global__ void __launch_bounds__(256) k_widen(const float* __restrict__ B, double* __restrict__ X, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    X[i] = widen_exact(B[i]);
}

// BS_REFINE_AUTO: below 256 systems per SM the one-thread FP32 passes are
// bound by their chains of dependent rows, and an FP64 solve of the widened
// input -- row-partitioned or two-ended as bs_solve picks -- is faster and
// exact to FP64 rounding.  Measured (refine / widen + FP64 solve): N = 512
// penta M = 1024: 127 / 77 us, M = 16384: 134 / 120 us, M = 65536: 252 /
// 350 us; N = 1024 tri M = 1024: 226 / 66 us, M = 16384: 235 / 178 us,
// M = 65536: 543 / 635 us (the widening pass then costs 0.16 ms).
static bool refine_direct(int64_t M) { return M < (int64_t)device_info().sms * 256; }

bs_status launch_refine(bs_handle h, const void* B, bs_dtype b_t, double* X, int64_t M, int steps, int mode,
                        cudaStream_t st) {
  if (b_t != BS_F32) return set_error(BS_EUNSUPPORTED, "bs_solve_refine: B must be BS_F32 here");
  if (mode == BS_REFINE_AUTO) {
    if (steps == 1 && refine_direct(M)) {
      const int64_t n = h->N * M;
      int64_t g = (n + 255) / 256;
      const int64_t cap = (int64_t)device_info().sms * 8;
      if (g > cap) g = cap;
      k_widen<<<(int)g, 256, 0, st>>>(static_cast<const float*>(B), X, n);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_error(e, "bs_solve_refine launch");
      return bs_solve(h, X, BS_F64, BS_INTERLEAVED, M, reinterpret_cast<bs_stream>(st));
    }
    mode = BS_REFINE_FACTOR;
  }
  cudaError_t e;
  if (steps == 1 && mode == BS_REFINE_FACTOR)
    e = h->width == 3 ? launch_refine_factor_bw<1>(h, (const float*)B, X, M, st)
                      : launch_refine_factor_bw<2>(h, (const float*)B, X, M, st);
  else
    e = h->width == 3 ? launch_refine_bw<1>(h, (const float*)B, X, M, steps, st)
                      : launch_refine_bw<2>(h, (const float*)B, X, M, steps, st);
  if (e != cudaSuccess) return cuda_error(e, "bs_solve_refine launch");
  return BS_OK;
}

// ------------------------------------------------------------------------
// More refinement steps, BF16 input, strided layout.
//
// Steps beyond the first run on the whole system: r = B - A X in FP64 (the
// FP64 bands, FP64 FMAs), rounded to FP32; A d = r solved by the FP32 sweeps
// (bs_solve, in place on r); X += d.  Each step multiplies the error by about
// kappa(A) 2^-24, so ill-conditioned bands that one step leaves short of FP64
// accuracy get there in a few (the FP64 residual bounds what is reachable:
// about kappa(A) 2^-53).

// r = fl32(B - A X), interleaved, FP64 arithmetic
template <int W>
__global__ void __launch_bounds__(256) k_resid32(const double* __restrict__ bands, int N, const float* __restrict__ B,
                                                 const double* __restrict__ X, int64_t M, float* __restrict__ r) {
  constexpr int H = W / 2;
  const int64_t total = (int64_t)N * M;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / M);
    double s = widen_exact(B[q]);
#pragma unroll
    for (int k = 0; k < W; k++) {
      const int col = i + k - H;
      if (col >= 0 && col < N) s = fma(-bands[(int64_t)k * N + i], X[q + (int64_t)(k - H) * M], s);
    }
    r[q] = (float)s;
  }
}

// X += d (d exact in FP64)
__global__ void __launch_bounds__(256) k_add_widened(double* __restrict__ X, const float* __restrict__ d, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    X[q] += widen_exact(d[q]);
}

// out (interleaved N x M, float) = in, from an interleaved or a strided
// (M x N) batch of float or bf16 (bf16 widened exactly); 32 x 32 tiles
// through shared memory for the strided case
template <typename Sin>
__global__ void __launch_bounds__(256) k_to_interleaved_f32(const Sin* __restrict__ in, int N, int64_t M, int strided,
                                                            float* __restrict__ out) {
  __shared__ float tile[32][33];
  auto val = [](Sin v) -> float {
    if constexpr (std::is_same<Sin, float>::value)
      return v;
    else
      return __bfloat162float(v);
  };
  if (!strided) {
    const int64_t total = (int64_t)N * M;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
      out[q] = val(in[q]);
    return;
  }
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  const int64_t tiles_i = (N + 31) / 32, tiles_j = (M + 31) / 32;
  for (int64_t t = blockIdx.x; t < tiles_i * tiles_j; t += gridDim.x) {
    const int64_t i0 = (t % tiles_i) * 32, j0 = (t / tiles_i) * 32;
    for (int yy = ty; yy < 32; yy += 8) {  // read rows j0 + yy (system), columns i0 + tx
      const int64_t j = j0 + yy, i = i0 + tx;
      if (j < M && i < N) tile[yy][tx] = val(in[j * N + i]);
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {  // write rows i0 + yy, columns j0 + tx
      const int64_t i = i0 + yy, j = j0 + tx;
      if (i < N && j < M) out[i * M + j] = tile[tx][yy];
    }
    __syncthreads();
  }
}

// X (strided, M x N) = Xi (interleaved, N x M)
__global__ void __launch_bounds__(256) k_to_strided_f64(const double* __restrict__ Xi, int N, int64_t M,
                                                        double* __restrict__ X) {
  __shared__ double tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t tiles_i = (N + 31) / 32, tiles_j = (M + 31) / 32;
  for (int64_t t = blockIdx.x; t < tiles_i * tiles_j; t += gridDim.x) {
    const int64_t i0 = (t % tiles_i) * 32, j0 = (t / tiles_i) * 32;
    for (int yy = ty; yy < 32; yy += 8) {
      const int64_t i = i0 + yy, j = j0 + tx;
      if (i < N && j < M) tile[yy][tx] = Xi[i * M + j];
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
      const int64_t j = j0 + yy, i = i0 + tx;
      if (j < M && i < N) X[j * N + i] = tile[tx][yy];
    }
    __syncthreads();
  }
}

static int elementwise_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  const int64_t cap = (int64_t)device_info().sms * 8;
  return (int)(g > cap ? cap : (g < 1 ? 1 : g));
}

// Steps 2 .. steps on an interleaved FP32 B and FP64 X (scratch: N*M floats).
static bs_status refine_more(bs_handle h, const float* B, double* X, int64_t M, int steps, cudaStream_t st) {
  if (steps < 2) return BS_OK;
  const int N = (int)h->N;
  const int64_t n = (int64_t)N * M;
  float* r = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&r), (size_t)n * sizeof(float), st);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? set_error(BS_ENOMEM, "bs_solve_refine: scratch")
                                                               : cuda_error(e, "bs_solve_refine scratch");
  bs_status s = BS_OK;
  for (int k = 2; k <= steps && s == BS_OK; k++) {
    if (h->width == 3)
      k_resid32<3><<<elementwise_grid(n), 256, 0, st>>>(h->bands64, N, B, X, M, r);
    else
      k_resid32<5><<<elementwise_grid(n), 256, 0, st>>>(h->bands64, N, B, X, M, r);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      s = cuda_error(e, "bs_solve_refine residual");
      break;
    }
    s = bs_solve(h, r, BS_F32, BS_INTERLEAVED, M, reinterpret_cast<bs_stream>(st));
    if (s != BS_OK) break;
    k_add_widened<<<elementwise_grid(n), 256, 0, st>>>(X, r, n);
    e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_error(e, "bs_solve_refine update");
  }
  const cudaError_t e2 = cudaFreeAsync(r, st);
  if (s == BS_OK && e2 != cudaSuccess) s = cuda_error(e2, "bs_solve_refine scratch free");
  return s;
}

// Interleaved FP32 B: the one-step kernels, then the further steps.
static bs_status refine_interleaved(bs_handle h, const float* B, double* X, int64_t M, int steps, int mode,
                                    cudaStream_t st) {
  const bs_status s = launch_refine(h, B, BS_F32, X, M, steps > 1 ? 1 : steps, mode, st);
  if (s != BS_OK) return s;
  return refine_more(h, B, X, M, steps, st);
}

}  // namespace bs

extern "C" bs_status bs_solve_refine(bs_handle h, const void* B, bs_dtype b_dtype, double* X, bs_layout layout,
                                     int64_t M, int refine_steps, bs_refine_mode mode, bs_stream stream) {
  using namespace bs;
  if (!valid_handle(h)) return set_error(BS_EINVAL, "bs_solve_refine: unknown handle");
  if (h->periodic) return set_error(BS_EUNSUPPORTED, "bs_solve_refine: not available for a periodic handle");
  if (!B || !X) return set_error(BS_EINVAL, "bs_solve_refine: null data pointer");
  if (M < 1) return set_error(BS_EINVAL, "bs_solve_refine: M must be >= 1");
  if (layout != BS_INTERLEAVED && layout != BS_STRIDED) return set_error(BS_EINVAL, "bs_solve_refine: bad layout");
  if (b_dtype != BS_F32 && b_dtype != BS_BF16)
    return set_error(BS_EINVAL, "bs_solve_refine: B must be BS_F32 or BS_BF16");
  if (refine_steps < 0 || refine_steps > 8) return set_error(BS_EINVAL, "bs_solve_refine: refine_steps must be 0..8");
  if (M > INT64_MAX / 16 / h->N) return set_error(BS_EINVAL, "bs_solve_refine: N*M too large");
  if (mode != BS_REFINE_FACTOR && mode != BS_REFINE_SYSTEM && mode != BS_REFINE_AUTO)
    return set_error(BS_EINVAL, "bs_solve_refine: bad refinement mode");
  if (refine_steps > 0 && mode == BS_REFINE_SYSTEM && !h->has_ul)
    return set_error(BS_ESINGULAR, "bs_solve_refine: the reversed elimination of this matrix met a bad pivot");
  const size_t es = b_dtype == BS_BF16 ? 2 : 4;
  if (reinterpret_cast<uintptr_t>(X) % 8 || reinterpret_cast<uintptr_t>(B) % es)
    return set_error(BS_EINVAL, "bs_solve_refine: misaligned pointer");
  const char* b0 = static_cast<const char*>(B);
  const char* x0 = reinterpret_cast<const char*>(X);
  const size_t nm = (size_t)h->N * (size_t)M;
  if (b0 < x0 + nm * 8 && x0 < b0 + nm * es) return set_error(BS_EINVAL, "bs_solve_refine: B and X overlap");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) return set_error(BS_EINVAL, "bs_solve_refine: handle belongs to another device");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (b_dtype == BS_F32 && layout == BS_INTERLEAVED)
    return refine_interleaved(h, static_cast<const float*>(B), X, M, refine_steps, (int)mode, st);
  // BF16 input and the strided layout: an interleaved FP32 copy of B (bf16
  // widened exactly) and, for the strided layout, an interleaved FP64
  // result, in stream-ordered scratch
  const bool strided = layout == BS_STRIDED;
  float* Bi = nullptr;
  double* Xi = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&Bi), nm * sizeof(float), st);
  if (e == cudaSuccess && strided) e = cudaMallocAsync(reinterpret_cast<void**>(&Xi), nm * sizeof(double), st);
  if (e != cudaSuccess) {
    if (Bi) cudaFreeAsync(Bi, st);
    return e == cudaErrorMemoryAllocation ? set_error(BS_ENOMEM, "bs_solve_refine: scratch")
                                          : cuda_error(e, "bs_solve_refine scratch");
  }
  const int64_t tiles = ((int64_t)h->N + 31) / 32 * ((M + 31) / 32);
  const int g = strided ? (int)std::min<int64_t>(tiles, (int64_t)device_info().sms * 8) : elementwise_grid((int64_t)nm);
  if (b_dtype == BS_BF16)
    k_to_interleaved_f32<__nv_bfloat16><<<g, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(B), (int)h->N, M,
                                                           strided, Bi);
  else
    k_to_interleaved_f32<float><<<g, 256, 0, st>>>(static_cast<const float*>(B), (int)h->N, M, strided, Bi);
  bs_status s = BS_OK;
  e = cudaGetLastError();
  if (e != cudaSuccess) s = cuda_error(e, "bs_solve_refine input copy");
  if (s == BS_OK) s = refine_interleaved(h, Bi, strided ? Xi : X, M, refine_steps, (int)mode, st);
  if (s == BS_OK && strided) {
    k_to_strided_f64<<<(int)std::min<int64_t>(tiles, (int64_t)device_info().sms * 8), 256, 0, st>>>(Xi, (int)h->N, M, X);
    e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_error(e, "bs_solve_refine output copy");
  }
  cudaFreeAsync(Bi, st);
  if (Xi) cudaFreeAsync(Xi, st);
  return s;
}
