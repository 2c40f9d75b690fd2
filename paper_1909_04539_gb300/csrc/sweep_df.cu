// FP64 solves carried in pairs of FP32 numbers (df_math.cuh): FP64 data in
// and out, FP64-accurate results (a few units of 2^-48), no FP64 instruction
// on the fast path.
//
// The sweeps are the paper's (Sec. 3.1 Thomas, Sec. 4.1 pentadiagonal A = L R)
// in the recurrence form every solve of the library uses,
//   forward : w_i = s_i f_i - l1_i w_{i-1} - l2_i w_{i-2}
//   backward: x_i = t_i w_i - u1_i x_{i+1} - u2_i x_{i+2}
// (primal t == 1, adjoint s == 1), one thread per V systems, as in the FP64
// streaming kernel k_sweep_il2: rows arrive through a per-lane cp.async ring
// of D slots; the forward values, as pairs (8 bytes, the size of the FP64
// element they replace), go to the output buffer in place, the last D stay
// in the ring; the backward sweep streams them back and writes X in FP64.
//
// Each row's coefficients are staged in shared memory as FP32 pairs packed
// into one float4 and (pentadiagonal, three pairs) one float2 per sweep,
// precomputed with the handle (SweepPlan::dfrec).
//
// FP64 inputs outside the pairs' range (df::split !ok: nonzero |f| < 2^-72
// or >= 2^101, inf, NaN, FP64 subnormals) switch the lane that meets them to
// native FP64 for the rest of its systems: the two recurrence values convert
// exactly, later forward values are kept as FP64, and the backward sweep of
// that lane runs in FP64 reading pairs below the switch row and FP64 values
// from it on (df_sweep.cuh: each result depends only on its own system).  The
// handle admits a matrix only if its sweep gains keep every intermediate
// inside the FP32 range for inputs in that range (factor.cpp).
#include "df_sweep.cuh"

namespace bs {

namespace {

constexpr int kDfThreadsMax = 512;

template <int BW, bool ADJ, bool SMEM, int V, int D, bool PER>
__global__ void __launch_bounds__(kDfThreadsMax)
k_sweep_df(DfRecs rg, Coefs<double> c64, int N, double* X, int64_t M) {
  static_assert(D % 4 == 0, "ring depth must be a multiple of the block");
  constexpr int SLOT = 8 * V;
  constexpr bool F2 = DfCount<ADJ, BW>::F > 2, B2 = DfCount<ADJ, BW>::B > 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DfRecs rc = rg;
  size_t rec_bytes = 0;
  if constexpr (SMEM) {
    float4* f4 = reinterpret_cast<float4*>(smem_raw);
    float4* b4 = f4 + N;
    float2* f2 = reinterpret_cast<float2*>(b4 + N);
    float2* b2 = f2 + N;
    float4* pq = reinterpret_cast<float4*>(b2 + N);  // periodic: the (pw', pc') pairs
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      f4[i] = rg.f4[i];
      b4[i] = rg.b4[i];
      if (F2) f2[i] = rg.f2[i];
      if (B2) b2[i] = rg.b2[i];
      if (PER) pq[i] = rg.pq[i];
    }
    rc = DfRecs{f4, b4, f2, b2, PER ? pq : nullptr, rg.per_unscale};
    rec_bytes = (size_t)N * (PER ? 64 : 48);
    __syncthreads();
  }
  unsigned char* ring = smem_raw + rec_bytes + (size_t)threadIdx.x * SLOT;
  const uint32_t ring_s = smem_u32(ring);
  const uint32_t pitch = blockDim.x * SLOT;
  const int64_t ngroups = M / V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride)
    df_sweep_systems<BW, ADJ, V, D, PER>(rc, c64, N, X + g * V, M, ring, ring_s, pitch);
}

template <int BW, bool ADJ, int V, bool PER>
cudaError_t launch_df(const SweepPlan& p, int N, double* X, int64_t M, cudaStream_t st) {
  // 16 rows in flight per lane, blocks of 4 rows: measured on the penta
  // N = 512, M = 65536 batch against (rows, depth) = (4, 8), (4, 32), (8, 16),
  // (8, 32), (2, 16): 0.190 ms against 0.203 - 0.236 ms
  constexpr int D = 16;
  DfRecs rg = df_recs_of(p.dfrec, N);
  Coefs<double> c64 = coefs_of<double>(p.c64, N);
  if (PER) {  // the Sherman-Morrison weights and the rows without correction terms
    rg.pq = reinterpret_cast<const float4*>(p.dfper);
    rg.per_unscale = p.dfper_unscale;
    c64.per_lo = p.per_lo;
    c64.per_hi = p.per_hi;
  }
  // CTA size: any warp multiple the shared memory and registers allow; the
  // busiest SM's warps set the time of this issue-bound kernel (penta N =
  // 512, M = 65536: one 448-thread CTA per SM, 14 warps on the busiest SM,
  // against 16 with four 128-thread CTAs on 56 of the SMs: 0.188 -> 0.170 ms).
  // Ties go to 128 threads: the tri N = 1024, M = 2^20 batch (many passes, all
  // sizes tie) took 5.30 ms with 128, 5.56 - 5.82 ms with 384 - 512.
  auto ks = k_sweep_df<BW, ADJ, true, V, D, PER>;
  auto kg = k_sweep_df<BW, ADJ, false, V, D, PER>;
  const size_t rec = (size_t)N * (PER ? 64 : 48);
  const StagedShape sh = staged_shape(M / V, rec, (size_t)D * 8 * V, kernel_regs((const void*)ks), kDfThreadsMax, true,
                                        128);
  if (sh.threads == 0) return cudaErrorInvalidValue;
  const size_t bytes = (sh.staged ? rec : 0) + (size_t)sh.threads * D * 8 * V;
  auto k = sh.staged ? ks : kg;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k<<<sh.grid, sh.threads, bytes, st>>>(rg, c64, N, X, M);
  return cudaGetLastError();
}

}  // namespace

// Whether sweep_df can take an unpartitioned FP64 solve with plan p: the
// handle admitted the plan (gains, coefficient range) and the option allows.
bool df_eligible(const SweepPlan& p, bs_layout layout) {
  return p.df_ok && p.dfrec != nullptr && layout == BS_INTERLEAVED && (!p.periodic || p.dfper != nullptr) &&
         option(BS_OPT_F64_PAIRS) != 1;
}

// FP64 solve (adjoint: the adjoint plan) in place on X, interleaved layout.
cudaError_t sweep_df(const SweepPlan& p, bool adjoint, int N, double* X, int64_t M, cudaStream_t st) {
  const bool vec2 = (M % 2 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0) &&
                    (option(BS_OPT_F64_PAIRS) == 3 ||
                     (option(BS_OPT_F64_PAIRS) != 2 && M / 2 >= (int64_t)device_info().sms * 32 * 8));
  if (p.periodic) {  // tridiagonal only
    if (vec2) return adjoint ? launch_df<1, true, 2, true>(p, N, X, M, st) : launch_df<1, false, 2, true>(p, N, X, M, st);
    return adjoint ? launch_df<1, true, 1, true>(p, N, X, M, st) : launch_df<1, false, 1, true>(p, N, X, M, st);
  }
  if (p.bw == 1) {
    if (vec2) return adjoint ? launch_df<1, true, 2, false>(p, N, X, M, st) : launch_df<1, false, 2, false>(p, N, X, M, st);
    return adjoint ? launch_df<1, true, 1, false>(p, N, X, M, st) : launch_df<1, false, 1, false>(p, N, X, M, st);
  }
  if (vec2) return adjoint ? launch_df<2, true, 2, false>(p, N, X, M, st) : launch_df<2, false, 2, false>(p, N, X, M, st);
  return adjoint ? launch_df<2, true, 1, false>(p, N, X, M, st) : launch_df<2, false, 1, false>(p, N, X, M, st);
}

}  // namespace bs
