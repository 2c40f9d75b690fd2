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

// V lane-rows of 8-byte values (pairs or FP64) in a ring slot or in memory
template <int V>
__device__ __forceinline__ void ld8(const void* p, uint2 (&o)[V]) {
  if constexpr (V == 2) {
    const uint4 t = *reinterpret_cast<const uint4*>(p);
    o[0] = make_uint2(t.x, t.y);
    o[1] = make_uint2(t.z, t.w);
  } else {
    o[0] = *reinterpret_cast<const uint2*>(p);
  }
}
template <int V>
__device__ __forceinline__ void st8(void* p, const uint2 (&x)[V]) {
  if constexpr (V == 2)
    *reinterpret_cast<uint4*>(p) = make_uint4(x[0].x, x[0].y, x[1].x, x[1].y);
  else
    *reinterpret_cast<uint2*>(p) = x[0];
}
template <int V>
__device__ __forceinline__ void ld_f64v(const void* p, double (&o)[V]) {
  if constexpr (V == 2) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    o[0] = t.x;
    o[1] = t.y;
  } else {
    o[0] = *reinterpret_cast<const double*>(p);
  }
}
template <int V>
__device__ __forceinline__ void st_f64v(void* p, const double (&x)[V]) {
  if constexpr (V == 2)
    *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
  else
    *reinterpret_cast<double*>(p) = x[0];
}

template <int BW, bool ADJ, bool SMEM, int V, int D>
__global__ void __launch_bounds__(kDfThreadsMax)
k_sweep_df(DfRecs rg, Coefs<double> c64, int N, double* X, int64_t M) {
  constexpr int U = 4;  // rows per block; D is a multiple of U
  static_assert(D % U == 0, "ring depth must be a multiple of the block");
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
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      f4[i] = rg.f4[i];
      b4[i] = rg.b4[i];
      if (F2) f2[i] = rg.f2[i];
      if (B2) b2[i] = rg.b2[i];
    }
    rc = DfRecs{f4, b4, f2, b2};
    rec_bytes = (size_t)N * 48;
    __syncthreads();
  }
  unsigned char* ring = smem_raw + rec_bytes + (size_t)threadIdx.x * SLOT;
  const uint32_t ring_s = smem_u32(ring);
  const uint32_t pitch = blockDim.x * SLOT;
  const int64_t ngroups = M / V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
    double* const pout = X + g * V;
    DfState<V> st;
    st.reset_values();
    st.f64 = false;
    st.rsw = N;
    // forward sweep: rows 0..D-1 requested up front (one copy group per
    // block of U rows); each block then waits for its group, computes and
    // refills its slots with the rows D further down
    const double* pnext = pout;
#pragma unroll 1
    for (int r = 0; r < D; r++) {
      if (r < N) copy_row<double, V>(ring_s + r * pitch, pnext);
      pnext += M;
      if ((r + 1) % U == 0) cp_commit();
    }
    double* prow = pout;
    auto fwd = [&](auto full_tag, int i0) {
      constexpr bool FULL = decltype(full_tag)::value;
      cp_wait<D / U - 1>();
      const int n = FULL ? U : ((N - i0) < U ? (N - i0) : U);
      const int s0 = i0 % D;
      double f[U][V];
      uint2 w[U][V];
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (FULL || u < n)
          ld_f64v<V>(ring + (size_t)(s0 + u) * pitch, f[u]);
        else
#pragma unroll
          for (int v = 0; v < V; v++) f[u][v] = 0.0;
      }
      df_fwd_group<BW, ADJ, V, U, FULL>(rc, c64, i0, n, f, w, st);
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int i = i0 + u;
        if (FULL || u < n) {
          const bool keep = !FULL && i + D >= N;  // tail row: stays in the ring
          st8<V>(keep ? static_cast<void*>(ring + (size_t)(s0 + u) * pitch) : static_cast<void*>(prow), w[u]);
          if (!keep) copy_row<double, V>(ring_s + (s0 + u) * pitch, pnext);
        }
        prow += M;
        pnext += M;
      }
      cp_commit();
    };
    int i0 = 0;
#pragma unroll 1
    for (; i0 + U + D <= N; i0 += U) fwd(std::true_type{}, i0);
#pragma unroll 1
    for (; i0 < N; i0 += U) fwd(std::false_type{}, i0);

    // backward sweep: rows N-1 .. N-D are in the ring; row i - D is requested
    // into the slot row i frees (blocks aligned to N - 1, one group each)
    const int tail = N - D;
    prow = pout + (int64_t)(N - 1) * M;
    const double* pback = pout + (int64_t)(N - 1 - D) * M;
    st.reset_values();
    auto bwd = [&](auto full_tag, int top) {
      constexpr bool FULL = decltype(full_tag)::value;
      const int n = FULL ? U : ((top + 1) < U ? (top + 1) : U);
      if (FULL || top - (n - 1) < tail) cp_wait<D / U - 1>();
      uint2 w[U][V];
      double x[U][V];
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (FULL || u < n)
          ld8<V>(ring + (size_t)((top - u) % D) * pitch, w[u]);
        else
#pragma unroll
          for (int v = 0; v < V; v++) w[u][v] = make_uint2(0u, 0u);
      }
      df_bwd_group<BW, ADJ, V, U, FULL>(rc, c64, top, n, w, x, st);
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int i = top - u;
        if (FULL || u < n) {
          st_f64v<V>(prow, x[u]);
          if (FULL || i - D >= 0) copy_row<double, V>(ring_s + (i % D) * pitch, pback);
        }
        prow -= M;
        pback -= M;
      }
      cp_commit();
    };
    int top = N - 1;
#pragma unroll 1
    for (; top >= D + U - 1; top -= U) bwd(std::true_type{}, top);
#pragma unroll 1
    for (; top >= 0; top -= U) bwd(std::false_type{}, top);
    cp_wait<0>();
  }
}

template <int BW, bool ADJ, int V>
cudaError_t launch_df(const SweepPlan& p, int N, double* X, int64_t M, cudaStream_t st) {
  // 16 rows in flight per lane, blocks of 4 rows: measured on the penta
  // N = 512, M = 65536 batch against (rows, depth) = (4, 8), (4, 32), (8, 16),
  // (8, 32), (2, 16): 0.190 ms against 0.203 - 0.236 ms
  constexpr int D = 16;
  const DfRecs rg = df_recs_of(p.dfrec, N);
  Coefs<double> c64 = coefs_of<double>(p.c64, N);
  // CTA size: any warp multiple the shared memory and registers allow; the
  // busiest SM's warps set the time of this issue-bound kernel (penta N =
  // 512, M = 65536: one 448-thread CTA per SM, 14 warps on the busiest SM,
  // against 16 with four 128-thread CTAs on 56 of the SMs: 0.188 -> 0.170 ms).
  // Ties go to 128 threads: the tri N = 1024, M = 2^20 batch (many passes, all
  // sizes tie) took 5.30 ms with 128, 5.56 - 5.82 ms with 384 - 512.
  auto ks = k_sweep_df<BW, ADJ, true, V, D>;
  auto kg = k_sweep_df<BW, ADJ, false, V, D>;
  const size_t rec = (size_t)N * 48;
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
  return p.df_ok && p.dfrec != nullptr && layout == BS_INTERLEAVED && !p.periodic &&
         option(BS_OPT_F64_PAIRS) != 1;
}

// FP64 solve (adjoint: the adjoint plan) in place on X, interleaved layout.
cudaError_t sweep_df(const SweepPlan& p, bool adjoint, int N, double* X, int64_t M, cudaStream_t st) {
  const bool vec2 = (M % 2 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0) &&
                    (option(BS_OPT_F64_PAIRS) == 3 ||
                     (option(BS_OPT_F64_PAIRS) != 2 && M / 2 >= (int64_t)device_info().sms * 32 * 8));
  if (p.bw == 1) {
    if (vec2) return adjoint ? launch_df<1, true, 2>(p, N, X, M, st) : launch_df<1, false, 2>(p, N, X, M, st);
    return adjoint ? launch_df<1, true, 1>(p, N, X, M, st) : launch_df<1, false, 1>(p, N, X, M, st);
  }
  if (vec2) return adjoint ? launch_df<2, true, 2>(p, N, X, M, st) : launch_df<2, false, 2>(p, N, X, M, st);
  return adjoint ? launch_df<2, true, 1>(p, N, X, M, st) : launch_df<2, false, 1>(p, N, X, M, st);
}

}  // namespace bs
