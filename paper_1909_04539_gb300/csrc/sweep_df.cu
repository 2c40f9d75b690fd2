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
// or >= 2^101, inf, NaN, FP64 subnormals) switch the warp that meets them to
// native FP64 for the rest of its systems: the two recurrence values convert
// exactly, later forward values are kept as FP64, and the backward sweep of
// that warp runs in FP64 reading pairs below the switch row and FP64 values
// from it on.  The handle admits a matrix only if its sweep gains keep every
// intermediate inside the FP32 range for inputs in that range (factor.cpp).
#include "df_math.cuh"
#include "sweep_kernels.cuh"

namespace bs {

namespace {

constexpr int kDfThreadsMax = 256;

// Coefficient records of one plan (layout of SweepPlan::dfrec): per sweep a
// float4 of the first two coefficient pairs and a float2 of the third; the
// pairs present, in order, are (s), l1, (l2) forward and (t), u1, (u2)
// backward.
struct DfRecs {
  const float4* f4;
  const float4* b4;
  const float2* f2;
  const float2* b2;
};

template <bool ADJ, int BW>
struct DfCount {
  static constexpr int F = (ADJ ? 0 : 1) + BW;  // forward pairs
  static constexpr int B = (ADJ ? 1 : 0) + BW;  // backward pairs
};

__device__ __forceinline__ df::Pair pr(float h, float l) { return df::Pair{h, l}; }

// One step of either sweep from its packed record: HAS_A = the scale pair is
// present (primal forward, adjoint backward).  Pairs in record order: scale
// (if present), first coefficient, second coefficient (BW == 2).
template <bool HAS_A, int BW>
__device__ __forceinline__ df::Pair df_row(float4 q, float2 q2, df::Pair F, df::Pair Y1, df::Pair Y2) {
  df::Pair A{1.f, 0.f}, B1, B2{0.f, 0.f};
  if (HAS_A) {
    A = pr(q.x, q.y);
    B1 = pr(q.z, q.w);
    if (BW == 2) B2 = pr(q2.x, q2.y);
  } else {
    B1 = pr(q.x, q.y);
    if (BW == 2) B2 = pr(q.z, q.w);
  }
  return df::rec_step<HAS_A, BW>(A, F, B1, Y1, B2, Y2);
}

__device__ __forceinline__ double pair_to_f64(df::Pair p) { return (double)p.h + (double)p.l; }

template <int V>
struct Slot;
template <>
struct Slot<1> {
  static __device__ __forceinline__ void ld_f64(const unsigned char* s, double (&o)[1]) {
    o[0] = *reinterpret_cast<const double*>(s);
  }
  static __device__ __forceinline__ void ld_pair(const unsigned char* s, df::Pair (&o)[1]) {
    const float2 t = *reinterpret_cast<const float2*>(s);
    o[0] = pr(t.x, t.y);
  }
  static __device__ __forceinline__ void st_pair(void* d, const df::Pair (&v)[1]) {
    *reinterpret_cast<float2*>(d) = make_float2(v[0].h, v[0].l);
  }
  static __device__ __forceinline__ void st_f64(void* d, const double (&v)[1]) { *reinterpret_cast<double*>(d) = v[0]; }
};
template <>
struct Slot<2> {
  static __device__ __forceinline__ void ld_f64(const unsigned char* s, double (&o)[2]) {
    const double2 t = *reinterpret_cast<const double2*>(s);
    o[0] = t.x;
    o[1] = t.y;
  }
  static __device__ __forceinline__ void ld_pair(const unsigned char* s, df::Pair (&o)[2]) {
    const float4 t = *reinterpret_cast<const float4*>(s);
    o[0] = pr(t.x, t.y);
    o[1] = pr(t.z, t.w);
  }
  static __device__ __forceinline__ void st_pair(void* d, const df::Pair (&v)[2]) {
    *reinterpret_cast<float4*>(d) = make_float4(v[0].h, v[0].l, v[1].h, v[1].l);
  }
  static __device__ __forceinline__ void st_f64(void* d, const double (&v)[2]) {
    *reinterpret_cast<double2*>(d) = make_double2(v[0], v[1]);
  }
};

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
    const unsigned warp_mask = __activemask();
    df::Pair w1[V], w2[V];
    double d1[V], d2[V];
#pragma unroll
    for (int v = 0; v < V; v++) {
      w1[v] = w2[v] = pr(0.f, 0.f);
      d1[v] = d2[v] = 0.0;
    }
    bool f64 = false;  // warp-uniform: this warp's systems continue in native FP64
    int rsw = N;       // first row computed in FP64
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
#pragma unroll
      for (int u = 0; u < U; u++)
        if (FULL || u < n) Slot<V>::ld_f64(ring + (size_t)(s0 + u) * pitch, f[u]);
      df::Pair y[U][V];
      if (!f64) {
        bool fast = true;
#pragma unroll
        for (int u = 0; u < U; u++)
#pragma unroll
          for (int v = 0; v < V; v++) {
            y[u][v] = pr(0.f, 0.f);
            if (FULL || u < n) fast &= df::split_fast(f[u][v], y[u][v]);
          }
        bool bad = false;
        if (!__all_sync(warp_mask, fast)) {  // zeros or range edges in the warp
#pragma unroll
          for (int u = 0; u < U; u++)
#pragma unroll
            for (int v = 0; v < V; v++) {
              bool ok = true;
              y[u][v] = (FULL || u < n) ? df::split(f[u][v], ok) : pr(0.f, 0.f);
              bad |= !ok;
            }
        }
        if (__any_sync(warp_mask, bad)) {  // rare: continue this warp in FP64
          f64 = true;
          rsw = i0;
#pragma unroll
          for (int v = 0; v < V; v++) {
            d1[v] = pair_to_f64(w1[v]);
            d2[v] = pair_to_f64(w2[v]);
          }
        }
      }
      if (!f64) {
        float4 q[U];
        float2 q2[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int i = (FULL || u < n) ? i0 + u : i0;
          q[u] = rc.f4[i];
          q2[u] = F2 ? rc.f2[i] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; u++)
          if (FULL || u < n)
#pragma unroll
            for (int v = 0; v < V; v++) {
              const df::Pair w = df_row<!ADJ, BW>(q[u], q2[u], y[u][v], w1[v], w2[v]);
              w2[v] = w1[v];
              w1[v] = w;
              y[u][v] = w;
            }
      } else {
        fwd_block<BW, ADJ, double, V, U, false>(c64, i0, n, f, d1, d2);
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int i = i0 + u;
        if (FULL || u < n) {
          const bool keep = !FULL && i + D >= N;  // tail row: stays in the ring
          void* dst = keep ? static_cast<void*>(ring + (size_t)(s0 + u) * pitch) : static_cast<void*>(prow);
          if (!f64)
            Slot<V>::st_pair(dst, y[u]);
          else
            Slot<V>::st_f64(dst, f[u]);
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
#pragma unroll
    for (int v = 0; v < V; v++) {
      w1[v] = w2[v] = pr(0.f, 0.f);
      d1[v] = d2[v] = 0.0;
    }
    auto bwd = [&](auto full_tag, int top) {
      constexpr bool FULL = decltype(full_tag)::value;
      const int n = FULL ? U : ((top + 1) < U ? (top + 1) : U);
      if (FULL || top - (n - 1) < tail) cp_wait<D / U - 1>();
      double out[U][V];
      if (!f64) {
        df::Pair y[U][V];
        float4 q[U];
        float2 q2[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int i = (FULL || u < n) ? top - u : top;
          if (FULL || u < n) Slot<V>::ld_pair(ring + (size_t)(i % D) * pitch, y[u]);
          q[u] = rc.b4[i];
          q2[u] = B2 ? rc.b2[i] : make_float2(0.f, 0.f);
        }
        bool cok = true;
#pragma unroll
        for (int u = 0; u < U; u++)
          if (FULL || u < n)
#pragma unroll
            for (int v = 0; v < V; v++) {
              const df::Pair x = df_row<ADJ, BW>(q[u], q2[u], y[u][v], w1[v], w2[v]);
              w2[v] = w1[v];
              w1[v] = x;
              y[u][v] = x;
              cok &= df::combine_ok(x.h);
            }
        // one FP64 add per value; the integer conversion where the warp
        // holds a value below 2^-70 (zeros)
        if (__all_sync(warp_mask, cok)) {
#pragma unroll
          for (int u = 0; u < U; u++)
#pragma unroll
            for (int v = 0; v < V; v++) out[u][v] = df::combine_fast(y[u][v].h, y[u][v].l);
        } else {
#pragma unroll
          for (int u = 0; u < U; u++)
#pragma unroll
            for (int v = 0; v < V; v++) out[u][v] = df::combine(y[u][v].h, y[u][v].l);
        }
      } else {
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int i = top - u;
          if (FULL || u < n) {
            if (i >= rsw) {
              Slot<V>::ld_f64(ring + (size_t)(i % D) * pitch, out[u]);
            } else {
              df::Pair y[V];
              Slot<V>::ld_pair(ring + (size_t)(i % D) * pitch, y);
#pragma unroll
              for (int v = 0; v < V; v++) out[u][v] = pair_to_f64(y[v]);
            }
          }
        }
        bwd_block<BW, ADJ, double, V, U, false>(c64, top, n, out, d1, d2);
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int i = top - u;
        if (FULL || u < n) {
          Slot<V>::st_f64(prow, out[u]);
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
  const float4* f4 = reinterpret_cast<const float4*>(p.dfrec);
  const DfRecs rg{f4, f4 + N, reinterpret_cast<const float2*>(f4 + 2 * N),
                  reinterpret_cast<const float2*>(f4 + 2 * N) + N};
  Coefs<double> c64 = coefs_of<double>(p.c64, N);
  // 12 FP32 values of records per row: pass them as (1 + 2 bw + extra) arrays
  const LaunchShape sh = sweep_shape(BW, N, M / V, 4, 8, V, D * 8 * V, 0, 0, 12 - (1 + 2 * BW));
  const size_t rec = sh.smem_coefs ? (size_t)N * 48 : 0;
  const size_t bytes = rec + (size_t)sh.threads * D * 8 * V;
  auto k = sh.smem_coefs ? k_sweep_df<BW, ADJ, true, V, D> : k_sweep_df<BW, ADJ, false, V, D>;
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
