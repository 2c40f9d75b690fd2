// Windowed sweeps: the forward-sweep values stay on chip.
//
// The paper's solve (Sec. 2, Sec. 3.1, Sec. 4.1) runs a forward sweep over
// all N rows and then a backward sweep over all of them, so every forward
// value w_i is kept until the backward sweep comes back to row i -- the
// paper keeps them in the RHS array itself, in place, which moves each row
// through memory twice more.  For the diagonally dominant matrices of the
// method the backward recurrence x_i = t_i w_i - u1_i x_{i+1} - u2_i x_{i+2}
// forgets where it started: started from zero at a row e instead of from the
// true x_e, x_{e+1}, it is off at row e - d by a factor that decays
// geometrically in d (for I + 0.1 D4, [1,4,1]/6 or I - 0.5 d2 below 2^-50
// after ~28 rows).  The factorisation measures, per plan, the number Lw of
// rows after which that factor stays below 2^-50 (pair and FP64 arithmetic)
// or 2^-28 (FP32): make_windows in factor.cpp.
//
// So each system is swept in blocks of K rows.  After the forward sweep has
// reached the end e of a block, a backward sweep runs from e - 1 down to the
// first row not yet written, starting from zero at e: every row more than Lw
// rows above e is then exact (to the factor above times the system's largest
// value) and is written out; the last Lw rows of the block are recomputed by
// the next block's backward sweep, which passes through them on its way.
// The last block starts from the true boundary (x_N = x_{N+1} = 0) and
// writes all its rows.  Per system only the rows between the oldest row not
// yet written and the newest row requested -- at most K + Lw + D -- live in
// a per-lane ring of R slots in shared memory (cp.async, D rows in flight);
// B is read once and X written once.  The price is Lw extra backward steps
// per block of K.
//
// Arithmetic: FP32 (FP32 data), or FP32 pairs for FP64 data (df_math.cuh)
// with the same per-warp switch to native FP64 as sweep_df.cu: a warp that
// meets an input the pairs cannot hold converts the pair values of its live
// rows to FP64 in place and continues the windowed sweep in FP64.
#include "df_math.cuh"
#include "sweep_kernels.cuh"

namespace bs {

namespace {

constexpr int kWU = 4;           // rows per group
constexpr int kWinThreads = 512;  // largest CTA

__device__ __forceinline__ df::Pair wpr(float h, float l) { return df::Pair{h, l}; }

// Packed per-row coefficient records.  FP32: forward (s, l1, l2, -),
// backward (t, u1, u2, -) as one float4 each.  Pairs: the layout of
// SweepPlan::dfrec (float4 of the first two pairs, float2 of the third).
struct WinRecs {
  const float4* f4;
  const float4* b4;
  const float2* f2;
  const float2* b2;
};

template <bool HAS_A, int BW>
__device__ __forceinline__ df::Pair pair_row(float4 q, float2 q2, df::Pair F, df::Pair Y1, df::Pair Y2) {
  df::Pair A{1.f, 0.f}, B1, B2{0.f, 0.f};
  if (HAS_A) {
    A = wpr(q.x, q.y);
    B1 = wpr(q.z, q.w);
    if (BW == 2) B2 = wpr(q2.x, q2.y);
  } else {
    B1 = wpr(q.x, q.y);
    if (BW == 2) B2 = wpr(q.z, q.w);
  }
  return df::rec_step<HAS_A, BW>(A, F, B1, Y1, B2, Y2);
}

// lane-row accessors: V values of E bytes each
template <typename T, int V>
__device__ __forceinline__ void ld_row(const unsigned char* s, T (&o)[V]) {
#pragma unroll
  for (int v = 0; v < V; v++) o[v] = reinterpret_cast<const T*>(s)[v];
}
template <typename T, int V>
__device__ __forceinline__ void st_row(unsigned char* s, const T (&x)[V]) {
  if constexpr (V * sizeof(T) == 16) {
    const uint4* p = reinterpret_cast<const uint4*>(x);
    *reinterpret_cast<uint4*>(s) = *p;
  } else if constexpr (V * sizeof(T) == 8) {
    *reinterpret_cast<uint2*>(s) = *reinterpret_cast<const uint2*>(x);
  } else {
#pragma unroll
    for (int v = 0; v < V; v++) reinterpret_cast<T*>(s)[v] = x[v];
  }
}
template <int V>
__device__ __forceinline__ void ld_pairs(const unsigned char* s, df::Pair (&o)[V]) {
#pragma unroll
  for (int v = 0; v < V; v++) {
    const float2 t = reinterpret_cast<const float2*>(s)[v];
    o[v] = wpr(t.x, t.y);
  }
}
template <int V>
__device__ __forceinline__ void st_pairs(unsigned char* s, const df::Pair (&x)[V]) {
  if constexpr (V == 2) {
    *reinterpret_cast<float4*>(s) = make_float4(x[0].h, x[0].l, x[1].h, x[1].l);
  } else {
#pragma unroll
    for (int v = 0; v < V; v++) reinterpret_cast<float2*>(s)[v] = make_float2(x[v].h, x[v].l);
  }
}

// One lane-row of V elements of T to global memory (in the layout's vector width)
template <typename T, int V>
__device__ __forceinline__ void st_global(T* p, const T (&x)[V]) {
  if constexpr (V * sizeof(T) == 16) {
    *reinterpret_cast<uint4*>(p) = *reinterpret_cast<const uint4*>(x);
  } else if constexpr (V * sizeof(T) == 8) {
    *reinterpret_cast<uint2*>(p) = *reinterpret_cast<const uint2*>(x);
  } else {
#pragma unroll
    for (int v = 0; v < V; v++) p[v] = x[v];
  }
}

// DFK = true: FP64 data in pair arithmetic (Sin = Sout = double); false:
// FP32 arithmetic on Sin = float or bf16 input, Sout = float.  R (a power of
// two) slots per lane; groups of U rows start at multiples of U, so a group's
// slots are consecutive.
template <int BW, bool ADJ, int V, int R, int D, bool SMEM, bool DFK, typename Sin, typename Sout>
__global__ void __launch_bounds__(kWinThreads)
k_sweep_win(WinRecs rg, Coefs<double> c64, int N, int K, int Lw, const Sin* in, Sout* out, int64_t M) {
  static_assert(D % kWU == 0 && R % kWU == 0 && (R & (R - 1)) == 0, "ring: a power of two of whole groups");
  constexpr int U = kWU;
  constexpr int EB = DFK ? 8 : 4;     // bytes of one stored value per system
  constexpr int SB = V * EB;          // slot bytes
  constexpr int IB = V * (int)sizeof(Sin);  // input bytes per lane-row
  static_assert(IB == 4 || IB == 8 || IB == 16, "a lane-row of input must be 4, 8 or 16 bytes");
  constexpr bool F2 = DFK && (ADJ ? 0 : 1) + BW > 2;
  constexpr bool B2 = DFK && (ADJ ? 1 : 0) + BW > 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WinRecs rc = rg;
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
    rc = WinRecs{f4, b4, f2, b2};
    rec_bytes = DFK ? (size_t)N * 48 : (size_t)N * 32;
    __syncthreads();
  }
  unsigned char* const ring = smem_raw + rec_bytes + (size_t)threadIdx.x * SB;
  const uint32_t ring_s = smem_u32(ring);
  const uint32_t pitch = blockDim.x * SB;
  // one lane-row of input into the slot at shared address a
  auto request = [&](uint32_t a, const Sin* p) {
    if constexpr (IB == 4) {
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(p) : "memory");
    } else if constexpr (IB == 8) {
      cp_async8(a, p);
    } else {
      cp_async16(a, p);
    }
  };
  const int64_t ngroups = M / V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t M4 = (int64_t)U * M;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
    const Sin* const pin = in + g * V;
    Sout* const pout = out + g * V;
    const unsigned warp_mask = __activemask();
    float f1[V], f2[V];
    df::Pair p1[V], p2[V];
    double d1[V], d2[V];
#pragma unroll
    for (int v = 0; v < V; v++) {
      f1[v] = f2[v] = 0.f;
      p1[v] = p2[v] = wpr(0.f, 0.f);
      d1[v] = d2[v] = 0.0;
    }
    bool f64 = false;  // (pairs) warp-uniform: continue in native FP64
    {
      const Sin* p = pin;
#pragma unroll 1
      for (int r = 0; r < D; r++) {
        if (r < N) request(ring_s + (uint32_t)r * pitch, p);
        p += M;
        if ((r + 1) % U == 0) cp_commit();
      }
    }
    const Sin* pnext = pin + (int64_t)D * M;  // row i0 + D of the current group
    int lo = 0;                                // oldest row not yet written

    // ------------------------------------------------------ forward group
    // rows i0 .. i0+n-1 (n = U when FULL), then the requests of rows D ahead
    auto fwd = [&](auto full_tag, int i0, int n) {
      constexpr bool FULL = decltype(full_tag)::value;
      cp_wait<D / U - 1>();
      unsigned char* const sb = ring + (size_t)(i0 & (R - 1)) * pitch;
      if constexpr (!DFK) {
        float x[U][V];
        float4 q[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          q[u] = rc.f4[(FULL || u < n) ? i0 + u : i0];
          if (FULL || u < n) {
            if constexpr (std::is_same<Sin, float>::value) {
              ld_row<float, V>(sb + u * pitch, x[u]);
            } else {
              __nv_bfloat16 b[V];
              ld_row<__nv_bfloat16, V>(sb + u * pitch, b);
#pragma unroll
              for (int v = 0; v < V; v++) x[u][v] = __bfloat162float(b[v]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; u++)
          if (FULL || u < n) {
#pragma unroll
            for (int v = 0; v < V; v++) {
              float w = ADJ ? x[u][v] : x[u][v] * q[u].x;
              if (BW == 2) w = fmaf(-q[u].z, f2[v], w);
              w = fmaf(-q[u].y, f1[v], w);
              f2[v] = f1[v];
              f1[v] = w;
              x[u][v] = w;
            }
            st_row<float, V>(sb + u * pitch, x[u]);
          }
      } else {
        double x[U][V];
#pragma unroll
        for (int u = 0; u < U; u++)
          if (FULL || u < n) ld_row<double, V>(sb + u * pitch, x[u]);
        if (!f64) {
          df::Pair y[U][V];
          bool fast = true;
#pragma unroll
          for (int u = 0; u < U; u++)
#pragma unroll
            for (int v = 0; v < V; v++) {
              y[u][v] = wpr(0.f, 0.f);
              if (FULL || u < n) fast &= df::split_fast(x[u][v], y[u][v]);
            }
          bool bad = false;
          if (!__all_sync(warp_mask, fast)) {  // zeros or range edges in the warp
#pragma unroll
            for (int u = 0; u < U; u++)
#pragma unroll
              for (int v = 0; v < V; v++) {
                bool ok = true;
                y[u][v] = (FULL || u < n) ? df::split(x[u][v], ok) : wpr(0.f, 0.f);
                bad |= !ok;
              }
          }
          if (__any_sync(warp_mask, bad)) {
            // rare: this warp continues in native FP64; the pair values of
            // its live rows [lo, i0) become FP64 values in place
            f64 = true;
#pragma unroll 1
            for (int r = lo; r < i0; r++) {
              unsigned char* sr = ring + (size_t)(r & (R - 1)) * pitch;
              df::Pair t[V];
              ld_pairs<V>(sr, t);
              double dv[V];
#pragma unroll
              for (int v = 0; v < V; v++) dv[v] = (double)t[v].h + (double)t[v].l;
              st_row<double, V>(sr, dv);
            }
#pragma unroll
            for (int v = 0; v < V; v++) {
              d1[v] = (double)p1[v].h + (double)p1[v].l;
              d2[v] = (double)p2[v].h + (double)p2[v].l;
            }
          } else {
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
              if (FULL || u < n) {
#pragma unroll
                for (int v = 0; v < V; v++) {
                  const df::Pair w = pair_row<!ADJ, BW>(q[u], q2[u], y[u][v], p1[v], p2[v]);
                  p2[v] = p1[v];
                  p1[v] = w;
                  y[u][v] = w;
                }
                st_pairs<V>(sb + u * pitch, y[u]);
              }
          }
        }
        if (f64) {
          fwd_block<BW, ADJ, double, V, U, false>(c64, i0, n, x, d1, d2);
#pragma unroll
          for (int u = 0; u < U; u++)
            if (FULL || u < n) st_row<double, V>(sb + u * pitch, x[u]);
        }
      }
      // requests of rows i0 + D + u (their slots held rows already written)
      const uint32_t qa = ring_s + (uint32_t)((i0 + D) & (R - 1)) * pitch;
      const Sin* p = pnext;
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (FULL || (u < n && i0 + D + u < N)) request(qa + u * pitch, p);
        p += M;
      }
      pnext += M4;
      cp_commit();
    };

    // ----------------------------------------------------- backward group
    // rows gs+U-1 .. gs of the aligned group gs, those in [lo, e); written
    // when below hi.  WHOLE: all U rows in range; OUT: 0 none written, 1 all,
    // 2 per row.
    float y1[V], y2[V];
    df::Pair q1[V], q2v[V];
    double z1[V], z2[V];
    auto bwd = [&](auto whole_tag, auto out_tag, int gs, int lo_, int e, int hi) {
      constexpr bool WHOLE = decltype(whole_tag)::value;
      constexpr int OUT = decltype(out_tag)::value;
      unsigned char* const sb = ring + (size_t)(gs & (R - 1)) * pitch;
      Sout* const po = pout + (int64_t)gs * M;
      auto in_range = [&](int u) { return WHOLE || (gs + u >= lo_ && gs + u < e); };
      auto written = [&](int u) { return OUT == 1 || (OUT == 2 && gs + u < hi); };
      if constexpr (!DFK) {
        float x[U][V];
        float4 q[U];
#pragma unroll
        for (int u = U - 1; u >= 0; u--) {
          q[u] = rc.b4[in_range(u) ? gs + u : (gs + U - 1 < e ? gs + U - 1 : e - 1)];
          if (in_range(u)) ld_row<float, V>(sb + u * pitch, x[u]);
        }
#pragma unroll
        for (int u = U - 1; u >= 0; u--)
          if (in_range(u)) {
#pragma unroll
            for (int v = 0; v < V; v++) {
              float y = ADJ ? x[u][v] * q[u].x : x[u][v];
              if (BW == 2) y = fmaf(-q[u].z, y2[v], y);
              y = fmaf(-q[u].y, y1[v], y);
              y2[v] = y1[v];
              y1[v] = y;
              x[u][v] = y;
            }
            if (OUT != 0 && written(u)) st_global<Sout, V>(po + (int64_t)u * M, x[u]);
          }
      } else {
        if (!f64) {
          df::Pair w[U][V];
          float4 q[U];
          float2 qq[U];
#pragma unroll
          for (int u = U - 1; u >= 0; u--) {
            const int i = in_range(u) ? gs + u : (gs + U - 1 < e ? gs + U - 1 : e - 1);
            q[u] = rc.b4[i];
            qq[u] = B2 ? rc.b2[i] : make_float2(0.f, 0.f);
            if (in_range(u)) ld_pairs<V>(sb + u * pitch, w[u]);
          }
#pragma unroll
          for (int u = U - 1; u >= 0; u--)
            if (in_range(u)) {
#pragma unroll
              for (int v = 0; v < V; v++) {
                const df::Pair y = pair_row<ADJ, BW>(q[u], qq[u], w[u][v], q1[v], q2v[v]);
                q2v[v] = q1[v];
                q1[v] = y;
              }
              if (OUT != 0 && written(u)) {
                double o[V];
                bool cok = true;
#pragma unroll
                for (int v = 0; v < V; v++) cok &= df::combine_ok(q1[v].h);
                if (__all_sync(warp_mask, cok)) {
#pragma unroll
                  for (int v = 0; v < V; v++) o[v] = df::combine_fast(q1[v].h, q1[v].l);
                } else {
#pragma unroll
                  for (int v = 0; v < V; v++) o[v] = df::combine(q1[v].h, q1[v].l);
                }
                st_global<Sout, V>(po + (int64_t)u * M, o);
              }
            }
        } else {
          // native FP64 (cold): one row at a time
#pragma unroll 1
          for (int u = U - 1; u >= 0; u--)
            if (in_range(u)) {
              double x[1][V];
              ld_row<double, V>(sb + u * pitch, x[0]);
              bwd_block<BW, ADJ, double, V, 1, false>(c64, gs + u, 1, x, z1, z2);
              if (OUT != 0 && written(u)) st_global<Sout, V>(po + (int64_t)u * M, x[0]);
            }
        }
      }
    };

#pragma unroll 1
    for (int s = 0; s < N; s += K) {
      const int e = (s + K) < N ? (s + K) : N;
      // forward over [s, e)
      int i0 = s;
#pragma unroll 1
      for (; i0 + U <= e && i0 + D + U <= N; i0 += U) fwd(std::true_type{}, i0, U);
#pragma unroll 1
      for (; i0 < e; i0 += U) fwd(std::false_type{}, i0, (e - i0) < U ? (e - i0) : U);
      // backward from e - 1 down to lo, zero start at e; rows below hi exact
      const int hi = (e == N) ? N : ((e - Lw) > lo ? (e - Lw) : lo);
#pragma unroll
      for (int v = 0; v < V; v++) {
        y1[v] = y2[v] = 0.f;
        q1[v] = q2v[v] = wpr(0.f, 0.f);
        z1[v] = z2[v] = 0.0;
      }
      using T = std::true_type;
      using F = std::false_type;
      using O0 = std::integral_constant<int, 0>;
      using O1 = std::integral_constant<int, 1>;
      using O2 = std::integral_constant<int, 2>;
      int gs = (e - 1) & ~(U - 1);
      if (gs + U > e) {  // top group partial (last block)
        bwd(F{}, O2{}, gs, lo, e, hi);
        gs -= U;
      }
#pragma unroll 1
      for (; gs >= hi && gs >= lo; gs -= U) bwd(T{}, O0{}, gs, lo, e, hi);  // warm-up rows
      if (gs >= lo && gs + U > hi) {  // group containing hi
        bwd(T{}, O2{}, gs, lo, e, hi);
        gs -= U;
      }
#pragma unroll 1
      for (; gs >= lo; gs -= U) bwd(T{}, O1{}, gs, lo, e, hi);
      if (gs + U > lo) bwd(F{}, O2{}, gs, lo, e, hi);  // bottom group partial
      lo = hi;
    }
    cp_wait<0>();
  }
}

template <int BW, bool ADJ, int V, int R, int D, bool DFK, typename Sin, typename Sout>
cudaError_t launch_win(const SweepPlan& p, int N, int Lw, const Sin* in, Sout* out, int64_t M, cudaStream_t st) {
  const int K = (R - D - Lw) / kWU * kWU;
  if (K < kWU) return cudaErrorInvalidValue;
  WinRecs rg{};
  if constexpr (DFK) {
    const float4* f4 = reinterpret_cast<const float4*>(p.dfrec);
    rg = WinRecs{f4, f4 + N, reinterpret_cast<const float2*>(f4 + 2 * N), reinterpret_cast<const float2*>(f4 + 2 * N) + N};
  } else {
    const float4* r = reinterpret_cast<const float4*>(p.rec32);
    rg = WinRecs{r, r + N, nullptr, nullptr};
  }
  const Coefs<double> c64 = coefs_of<double>(p.c64, N);
  constexpr int SB = V * (DFK ? 8 : 4);
  const size_t rec = DFK ? (size_t)N * 48 : (size_t)N * 32;
  const size_t per_thread = (size_t)R * SB;
  // records staged in shared memory whenever some CTA size fits them (read
  // through L1/L2 instead they made the FP32 penta N = 512 solve twice as
  // slow); then 64, 128 or 256 threads (384 measured 5 % slower on the tri
  // N = 1024 batch, 32-thread CTAs stage the records too often)
  auto ks = k_sweep_win<BW, ADJ, V, R, D, true, DFK, Sin, Sout>;
  auto kg = k_sweep_win<BW, ADJ, V, R, D, false, DFK, Sin, Sout>;
  const StagedShape sh = staged_shape(M / V, rec, per_thread, kernel_regs((const void*)ks), kWinThreads, false,
                                        kWinThreads);
  if (sh.threads == 0) return cudaErrorInvalidValue;
  const bool smem = sh.staged;
  const size_t bytes = (smem ? rec : 0) + (size_t)sh.threads * per_thread;
  auto k = smem ? ks : kg;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k<<<sh.grid, sh.threads, bytes, st>>>(rg, c64, N, K, Lw, in, out, M);
  return cudaGetLastError();
}

// ring geometry per arithmetic: slots R, rows in flight D
constexpr int kRdf = 64, kDdf = 8;
constexpr int kR32 = 64, kD32 = 16;

}  // namespace

int win_rows(bool pairs) { return pairs ? kRdf - kDdf - kWU : kR32 - kD32 - kWU; }

// Windowed FP64 solve in pairs (plan p primal or adjoint), in place.
cudaError_t sweep_win_df(const SweepPlan& p, bool adjoint, int N, double* X, int64_t M, cudaStream_t st) {
  const int Lw = p.win_df;
  const bool vec2 = (M % 2 == 0) && (reinterpret_cast<uintptr_t>(X) % 16 == 0) && option(BS_OPT_F64_PAIRS) == 3;
#define BS_WIN(BWV, ADJV, VV) launch_win<BWV, ADJV, VV, kRdf, kDdf, true, double, double>(p, N, Lw, X, X, M, st)
  if (p.bw == 1) {
    if (vec2) return adjoint ? BS_WIN(1, true, 2) : BS_WIN(1, false, 2);
    return adjoint ? BS_WIN(1, true, 1) : BS_WIN(1, false, 1);
  }
  if (vec2) return adjoint ? BS_WIN(2, true, 2) : BS_WIN(2, false, 2);
  return adjoint ? BS_WIN(2, true, 1) : BS_WIN(2, false, 1);
#undef BS_WIN
}

// Windowed FP32-arithmetic solve: in (float or bf16) -> out (float); in may
// equal out for float input.
template <typename Sin>
cudaError_t sweep_win32(const SweepPlan& p, bool adjoint, int N, const Sin* in, float* out, int64_t M,
                        cudaStream_t st) {
  const int Lw = p.win32;
  // two systems per thread for large batches (bf16 input always: a lane-row
  // of input must be at least 4 bytes; the caller checks even M)
  constexpr bool kBf = !std::is_same<Sin, float>::value;
  const bool vec = kBf || ((M % 2 == 0) && (reinterpret_cast<uintptr_t>(in) % 8 == 0) &&
                           (reinterpret_cast<uintptr_t>(out) % 8 == 0) &&
                           M / 2 >= (int64_t)device_info().sms * 32 * 4);
#define BS_WIN(BWV, ADJV, VV) launch_win<BWV, ADJV, VV, kR32, kD32, false, Sin, float>(p, N, Lw, in, out, M, st)
  if constexpr (kBf) {
    if (p.bw == 1) return adjoint ? BS_WIN(1, true, 2) : BS_WIN(1, false, 2);
    return adjoint ? BS_WIN(2, true, 2) : BS_WIN(2, false, 2);
  } else {
    if (p.bw == 1) {
      if (vec) return adjoint ? BS_WIN(1, true, 2) : BS_WIN(1, false, 2);
      return adjoint ? BS_WIN(1, true, 1) : BS_WIN(1, false, 1);
    }
    if (vec) return adjoint ? BS_WIN(2, true, 2) : BS_WIN(2, false, 2);
    return adjoint ? BS_WIN(2, true, 1) : BS_WIN(2, false, 1);
  }
#undef BS_WIN
}

template cudaError_t sweep_win32<float>(const SweepPlan&, bool, int, const float*, float*, int64_t, cudaStream_t);
template cudaError_t sweep_win32<__nv_bfloat16>(const SweepPlan&, bool, int, const __nv_bfloat16*, float*, int64_t,
                                                cudaStream_t);

}  // namespace bs
