// Crank-Nicolson time steps C <- A^{-1} (2I - A) C on an interleaved batch,
// in place: the paper's benchmark problems (the periodic diffusion equation,
// Sec. 3.2-3.3, and the hyperdiffusion equation, Sec. 4.2) advance every
// system with A C^{n+1} = B C^n, where A = I - (dt/2) L is the shared LHS and
// B = I + (dt/2) L = 2I - A.  The paper forms the right-hand side with a
// separate stencil library pass; here the explicit side is applied to the
// rows as the forward sweep reads them (each thread keeps the rows it needs
// around row i in registers), so a step reads C once and writes it once plus
// the forward values' round trip of the ordinary solve.
//
// Per thread: V neighbouring systems, rows moved in blocks of U with a
// two-block register pipeline (as the plain V = 1 kernel).  The explicit
// bands e = 2I - A are formed once per CTA in shared memory (or read from
// the handle's bands in global memory for large N); in FP32 the sweep
// coefficients and the explicit bands are staged as per-row 16-byte records
// (one 128-bit load per row and use, as in the FP32 sweeps).  For a periodic handle
// the explicit side wraps around (rows 0 and N-1 are kept from the start of
// the step, before they are overwritten) and the Sherman-Morrison correction
// of the solve is applied as in the plain periodic sweeps.
#include <type_traits>

#include "df_sweep.cuh"

namespace bs {

constexpr int kCnThreads = 256;

template <int BW, bool PER, bool SMEM, typename C, int V, int U>
__global__ void __launch_bounds__(kCnThreads)
k_cn_il(Coefs<C> cf_g, const C* __restrict__ bands, int N, C* X, int64_t M) {
  constexpr int W = 2 * BW + 1;
  static_assert(U >= BW, "a block must cover the look-ahead rows");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  // FP32 with staged coefficients: records fr (forward), br (backward) and
  // er (explicit bands, one or two per row); pw, pc stay in global memory
  constexpr bool REC = SMEM && std::is_same<C, float>::value;
  constexpr int ER = BW == 1 ? 1 : 2;
  const float4* fr = reinterpret_cast<const float4*>(smem_raw);
  const float4* br = fr + N;
  const float4* er = br + N;
  Coefs<C> cf = cf_g;
  // explicit bands e_k(i) = [k == BW] * 2 - band_k(i)
  const C* eb = bands;
  if constexpr (REC) {
    float4* w4 = reinterpret_cast<float4*>(smem_raw);
    stage_records<BW, false, false>(cf_g, N, w4, w4 + N);
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      float e[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < W; k++) e[k] = (k == BW ? 2.f : 0.f) - (float)bands[(size_t)k * N + i];
      w4[2 * N + (size_t)i * ER] = make_float4(e[0], e[1], e[2], e[3]);
      if (ER == 2) w4[2 * N + (size_t)i * ER + 1] = make_float4(e[4], e[5], e[6], e[7]);
    }
    __syncthreads();
  } else {
    cf = stage_coefs<BW, false, SMEM, C, PER>(cf_g, N, sm);
    C* esm = sm + (SMEM ? coef_arrays<BW, PER>() * N : 0);
    if (SMEM) {
      for (int t = threadIdx.x; t < W * N; t += blockDim.x) esm[t] = ((t / N) == BW ? C(2) : C(0)) - bands[t];
      __syncthreads();
      eb = esm;
    }
  }
  auto e_at = [&](int k, int i) -> C {
    if (SMEM) return eb[k * N + i];
    return (k == BW ? C(2) : C(0)) - eb[k * N + i];  // e computed on the fly
  };
  const int64_t ngroups = M / V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
    C* px = X + g * V;
    auto load = [&](C (&o)[V], int row) { IO<C, C, V>::load(px + (int64_t)row * M, o); };
    C head[BW][V], prev[BW][V];
#pragma unroll
    for (int q = 0; q < BW; q++)
#pragma unroll
      for (int v = 0; v < V; v++) head[q][v] = prev[q][v] = C(0);
    if (PER) {  // rows 0..BW-1 and N-BW..N-1 before the step overwrites them
#pragma unroll
      for (int q = 0; q < BW; q++) {
        load(head[q], q);
        load(prev[q], N - BW + q);
      }
    }
    C cur[U][V], nxt[U][V], r1[V], r2[V], sig[V];
#pragma unroll
    for (int v = 0; v < V; v++) r1[v] = r2[v] = sig[v] = C(0);
#pragma unroll
    for (int u = 0; u < U; u++)
      if (u < N) load(cur[u], u);
    for (int i0 = 0; i0 < N; i0 += U) {
      const int n = (N - i0) < U ? (N - i0) : U;
#pragma unroll
      for (int u = 0; u < U; u++)
        if (i0 + U + u < N) load(nxt[u], i0 + U + u);
      // window of raw rows i0 - BW .. i0 + U - 1 + BW (all indexes static):
      // rows past N are the wrapped rows 0.. (periodic) or zero
      C win[U + 2 * BW][V];
#pragma unroll
      for (int q = 0; q < BW; q++)
#pragma unroll
        for (int v = 0; v < V; v++) win[q][v] = prev[q][v];
#pragma unroll
      for (int u = 0; u < U; u++) {
        C w[V];
#pragma unroll
        for (int v = 0; v < V; v++) w[v] = cur[u][v];
        if (u >= n) {  // row i0 + u >= N: the wrapped row u - n
#pragma unroll
          for (int v = 0; v < V; v++) w[v] = C(0);
          if (PER) {
#pragma unroll
            for (int q = 0; q < BW; q++)
              if (u - n == q)
#pragma unroll
                for (int v = 0; v < V; v++) w[v] = head[q][v];
          }
        }
#pragma unroll
        for (int v = 0; v < V; v++) win[BW + u][v] = w[v];
      }
#pragma unroll
      for (int q = 0; q < BW; q++) {
        const bool in = i0 + U + q < N;
#pragma unroll
        for (int v = 0; v < V; v++) win[BW + U + q][v] = in ? nxt[q][v] : (PER ? head[q][v] : C(0));
      }
      // F = e applied to the window
      C f[U][V];
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (u < n) {
          const int i = i0 + u;
          C e[W];
          if constexpr (REC) {
            const float4 a = er[(size_t)i * ER];
            const float ev[8] = {a.x, a.y, a.z, a.w, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < W && k < 4; k++) e[k] = ev[k];
            if constexpr (ER == 2) e[4] = er[(size_t)i * ER + 1].x;
          } else {
#pragma unroll
            for (int k = 0; k < W; k++) e[k] = e_at(k, i);
          }
#pragma unroll
          for (int v = 0; v < V; v++) {
            C sacc = e[0] * win[u][v];
#pragma unroll
            for (int k = 1; k < W; k++) sacc = fma(e[k], win[u + k][v], sacc);
            f[u][v] = sacc;
          }
        }
      }
      // raw rows i0 + n - BW .. i0 + n - 1 become the previous rows
      if (n == U) {
#pragma unroll
        for (int q = 0; q < BW; q++)
#pragma unroll
          for (int v = 0; v < V; v++) prev[q][v] = cur[U - BW + q][v];
      }
      if constexpr (PER)
        if (i0 < cf.per_lo || i0 + n > cf.per_hi) per_dot<C, V, U>(cf, i0, n, f, sig);
      if constexpr (REC)
        fwd_block_rec<BW, false, V, U, false>(fr, 0.f, i0, n, f, r1, r2);
      else
        fwd_block<BW, false, C, V, U>(cf, i0, n, f, r1, r2);
#pragma unroll
      for (int u = 0; u < U; u++)
        if (u < n) IO<C, C, V>::store(px + (int64_t)(i0 + u) * M, f[u]);
#pragma unroll
      for (int u = 0; u < U; u++)
#pragma unroll
        for (int v = 0; v < V; v++) cur[u][v] = nxt[u][v];
    }
    // backward sweep over the forward values, as in the plain solve, with the
    // next block's loads issued before the current block is computed
#pragma unroll
    for (int v = 0; v < V; v++) r1[v] = r2[v] = C(0);
    auto load_bwd = [&](C (&blk)[U][V], int top) {
#pragma unroll
      for (int u = 0; u < U; u++)
        if (top - u >= 0) load(blk[u], top - u);
    };
    auto run_bwd = [&](C (&blk)[U][V], int top) {
      const int n = (top + 1) < U ? (top + 1) : U;
      if constexpr (REC)
        bwd_block_rec<BW, false, V, U, false>(br, 0.f, top, n, blk, r1, r2);
      else
        bwd_block<BW, false, C, V, U>(cf, top, n, blk, r1, r2);
      if constexpr (PER)
        if (top + 1 - n < cf.per_lo || top + 1 > cf.per_hi) per_fix<C, V, U>(cf, top, n, blk, sig);
#pragma unroll
      for (int u = 0; u < U; u++)
        if (u < n) IO<C, C, V>::store(px + (int64_t)(top - u) * M, blk[u]);
    };
    load_bwd(cur, N - 1);
    for (int top = N - 1; top >= 0; top -= 2 * U) {
      if (top - U >= 0) load_bwd(nxt, top - U);
      run_bwd(cur, top);
      if (top - U < 0) break;
      if (top - 2 * U >= 0) load_bwd(cur, top - 2 * U);
      run_bwd(nxt, top - U);
    }
  }
}

template <int BW, bool PER, typename C, int V>
static cudaError_t launch_cn(const SweepPlan& p, const C* bands, int N, C* X, int64_t M, cudaStream_t st) {
  constexpr int U = 8;
  const C* base;
  if constexpr (sizeof(C) == 8)
    base = reinterpret_cast<const C*>(p.c64);
  else
    base = reinterpret_cast<const C*>(p.c32);
  Coefs<C> cf = coefs_of<C>(base, N);
  cf.per_lo = p.per_lo;
  cf.per_hi = p.per_hi;
  const int64_t groups = M / V;
  // the explicit bands add 2 BW + 1 arrays to the staged coefficients
  // 256-thread CTAs when the batch fills the device: the staged coefficient
  // and explicit-band arrays are shared by twice the threads
  const int tpb = groups >= (int64_t)device_info().sms * kCnThreads ? kCnThreads : 0;
  // FP32: records of 16 bytes, 2 + (1 or 2) per row
  constexpr int kExtra = sizeof(C) == 4 ? 4 * (2 + (BW == 1 ? 1 : 2)) - (1 + 2 * BW) : (PER ? 2 : 0) + 2 * BW + 1;
  const LaunchShape sh = sweep_shape(BW, N, groups, sizeof(C), sizeof(C), V, 0, 0, tpb, kExtra);
  if (sh.smem_coefs) {
    auto k = k_cn_il<BW, PER, true, C, V, U>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
    if (e != cudaSuccess) return e;
    k<<<sh.grid, sh.threads, sh.smem, st>>>(cf, bands, N, X, M);
  } else {
    k_cn_il<BW, PER, false, C, V, U><<<sh.grid, sh.threads, 0, st>>>(cf, bands, N, X, M);
  }
  return cudaGetLastError();
}

// ------------------------------------------------ FP64 steps in FP32 pairs
//
// The native FP64 kernel above issues 2 W FP64 instructions per unknown (the
// explicit product and the two sweeps), so the FP64 pipe bounds it.  For an
// FP64 batch whose handle allows pairs (cn_pairs: the band entries and the
// explicit side's row sums in range, factor.cpp; and the pair sweeps' own
// check) a step runs instead in k_cn_df: the FP64 solve in FP32 pairs of
// sweep_df.cu whose forward sweep takes as its input the explicit side
// (2I - A) C, formed in pairs from the rows as they arrive -- each product
// e_k(i) C_{i+k-BW} a TwoProduct of the high parts plus the two cross terms,
// the sum TwoSums of the high parts with the rest in the low part -- so a
// step reads C once and writes it once plus the forward values' round trip.
// Measured (penta N = 512, M = 65536, ms per step): native 0.682; an
// explicit pass in pairs followed by the pair solve 0.396; fused 0.315.
//
// One thread per system; input rows arrive through the per-lane ring in
// blocks of 4 (rows 4b .. 4b+3 at step b), the thread keeps the window of
// input rows 4b - 2 BW .. 4b + 3 as pairs and FP64 values, and the forward
// sweep runs BW rows behind, over rows 4b - BW .. 4b + 3 - BW.
// A row's ring slot is refilled with row + D as soon as the row enters the
// window; the forward values of the last D rows stay in their slots, the
// others go to C in place, and the backward sweep is the pair solve's
// (df_sweep_backward).  A lane that meets an input outside the pairs' range
// runs the rest of its system in FP64 from the current block of rows on; the
// range is |C| < 2^97 (the explicit side's row sums are at most 16, so the
// sweep's inputs stay below the pair solve's 2^101), for a periodic handle
// 2^76 (its Sherman-Morrison sum then stays inside FP32, see df_sweep.cuh).
//
// PER (periodic tridiagonal handle): the explicit side wraps around -- row
// -1 of the window is C_{N-1}, read before the sweep, and row N is C_0,
// kept from the first block -- and the forward sweep accumulates the
// Sherman-Morrison sum over the explicit side's rows, the backward sweep
// applies the correction (df_sweep_backward with PER).
constexpr int kCnFusedThreadsMax = 512;

// |v| < 2^e (or v zero / any value below; NaN and inf fail)
template <int E>
__device__ __forceinline__ bool cn_pair_small(double v) {
  return ((uint32_t)__double2hiint(v) & 0x7fffffffu) < ((1023u + E) << 20);
}

template <int BW, bool SMEM, int D, bool PER>
__global__ void __launch_bounds__(kCnFusedThreadsMax)
k_cn_df(DfRecs rg, Coefs<double> c64, const float* __restrict__ bhi, const float* __restrict__ blo,
        const double* __restrict__ b64, int N, double* X, int64_t M) {
  constexpr int W = 2 * BW + 1;
  constexpr int U = 4;
  constexpr int NW = 2 * BW + U;
  constexpr int kTop = PER ? 76 : 97;
  static_assert(D % U == 0, "ring depth must be a multiple of the block");
  static_assert(!PER || BW == 1, "periodic handles are tridiagonal");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DfRecs rc = rg;
  size_t rec_bytes = 0;
  float2* bp = reinterpret_cast<float2*>(smem_raw);  // band pairs, bp[i W + k]
  if constexpr (SMEM) {
    constexpr bool F2 = DfCount<false, BW>::F > 2, B2 = DfCount<false, BW>::B > 2;
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
    bp = reinterpret_cast<float2*>(pq + (PER ? N : 0));
    rec_bytes = (size_t)N * (PER ? 64 : 48);
  }
  for (int t = threadIdx.x; t < N * W; t += blockDim.x) {
    const int i = t / W, k = t - i * W;
    bp[t] = make_float2(bhi[(size_t)k * N + i], blo[(size_t)k * N + i]);
  }
  __syncthreads();
  unsigned char* ring =
      smem_raw + align_up(rec_bytes + (size_t)N * W * sizeof(float2), 16) + (size_t)threadIdx.x * 8;
  const uint32_t ring_s = smem_u32(ring);
  const uint32_t pitch = blockDim.x * 8;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M; j += stride) {
    double* const pout = X + j;
    DfState<1> st;
    st.reset_values();
    if (PER) st.reset_sigma();
    st.f64 = false;
    st.rsw = N;
    double c0 = 0.0;  // periodic: C_0, row N of the window
    const double* pnext = pout;
#pragma unroll 1
    for (int r = 0; r < D; r++) {
      if (r < N) cp_async8(ring_s + r * pitch, pnext);
      pnext += M;
      if ((r + 1) % U == 0) cp_commit();
    }
    df::Pair y[NW];
    double d[NW];
#pragma unroll
    for (int q = 0; q < NW; q++) {
      y[q] = df::Pair{0.f, 0.f};
      d[q] = 0.0;
    }
    if constexpr (PER) {  // row -1 of the first window: C_{N-1}
      const double v = pout[(int64_t)(N - 1) * M];
      d[NW - 1] = v;
      bool ok = df::split_fast(v, y[NW - 1]) && cn_pair_small<kTop>(v);
      if (!ok) {
        ok = true;
        y[NW - 1] = df::split(v, ok);
        if (!(ok && cn_pair_small<kTop>(v))) {
          st.f64 = true;
          st.rsw = 0;
        }
      }
    }
    double* prow = pout - (int64_t)BW * M;  // forward output row 4b - BW
#pragma unroll 1
    for (int r0 = 0; r0 - BW < N; r0 += U) {
      cp_wait<D / U - 1>();
#pragma unroll
      for (int q = 0; q < 2 * BW; q++) {
        y[q] = y[q + U];
        d[q] = d[q + U];
      }
      const int s0 = r0 % D;
      bool need = false;
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int r = r0 + u;
        double v = 0.0;
        if (r < N) v = *reinterpret_cast<const double*>(ring + (size_t)(s0 + u) * pitch);
        if (PER && r == 0) c0 = v;
        if (PER && r == N) v = c0;
        d[2 * BW + u] = v;
        y[2 * BW + u] = df::Pair{0.f, 0.f};
        if ((r < N || (PER && r == N)) && !st.f64)
          need |= !df::split_fast(v, y[2 * BW + u]) || !cn_pair_small<kTop>(v);
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (r0 + u + D < N) cp_async8(ring_s + (s0 + u) * pitch, pnext);
        pnext += M;
      }
      cp_commit();
      const int i0 = r0 - BW;  // forward rows i0 .. i0 + 3 (those in [0, N))
      if (__any_sync(__activemask(), need)) {
        if (need) {  // zeros or range edges: the careful split, or FP64 from here on
          bool bad = false;
#pragma unroll
          for (int u = 0; u < U; u++) {
            bool ok = true;
            y[2 * BW + u] = df::split(d[2 * BW + u], ok);
            bad |= !(ok && cn_pair_small<kTop>(d[2 * BW + u]));
          }
          if (bad && !st.f64) {
            st.f64 = true;
            st.rsw = i0 > 0 ? i0 : 0;
            st.d1[0] = pair_to_f64(st.p1[0]);
            st.d2[0] = pair_to_f64(st.p2[0]);
            if (PER) st.dsig[0] = pair_to_f64(st.sig[0]) * rc.per_unscale;
          }
        }
      }
      uint2 wout[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int i = i0 + u;
        wout[u] = make_uint2(0u, 0u);
        if (i < 0 || i >= N) continue;
        const float2* ci = bp + (size_t)i * W;
        if (!st.f64) {
          // f = (2I - A) C at row i in pairs: window entries u .. u + 2 BW
          float sh = df::mul(2.f, y[u + BW].h), lo = df::mul(2.f, y[u + BW].l);
#pragma unroll
          for (int k = 0; k < W; k++) {
            const float2 c = ci[k];
            const df::Pair z = y[u + k];
            const float p = df::mul(c.x, z.h);
            float e = df::fma_(c.x, z.h, -p);
            e = df::fma_(c.x, z.l, e);
            e = df::fma_(c.y, z.h, e);
            float t;
            df::two_sum(sh, -p, sh, t);
            lo = df::add(lo, df::sub(t, e));
          }
          df::Pair f;
          df::fast_two_sum(sh, lo, f.h, f.l);
          if (PER && (i < c64.per_lo || i >= c64.per_hi)) {  // sigma' += pw'_i f_i
            const float4 w = rc.pq[i];
            st.sig[0] = df_muladd(st.sig[0], w.x, w.y, f);
          }
          const float4 q = rc.f4[i];
          const float2 q2 = BW == 2 ? rc.f2[i] : make_float2(0.f, 0.f);
          const df::Pair w = df_row<true, BW>(q, q2, f, st.p1[0], st.p2[0]);
          st.p2[0] = st.p1[0];
          st.p1[0] = w;
          wout[u] = pair_bits(w);
        } else {
          double f[1] = {2.0 * d[u + BW]};
#pragma unroll
          for (int k = 0; k < W; k++) f[0] = fma(-b64[(size_t)k * N + i], d[u + k], f[0]);
          if (PER && (i < c64.per_lo || i >= c64.per_hi)) st.dsig[0] = fma(c64.pw[i], f[0], st.dsig[0]);
          fwd_step<BW, false, double, 1>(c64, i, f, st.d1, st.d2);
          wout[u] = f64_bits(f[0]);
        }
      }
      // the forward values: the last D rows stay in their ring slots (not
      // refilled), the others go to C
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int i = i0 + u;
        if (i >= 0 && i < N) {
          if (i + D >= N)
            *reinterpret_cast<uint2*>(ring + (size_t)(i % D) * pitch) = wout[u];
          else
            *reinterpret_cast<uint2*>(prow) = wout[u];
        }
        prow += M;
      }
    }
    cp_wait<0>();
    df_sweep_backward<BW, false, 1, D, PER>(rc, c64, N, pout, M, ring, ring_s, pitch, st);
  }
}

// FP64 steps try the fused pair kernel when the handle allows pairs (the
// launch then checks that its staged records, band pairs and rings fit in
// shared memory).
static bool cn_pair_path(bs_handle h) {
  return h->cn_pairs && df_eligible(h->plan[0], BS_INTERLEAVED);
}

// The fused step; cudaErrorInvalidValue (nothing launched) when the staged
// records, band pairs and rings do not fit in shared memory.  CTA size from
// the busiest-SM model with ties to the largest (penta N = 512, M = 65536:
// 64-thread CTAs, four per SM by shared memory, 0.442 ms; ties to the largest
// 0.315 ms).
template <int BW, bool PER>
static cudaError_t launch_cn_df(bs_handle h, double* X, int64_t M, cudaStream_t st) {
  constexpr int D = 16;  // rows in flight per lane
  const int N = (int)h->N;
  const SweepPlan& p = h->plan[0];
  DfRecs rg = df_recs_of(p.dfrec, N);
  Coefs<double> c64 = coefs_of<double>(p.c64, N);
  if (PER) {
    rg.pq = reinterpret_cast<const float4*>(p.dfper);
    rg.per_unscale = p.dfper_unscale;
    c64.per_lo = p.per_lo;
    c64.per_hi = p.per_hi;
  }
  const size_t rec = align_up((size_t)N * (PER ? 64 : 48) + (size_t)N * (2 * BW + 1) * sizeof(float2), 16);
  auto k = k_cn_df<BW, true, D, PER>;
  const StagedShape sh =
      staged_shape(M, rec, (size_t)D * 8, kernel_regs((const void*)k), kCnFusedThreadsMax, true, kCnFusedThreadsMax);
  if (sh.threads == 0 || !sh.staged) return cudaErrorInvalidValue;
  const size_t bytes = rec + (size_t)sh.threads * D * 8;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k<<<sh.grid, sh.threads, bytes, st>>>(rg, c64, h->bands_hi, h->bands_lo, h->bands64, N, X, M);
  return cudaGetLastError();
}

template <typename C, int VEC>
static cudaError_t cn_dispatch(bs_handle h, C* X, int64_t M, cudaStream_t st) {
  if constexpr (sizeof(C) == 8) {
    if (cn_pair_path(h)) {  // the explicit side fused into the pair solve
      const cudaError_t e = h->periodic     ? launch_cn_df<1, true>(h, X, M, st)
                            : h->width == 3 ? launch_cn_df<1, false>(h, X, M, st)
                                            : launch_cn_df<2, false>(h, X, M, st);
      if (e != cudaErrorInvalidValue) return e;  // else: too large for shared memory, native below
    }
  }
  const SweepPlan& p = h->plan[0];
  const int N = (int)h->N;
  const C* bands;
  if constexpr (sizeof(C) == 8)
    bands = reinterpret_cast<const C*>(h->bands64);
  else
    bands = reinterpret_cast<const C*>(h->bands_hi);
  // systems per thread: the widest vector that still gives every SM at
  // least 256 threads (the FP64 pipe and the loads need the warps more than
  // the wide loads)
  const int64_t want = (int64_t)device_info().sms * 256;
  const uintptr_t a = reinterpret_cast<uintptr_t>(X);
  int v = 1;
  if (M % VEC == 0 && a % (VEC * sizeof(C)) == 0 && M / VEC >= want)
    v = VEC;
  else if (M % 2 == 0 && a % (2 * sizeof(C)) == 0 && M / 2 >= want)
    v = 2;
  auto go = [&](auto bwt, auto pert) -> cudaError_t {
    constexpr int BW = decltype(bwt)::value;
    constexpr bool PER = decltype(pert)::value;
    if (v == VEC) return launch_cn<BW, PER, C, VEC>(p, bands, N, X, M, st);
    if (v == 2) return launch_cn<BW, PER, C, 2>(p, bands, N, X, M, st);
    return launch_cn<BW, PER, C, 1>(p, bands, N, X, M, st);
  };
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  if (h->periodic) return go(I1{}, std::true_type{});
  if (h->width == 3) return go(I1{}, std::false_type{});
  return go(I2{}, std::false_type{});
}

}  // namespace bs

extern "C" bs_status bs_cn_steps(bs_handle h, void* C, bs_dtype dtype, bs_layout layout, int64_t M, int steps,
                                 bs_stream stream) {
  using namespace bs;
  if (!valid_handle(h)) return set_error(BS_EINVAL, "bs_cn_steps: unknown handle");
  if (!C) return set_error(BS_EINVAL, "bs_cn_steps: null data pointer");
  if (M < 1) return set_error(BS_EINVAL, "bs_cn_steps: M must be >= 1");
  if (steps < 0) return set_error(BS_EINVAL, "bs_cn_steps: steps must be >= 0");
  if (dtype != BS_F64 && dtype != BS_F32) return set_error(BS_EINVAL, "bs_cn_steps: dtype must be BS_F64 or BS_F32");
  if (layout != BS_INTERLEAVED)
    return set_error(BS_EUNSUPPORTED, "bs_cn_steps: only the interleaved layout is implemented");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) return set_error(BS_EINVAL, "bs_cn_steps: handle belongs to another device");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (int n = 0; n < steps; n++) {
    const cudaError_t e = dtype == BS_F64 ? cn_dispatch<double, 2>(h, static_cast<double*>(C), M, st)
                                          : cn_dispatch<float, 4>(h, static_cast<float*>(C), M, st);
    if (e != cudaSuccess) return cuda_error(e, "bs_cn_steps launch");
  }
  return BS_OK;
}
