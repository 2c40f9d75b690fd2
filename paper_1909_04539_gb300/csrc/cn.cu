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

#include "df_math.cuh"
#include "sweep_kernels.cuh"

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
// check) a step runs instead as two passes: the explicit side X <- (2I - A) X
// in FP32 pairs (k_cn_explicit_df, in place, each value rounded once to
// FP64), then the FP64 solve in pairs (sweep_df.cu).
//
// One thread per system; the rows arrive through a per-lane cp.async ring of
// kCnDfD slots, one copy group per block of 4 input rows; after the block of
// input rows r0 .. r0+3 the thread holds the window of rows r0 - 2 BW ..
// r0 + 3, as pairs and as the FP64 values, and forms the output rows
// r0 - BW .. r0 + 3 - BW (the rows it overwrites have all been read).  (Rows
// cut into blocks of 128 per thread, for four times the threads, need the
// result in a second batch -- neighbouring blocks read each other's rows --
// and measured slower with the copy back: penta N = 512, M = 65536, one step
// 0.446 against 0.397 ms.)  Each
// product e_k(i) C_{i+k-BW} is a TwoProduct of the high parts plus the two
// cross terms, the sum TwoSums of the high parts with the rest in the low
// part, as in the pair sweeps.  A lane that meets an input outside the pairs'
// range computes the rest of its system with FP64 FMAs, so each result
// depends only on its own system.  The band entries are staged per CTA as
// (hi, lo) pairs.
constexpr int kCnDfThreads = 256;
constexpr int kCnDfD = 16;

template <int BW>
__global__ void __launch_bounds__(kCnDfThreads)
k_cn_explicit_df(const float* __restrict__ bhi, const float* __restrict__ blo, const double* __restrict__ b64,
                 int N, double* X, int64_t M) {
  constexpr int W = 2 * BW + 1;
  constexpr int U = 4;
  constexpr int D = kCnDfD;
  constexpr int NW = 2 * BW + U;  // window: input rows r0 - 2 BW .. r0 + 3
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* rec = reinterpret_cast<float2*>(smem_raw);  // rec[i W + k]: band k of row i as (hi, lo)
  for (int t = threadIdx.x; t < N * W; t += blockDim.x) {
    const int i = t / W, k = t - i * W;
    rec[t] = make_float2(bhi[(size_t)k * N + i], blo[(size_t)k * N + i]);
  }
  __syncthreads();
  unsigned char* ring = smem_raw + align_up((size_t)N * W * sizeof(float2), 16) + (size_t)threadIdx.x * 8;
  const uint32_t ring_s = smem_u32(ring);
  const uint32_t pitch = blockDim.x * 8;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M; j += stride) {
    double* const px = X + j;
    const double* pnext = px;  // next input row to request
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
    bool f64 = false;  // this lane runs FP64 FMAs from here on
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
        d[2 * BW + u] = v;
        y[2 * BW + u] = df::Pair{0.f, 0.f};
        if (r < N && !f64) need |= !df::split_fast(v, y[2 * BW + u]);
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        if (r0 + u + D < N) cp_async8(ring_s + (s0 + u) * pitch, pnext);
        pnext += M;
      }
      cp_commit();
      if (__any_sync(__activemask(), need)) {
        if (need) {  // zeros or range edges: the careful split, or FP64 from here on
#pragma unroll
          for (int u = 0; u < U; u++) {
            bool ok = true;
            y[2 * BW + u] = df::split(d[2 * BW + u], ok);
            f64 |= !ok;
          }
        }
      }
      // output rows i = r0 + u - BW: window entries u .. u + 2 BW
      double out[U];
      float oh[U], ol[U];
      bool odd = false;
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int i = r0 + u - BW;
        out[u] = 0.0;
        if (i < 0 || i >= N) continue;
        const float2* ci = rec + (size_t)i * W;
        if (!f64) {
          float s = df::mul(2.f, y[u + BW].h), lo = df::mul(2.f, y[u + BW].l);
#pragma unroll
          for (int k = 0; k < W; k++) {
            const float2 c = ci[k];
            const df::Pair z = y[u + k];
            const float p = df::mul(c.x, z.h);
            float e = df::fma_(c.x, z.h, -p);
            e = df::fma_(c.x, z.l, e);
            e = df::fma_(c.y, z.h, e);
            float t;
            df::two_sum(s, -p, s, t);
            lo = df::add(lo, df::sub(t, e));
          }
          df::fast_two_sum(s, lo, oh[u], ol[u]);
          odd |= !df::combine_ok(oh[u]);
          out[u] = df::combine_fast(oh[u], ol[u]);  // replaced below where !combine_ok
        } else {
          double f = 2.0 * d[u + BW];
#pragma unroll
          for (int k = 0; k < W; k++) f = fma(-b64[(size_t)k * N + i], d[u + k], f);
          out[u] = f;
        }
      }
      if (__any_sync(__activemask(), odd)) {
        if (odd) {  // results below 2^-70 (zeros): the careful combination
#pragma unroll
          for (int u = 0; u < U; u++) {
            const int i = r0 + u - BW;
            if (i >= 0 && i < N && !f64 && !df::combine_ok(oh[u])) out[u] = df::combine(oh[u], ol[u]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int i = r0 + u - BW;
        if (i >= 0 && i < N) px[(int64_t)i * M] = out[u];
      }
    }
    cp_wait<0>();
  }
}

static size_t cn_df_smem(int width, int64_t N) {
  return align_up((size_t)N * width * sizeof(float2), 16) + (size_t)kCnDfThreads * kCnDfD * 8;
}

// FP64 steps take the pair passes when the handle allows them and the staged
// band pairs and rings fit in shared memory.
static bool cn_pair_path(bs_handle h) {
  const DeviceInfo& d = device_info();
  const size_t limit = (size_t)(d.smem_optin > 0 ? d.smem_optin : 48 * 1024);
  return h->cn_pairs && df_eligible(h->plan[0], BS_INTERLEAVED) && cn_df_smem(h->width, h->N) <= limit;
}

template <int BW>
static cudaError_t launch_cn_explicit_df(bs_handle h, double* X, int64_t M, cudaStream_t st) {
  const int N = (int)h->N;
  const size_t bytes = cn_df_smem(2 * BW + 1, N);
  auto k = k_cn_explicit_df<BW>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kCnDfThreads, bytes);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)device_info().sms * per_sm;
  const int64_t need = (M + kCnDfThreads - 1) / kCnDfThreads;
  if (grid > need) grid = need;
  k<<<(int)grid, kCnDfThreads, bytes, st>>>(h->bands_hi, h->bands_lo, h->bands64, N, X, M);
  return cudaGetLastError();
}

template <typename C, int VEC>
static cudaError_t cn_dispatch(bs_handle h, C* X, int64_t M, cudaStream_t st) {
  if constexpr (sizeof(C) == 8) {
    if (cn_pair_path(h)) {  // explicit side, then the solve, both in pairs
      const cudaError_t e =
          h->width == 3 ? launch_cn_explicit_df<1>(h, X, M, st) : launch_cn_explicit_df<2>(h, X, M, st);
      if (e != cudaSuccess) return e;
      return sweep_df(h->plan[0], false, (int)h->N, X, M, st);
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
