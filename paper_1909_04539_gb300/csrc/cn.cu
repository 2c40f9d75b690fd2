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

template <typename C, int VEC>
static cudaError_t cn_dispatch(bs_handle h, C* X, int64_t M, cudaStream_t st) {
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
