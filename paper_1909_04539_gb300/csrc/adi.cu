// Peaceman-Rachford ADI half-step for u_t = u_xx + u_yy on a 2D grid
// u[y * nx + x] with homogeneous Dirichlet boundaries (zero outside):
//   implicit along x:  S_x out = E_y u,   S_x = the factorised LHS along x,
//                                        E_y = I + r d2/dy2 (second difference)
//   implicit along y:  S_y out = E_x u.
// The shared LHS (for the heat equation I - r d2, one tridiagonal copy for all
// grid lines; the paper's motivation, Sec. 1) is the handle.  The explicit
// operator acts across systems, so it is applied while the forward sweep loads
// its rows (one neighbour on each side), and the result goes to a separate
// output buffer: the sweep cannot overwrite u in place because neighbouring
// systems still read it.
//
// Adjoint: for the map u -> S^{-1} E u the transpose is E^T S^{-T}.  E and S
// act on different axes and therefore commute, and E is symmetric, so the
// adjoint is the same fused step with the adjoint sweep coefficients.
//
// Implicit along y: system j = column x, row i = y, at u[i * nx + j]
//   (interleaved, M = nx).  Implicit along x: system j = row y, row i = x, at
//   u[j * nx + i] (system-contiguous); a warp moves 32 rows of 34 systems (its
//   32 plus one neighbour each side) through a shared-memory tile.
#include <type_traits>

#include "sweep_kernels.cuh"

namespace bs {

// FP64 primal plans with staged coefficients fold the forward sweep's row
// scale s_i into the explicit operator: s_i (c + r (left - 2c + right)) =
// e0_i c + e1_i (left + right) with e0_i = s_i (1 - 2r), e1_i = s_i r, staged
// once per CTA as one 16-byte pair per row (ahead of the plan's arrays, so a
// row still takes two shared loads in the tridiagonal case).  Per unknown
// that is one ADD, one MUL and one FMA before the unscaled forward
// recurrence, against two FMAs, an ADD and the scale's MUL: one FP64
// instruction fewer, and the FP64 half-steps are bound by the FP64 pipe.
// (FP32 half-steps are bound by latency and keep the plain form.)
__device__ __forceinline__ void fuse_explicit(const double* s, double2* pr, int N, double r) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double si = s[i];
    pr[i] = make_double2(si * (1.0 - 2.0 * r), si * r);
  }
  __syncthreads();
}

// Forward block of the fused step: f[u] holds the centre value c and nb[u]
// the sum of the two neighbours of row i0 + u on entry, the forward value
// w = e0 c + e1 nb - l2 w2 - l1 w1 on exit.  All coefficient loads are issued
// first, as in fwd_block.
template <int BW, int U>
__device__ __forceinline__ void adi_fwd_fused(const Coefs<double>& cf, const double2* pr, int i0, int n,
                                              double (&f)[U][1], const double (&nb)[U], double (&w1)[1],
                                              double (&w2)[1]) {
  double2 e[U];
  double l1[U], l2[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    const int i = (u < n) ? i0 + u : i0;
    e[u] = pr[i];
    l1[u] = cf.l1[i];
    l2[u] = BW == 2 ? cf.l2[i] : 0.0;
  }
#pragma unroll
  for (int u = 0; u < U; u++) {
    if (u < n) {
      double w = fma(e[u].y, nb[u], e[u].x * f[u][0]);
      if (BW == 2) w = fma(-l2[u], w2[0], w);
      w = fma(-l1[u], w1[0], w);
      if (BW == 2) w2[0] = w1[0];
      w1[0] = w;
      f[u][0] = w;
    }
  }
}

// Shared elements (of C) ahead of the plan's staged arrays: the (e0, e1)
// pairs of a fused launch.
template <typename C, bool FUSE>
__host__ __device__ constexpr size_t fuse_elems(int N) {
  return FUSE ? (size_t)N * 2 : 0;
}

// ----------------------------------------------------- implicit along y

// Y-implicit half-step: one warp owns 32
// consecutive columns (systems), each lane streams its column's rows through
// a ring of D slots in shared memory (cp.async), so D rows per lane are in
// flight -- with 4096 grid lines there is less than one warp per SM, so depth
// has to come from each lane.  The explicit operator needs the neighbouring
// columns' values: inside the warp they come from the adjacent lanes by
// shuffle, the two outer neighbours are copied by lanes 0 and 31 into a second
// half of their slots.  The forward values go to `out` and come back through
// the same ring for the backward sweep.
template <int BW, bool ADJ, bool SMEM, typename C, int D>
__global__ void __launch_bounds__(kSweepThreads)
k_adi_il2(Coefs<C> cf_g, int N, const C* __restrict__ u, C* __restrict__ out, int64_t M, C r, int L) {
  constexpr int U = 4;
  static_assert(D % U == 0, "ring depth must be a multiple of the block");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  {  // row block of a partitioned launch (blockIdx.y; L = N otherwise)
    const int r0 = blockIdx.y * L;
    N = (N - r0) < L ? (N - r0) : L;
    cf_g = shift_coefs(cf_g, r0);
    u += (int64_t)r0 * M;
    out += (int64_t)r0 * M;
  }
  // FP32 with staged coefficients: one 16-byte record per row and sweep
  // (stage_records)
  constexpr bool REC = SMEM && std::is_same<C, float>::value;
  const float4* fr = reinterpret_cast<const float4*>(smem_raw);
  const float4* br = fr + N;
  constexpr bool FUSE = SMEM && !ADJ && sizeof(C) == 8;
  Coefs<C> cf = cf_g;
  const double2* pr = reinterpret_cast<const double2*>(smem_raw);
  size_t coef_bytes;
  if constexpr (REC) {
    stage_records<BW, ADJ, false>(cf_g, N, reinterpret_cast<float4*>(smem_raw), reinterpret_cast<float4*>(smem_raw) + N);
    coef_bytes = (size_t)N * 2 * sizeof(float4);
  } else {
    C* smc = reinterpret_cast<C*>(smem_raw) + fuse_elems<C, FUSE>(N);
    cf = stage_coefs<BW, ADJ, SMEM>(cf_g, N, smc);
    if constexpr (FUSE) fuse_explicit(cf.s, reinterpret_cast<double2*>(smem_raw), N, r);
    coef_bytes = SMEM ? align_up((fuse_elems<C, FUSE>(N) + (size_t)coef_arrays<BW>() * N) * sizeof(C), 16) : 0;
  }
  const int lane = threadIdx.x & 31;
  // slot layout per lane: [own value | outer neighbour], 2 * sizeof(C) bytes
  constexpr int kSlot = 2 * sizeof(C);
  unsigned char* ring = smem_raw + coef_bytes + (size_t)threadIdx.x * kSlot;
  const uint32_t ring_s = smem_u32(ring);
  const uint32_t pitch = blockDim.x * kSlot;
  const int64_t nwarps_total = (int64_t)gridDim.x * (blockDim.x / 32);
  const int64_t ngroups = (M + 31) / 32;
  auto cp = [&](uint32_t dst, const C* src) {
    if constexpr (sizeof(C) == 8)
      cp_async8(dst, src);
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
  };
  for (int64_t wg = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); wg < ngroups; wg += nwarps_total) {
    const int64_t j = wg * 32 + lane;
    const bool valid = j < M;
    // the column this lane copies into the second half of its slot, if any
    const int64_t jn = lane == 0 ? j - 1 : (lane == 31 ? j + 1 : -1);
    const bool has_n = (lane == 0 || lane == 31) && jn >= 0 && jn < M;
    const C* pu = u + (valid ? j : 0);
    const C* pn = u + (has_n ? jn : 0);
    C* po = out + (valid ? j : 0);
    auto request = [&](int slot, int row) {
      if (valid) cp(ring_s + slot * pitch, pu + (int64_t)row * M);
      if (has_n) cp(ring_s + slot * pitch + sizeof(C), pn + (int64_t)row * M);
    };
    C r1[1] = {C(0)}, r2[1] = {C(0)};
#pragma unroll 1
    for (int q = 0; q < D; q++) {
      if (q < N) request(q, q);
      cp_commit();
    }
#pragma unroll 1
    for (int i0 = 0; i0 < N; i0 += U) {
      cp_wait<D - U>();
      __syncwarp();
      const int n = (N - i0) < U ? (N - i0) : U;
      const int s0 = i0 % D;
      C f[U][1], nb[U];
#pragma unroll
      for (int q = 0; q < U; q++) {
        const C* sl = reinterpret_cast<const C*>(ring + (size_t)(s0 + q) * pitch);
        const C c = valid ? sl[0] : C(0);
        const C outer = has_n ? sl[1] : C(0);
        C left = __shfl_up_sync(0xffffffffu, c, 1);
        C right = __shfl_down_sync(0xffffffffu, c, 1);
        if (lane == 0) left = outer;
        if (lane == 31) right = outer;
        if constexpr (FUSE) {
          f[q][0] = c;
          nb[q] = left + right;
        } else {
          f[q][0] = c + r * (left - C(2) * c + right);
        }
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < U; q++) {
        if (q < n && i0 + q + D < N) request(s0 + q, i0 + q + D);
        cp_commit();
      }
      if (valid) {
        if constexpr (FUSE)
          adi_fwd_fused<BW, U>(cf, pr, i0, n, f, nb, r1, r2);
        else if constexpr (REC)
          fwd_block_rec<BW, ADJ, 1, U, false>(fr, 0.f, i0, n, f, r1, r2);
        else
          fwd_block<BW, ADJ, C, 1, U>(cf, i0, n, f, r1, r2);
#pragma unroll
        for (int q = 0; q < U; q++)
          if (q < n) po[(int64_t)(i0 + q) * M] = f[q][0];
      }
    }
    cp_wait<0>();
    __syncwarp();
    // backward sweep: the lane's own forward values come back through the ring
    r1[0] = r2[0] = C(0);
#pragma unroll 1
    for (int q = 0; q < D; q++) {
      const int row = N - 1 - q;
      if (row >= 0 && valid) cp(ring_s + q * pitch, po + (int64_t)row * M);
      cp_commit();
    }
#pragma unroll 1
    for (int top = N - 1; top >= 0; top -= U) {
      cp_wait<D - U>();
      const int n = (top + 1) < U ? (top + 1) : U;
      const int s0 = (N - 1 - top) % D;
      C f[U][1];
#pragma unroll
      for (int q = 0; q < U; q++) f[q][0] = *reinterpret_cast<const C*>(ring + (size_t)(s0 + q) * pitch);
#pragma unroll
      for (int q = 0; q < U; q++) {
        const int row = top - q - D;
        if (q < n && row >= 0 && valid) cp(ring_s + (s0 + q) * pitch, po + (int64_t)row * M);
        cp_commit();
      }
      if (valid) {
        if constexpr (REC)
          bwd_block_rec<BW, ADJ, 1, U, false>(br, 0.f, top, n, f, r1, r2);
        else
          bwd_block<BW, ADJ, C, 1, U>(cf, top, n, f, r1, r2);
#pragma unroll
        for (int q = 0; q < U; q++)
          if (q < n) po[(int64_t)(top - q) * M] = f[q][0];
      }
    }
    cp_wait<0>();
    __syncwarp();
  }
}

// ----------------------------------------------------- implicit along x

constexpr int kAdiTile = 35;  // 34 systems (32 + one neighbour each side), padded

// X-implicit half-step: each warp owns 32 rows of the grid (systems) at a
// time; the warps of a CTA share its staged coefficients and each has its
// own ring.  Chunks of R grid columns (rows of the systems) move through a
// ring of K tiles in shared memory by cp.async -- the lanes with lane % R == q
// copy row q of the chunk for the 34 systems the warp touches (its 32 plus
// one neighbour each side), 32 / R lanes sharing a row -- so K chunks are in
// flight while one is swept.  The forward values overwrite the swept tile,
// leave from it with coalesced stores and come back through the same ring for
// the backward sweep.  Warps synchronise only within themselves.
constexpr int kAdiStThreads = 128;  // largest CTA (warps per CTA: blockDim.x / 32)

template <int BW, bool ADJ, bool SMEM, typename C, int K, int R>
__global__ void __launch_bounds__(kAdiStThreads)
k_adi_st2(Coefs<C> cf_g, int N, const C* __restrict__ u, C* __restrict__ out, int64_t M, C r, int64_t ld, int L) {
  static_assert(R == 16 || R == 32, "chunk rows");
  static_assert(kStPad <= kAdiTile, "backward tiles reuse the ring");
  constexpr int U = 8;
  constexpr int kTile = R * kAdiTile;  // one ring tile (input layout)
  constexpr int kParts = 32 / R;       // lanes per chunk row
  extern __shared__ __align__(16) unsigned char smem_raw[];
  {  // row block of a partitioned launch (blockIdx.y; L = N otherwise); ld = system stride
    const int r0 = blockIdx.y * L;
    N = (N - r0) < L ? (N - r0) : L;
    cf_g = shift_coefs(cf_g, r0);
    u += r0;
    out += r0;
  }
  constexpr bool FUSE = SMEM && !ADJ && sizeof(C) == 8;
  const double2* pr = reinterpret_cast<const double2*>(smem_raw);
  C* smc = reinterpret_cast<C*>(smem_raw) + fuse_elems<C, FUSE>(N);
  const Coefs<C> cf = stage_coefs<BW, ADJ, SMEM>(cf_g, N, smc);
  if constexpr (FUSE) fuse_explicit(cf.s, reinterpret_cast<double2*>(smem_raw), N, r);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int crow = lane % R, cph = lane / R;  // chunk row and system phase of this lane's copies
  C* ringt = reinterpret_cast<C*>(smem_raw) +
             (SMEM ? align_up((fuse_elems<C, FUSE>(N) + (size_t)coef_arrays<BW>() * N) * sizeof(C), 16) / sizeof(C)
                   : 0) +
             (size_t)warp * K * kTile;
  auto cp = [&](C* dst, const C* src) {
    const uint32_t d = smem_u32(dst);
    if constexpr (sizeof(C) == 8)
      cp_async8(d, src);
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
  };
  const int nch = (N + R - 1) / R;
  for (int64_t wg = (int64_t)blockIdx.x * nwarps + warp; wg * 32 < M; wg += (int64_t)gridDim.x * nwarps) {
    const int64_t j0 = wg * 32;
    const int nsys = (int)((M - j0) < 32 ? (M - j0) : 32);
    const bool mine = lane < nsys;
    // forward: chunk c lands in tile c % K; tile column s + 1 = system j0 + s
    auto request_in = [&](int c) {
      C* t = ringt + (c % K) * kTile + crow * kAdiTile;
      const int row = c * R + crow;
      if (row < N)
        for (int s = -1 + cph; s <= nsys; s += kParts) {
          const int64_t jj = j0 + s;
          if (jj >= 0 && jj < M) cp(t + s + 1, u + jj * ld + row);
          else t[s + 1] = C(0);
        }
    };
#pragma unroll 1
    for (int c = 0; c < K; c++) {
      if (c < nch) request_in(c);
      cp_commit();
    }
    C r1[1] = {C(0)}, r2[1] = {C(0)};
#pragma unroll 1
    for (int c = 0; c < nch; c++) {
      cp_wait<K - 1>();
      __syncwarp();
      const int c0 = c * R;
      const int rows = (N - c0) < R ? (N - c0) : R;
      // the forward values overwrite the tile's own entries (each block of U
      // rows is read by every lane before any lane writes it)
      C* tin = ringt + (c % K) * kTile;
      for (int q0 = 0; q0 < rows; q0 += U) {
        const int n = (rows - q0) < U ? (rows - q0) : U;
        C f[U][1], nb[U];
        if (mine) {
#pragma unroll
          for (int q = 0; q < U; q++) {
            const C* t = tin + (q0 + q) * kAdiTile + lane;
            if constexpr (FUSE) {
              f[q][0] = t[1];
              nb[q] = t[0] + t[2];
            } else {
              f[q][0] = t[1] + r * (t[0] - C(2) * t[1] + t[2]);
            }
          }
        }
        __syncwarp();
        if (mine) {
          if constexpr (FUSE)
            adi_fwd_fused<BW, U>(cf, pr, c0 + q0, n, f, nb, r1, r2);
          else
            fwd_block<BW, ADJ, C, 1, U>(cf, c0 + q0, n, f, r1, r2);
#pragma unroll
          for (int q = 0; q < U; q++)
            if (q < n) tin[(q0 + q) * kAdiTile + lane + 1] = f[q][0];
        }
      }
      __syncwarp();
      if (crow < rows)
        for (int s = cph; s < nsys; s += kParts) out[(j0 + s) * ld + c0 + crow] = tin[crow * kAdiTile + s + 1];
      __syncwarp();
      if (c + K < nch) request_in(c + K);  // the tile is free again
      cp_commit();
    }
    cp_wait<0>();
    __syncwarp();
    // backward: chunks in decreasing order through the ring (output layout)
    auto request_back = [&](int c) {
      C* t = ringt + (c % K) * kTile + crow * kStPad;
      const int row = c * R + crow;
      if (row < N)
        for (int s = cph; s < nsys; s += kParts) cp(t + s, out + (j0 + s) * ld + row);
    };
#pragma unroll 1
    for (int q = 0; q < K; q++) {
      const int c = nch - 1 - q;
      if (c >= 0) request_back(c);
      cp_commit();
    }
    r1[0] = r2[0] = C(0);
#pragma unroll 1
    for (int c = nch - 1; c >= 0; c--) {
      cp_wait<K - 1>();
      __syncwarp();
      const int c0 = c * R;
      const int rows = (N - c0) < R ? (N - c0) : R;
      C* tw = ringt + (c % K) * kTile;
      if (mine)
        for (int top = rows - 1; top >= 0; top -= U) {
          const int n = (top + 1) < U ? (top + 1) : U;
          C f[U][1];
#pragma unroll
          for (int q = 0; q < U; q++) f[q][0] = tw[(q < n ? top - q : top) * kStPad + lane];
          bwd_block<BW, ADJ, C, 1, U>(cf, c0 + top, n, f, r1, r2);
#pragma unroll
          for (int q = 0; q < U; q++)
            if (q < n) tw[(top - q) * kStPad + lane] = f[q][0];
        }
      __syncwarp();
      if (crow < rows)
        for (int s = cph; s < nsys; s += kParts) out[(j0 + s) * ld + c0 + crow] = tw[crow * kStPad + s];
      __syncwarp();
      if (c - K >= 0) request_back(c - K);
      cp_commit();
    }
    cp_wait<0>();
    __syncwarp();
  }
}

template <int BW, bool ADJ, typename C>
static cudaError_t launch_adi(const SweepPlan& p, int N, const C* u, C* out, int64_t M, C r, int axis, int L, int P,
                              cudaStream_t st) {
  const C* base;
  if constexpr (sizeof(C) == 8)
    base = reinterpret_cast<const C*>(p.c64);
  else
    base = reinterpret_cast<const C*>(p.c32);
  const Coefs<C> cf = coefs_of<C>(base, N);
  // Ring depth: with one thread per grid line (P = 1) there is less than one
  // warp per SM and the depth must come from each lane (64 rows, 8 chunks);
  // a partitioned launch has P times the threads, and shallow rings leave
  // room for more resident CTAs.
  // FP32 along y stages two 16-byte records per row (8 values) instead of
  // 1 + 2 BW arrays (k_adi_il2; 0.115 -> 0.108 ms per 4096^2 half-step).  The
  // one-warp CTAs along x keep the arrays: records there cost resident CTAs
  // (0.113 -> 0.121 ms).
  // FP64 primal plans stage the (e0, e1) pairs beside the arrays (fuse_explicit).
  constexpr int kFuseExtra = (sizeof(C) == 8 && !ADJ) ? 2 : 0;
  constexpr int kRecExtra = sizeof(C) == 4 ? 8 - coef_arrays<BW>() : kFuseExtra;
  if (axis == 1) {
    auto go = [&](auto dtag) -> cudaError_t {
      constexpr int D = decltype(dtag)::value;
      const int64_t threads = ((M + 31) / 32) * 32;
      const LaunchShape sh =
          sweep_shape(BW, L, threads * P, sizeof(C), sizeof(C), 1, (size_t)D * 2 * sizeof(C), 0, 0, kRecExtra, P > 1);
      const size_t bytes = sh.smem + (size_t)sh.threads * D * 2 * sizeof(C);
      auto k = sh.smem_coefs ? k_adi_il2<BW, ADJ, true, C, D> : k_adi_il2<BW, ADJ, false, C, D>;
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
      k<<<dim3((sh.grid + P - 1) / P, P), sh.threads, bytes, st>>>(cf, N, u, out, M, r, L);
      return cudaGetLastError();
    };
    return P > 1 ? go(std::integral_constant<int, 16>{}) : go(std::integral_constant<int, 64>{});
  }
  // Warps per CTA: one for a whole-line launch (its ring alone is 8 tiles);
  // several for a partitioned launch, sharing the staged coefficients, so
  // that the 2048 warps of a 4096^2 half-step (16 blocks) fit in one round:
  // FP64 two (seven CTAs, 14 warps per SM; 0.296 ms with one warp, 0.238 with
  // two, 0.250 with four), FP32 four (0.094, 0.092, 0.090 ms).
  // BS_OPT_CTA_THREADS = 32, 64 or 128 (and above) forces one, two or four.
  const int64_t forced = option(BS_OPT_CTA_THREADS);
  const int tpb = forced > 0 ? (forced >= 128 ? 128 : (forced >= 64 ? 64 : 32))
                             : (P > 1 ? (sizeof(C) == 8 ? 64 : 128) : 32);
  auto go = [&](auto ktag, auto rtag) -> cudaError_t {
    constexpr int K = decltype(ktag)::value;
    constexpr int R = decltype(rtag)::value;
    const size_t tiles = (size_t)K * R * kAdiTile * sizeof(C);  // per warp
    const int64_t threads = ((M + 31) / 32) * 32;
    const LaunchShape sh = sweep_shape(BW, L, threads * P, sizeof(C), sizeof(C), 1, tiles / 32, 0, tpb, kFuseExtra);
    const size_t bytes = sh.smem + tiles * (tpb / 32);
    auto k = sh.smem_coefs ? k_adi_st2<BW, ADJ, true, C, K, R> : k_adi_st2<BW, ADJ, false, C, K, R>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k<<<dim3((sh.grid + P - 1) / P, P), tpb, bytes, st>>>(cf, N, u, out, M, r, (int64_t)N, L);
    return cudaGetLastError();
  };
  if (P == 1) return go(std::integral_constant<int, 8>{}, std::integral_constant<int, 32>{});
  // partitioned: two chunks in flight.  FP64 takes 16-row chunks (half the
  // shared memory per warp, so about twice the resident warps for the FP64
  // pipe: 0.313 against 0.342 ms per 4096^2 half-step); FP32, bound by
  // latency, keeps 32-row chunks (0.113 against 0.129 ms with 16 rows)
  if constexpr (sizeof(C) == 8)
    return go(std::integral_constant<int, 2>{}, std::integral_constant<int, 16>{});
  else
    return go(std::integral_constant<int, 2>{}, std::integral_constant<int, 32>{});
}

bool use_partition(bs_handle h, int64_t M);
bs_status part_correct(const PartPlan& pp, int N, void* X, bs_dtype t, bs_layout layout, int64_t M,
                       cudaStream_t st);

template <typename C>
static bs_status dispatch_adi(bs_handle h, int N, const C* u, C* out, int64_t M, C r, int axis, bool adj,
                              cudaStream_t st) {
  cudaError_t e;
  if (use_partition(h, M)) {
    // row-partitioned: the primal-form plan of the block-diagonal part of
    // A (or A^T), then the block-edge correction on `out`
    const PartPlan& pp = h->part[adj ? 1 : 0];
    e = h->width == 3 ? launch_adi<1, false, C>(pp.blk, N, u, out, M, r, axis, pp.L, pp.P, st)
                      : launch_adi<2, false, C>(pp.blk, N, u, out, M, r, axis, pp.L, pp.P, st);
    if (e != cudaSuccess) return cuda_error(e, "bs_adi_halfstep launch");
    return part_correct(pp, N, out, sizeof(C) == 8 ? BS_F64 : BS_F32, axis == 1 ? BS_INTERLEAVED : BS_STRIDED, M,
                        st);
  }
  const SweepPlan& p = h->plan[adj ? 1 : 0];
  if (h->width == 3)
    e = adj ? launch_adi<1, true, C>(p, N, u, out, M, r, axis, N, 1, st)
            : launch_adi<1, false, C>(p, N, u, out, M, r, axis, N, 1, st);
  else
    e = adj ? launch_adi<2, true, C>(p, N, u, out, M, r, axis, N, 1, st)
            : launch_adi<2, false, C>(p, N, u, out, M, r, axis, N, 1, st);
  if (e != cudaSuccess) return cuda_error(e, "bs_adi_halfstep launch");
  return BS_OK;
}

}  // namespace bs

extern "C" bs_status bs_adi_halfstep(bs_handle h, const void* U, void* out, bs_dtype dtype, int64_t ny, int64_t nx,
                                     double r, int implicit_axis, int adjoint, bs_stream stream) {
  using namespace bs;
  if (!valid_handle(h)) return set_error(BS_EINVAL, "bs_adi_halfstep: unknown handle");
  if (h->periodic) return set_error(BS_EUNSUPPORTED, "bs_adi_halfstep: not available for a periodic handle");
  if (!U || !out) return set_error(BS_EINVAL, "bs_adi_halfstep: null data pointer");
  if (ny < 1 || nx < 1) return set_error(BS_EINVAL, "bs_adi_halfstep: empty grid");
  if (implicit_axis != 0 && implicit_axis != 1) return set_error(BS_EINVAL, "bs_adi_halfstep: axis must be 0 or 1");
  if (adjoint != 0 && adjoint != 1) return set_error(BS_EINVAL, "bs_adi_halfstep: adjoint must be 0 or 1");
  const int64_t N = implicit_axis == 0 ? nx : ny;
  const int64_t M = implicit_axis == 0 ? ny : nx;
  if (N != h->N)
    return set_error(BS_EINVAL, "bs_adi_halfstep: the handle's N must equal the grid length along the implicit axis");
  if (dtype != BS_F64 && dtype != BS_F32) return set_error(BS_EINVAL, "bs_adi_halfstep: dtype must be F64 or F32");
  const size_t es = dtype == BS_F64 ? 8 : 4;
  const char* a = static_cast<const char*>(U);
  const char* b = static_cast<const char*>(out);
  const size_t n = (size_t)ny * (size_t)nx * es;
  if (a < b + n && b < a + n) return set_error(BS_EINVAL, "bs_adi_halfstep: U and out overlap");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) return set_error(BS_EINVAL, "bs_adi_halfstep: handle belongs to another device");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (dtype == BS_F64)
    return dispatch_adi<double>(h, (int)N, (const double*)U, (double*)out, M, r, implicit_axis, adjoint != 0, st);
  return dispatch_adi<float>(h, (int)N, (const float*)U, (float*)out, M, (float)r, implicit_axis, adjoint != 0, st);
}
