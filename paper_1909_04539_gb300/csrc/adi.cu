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

#include "df_math.cuh"
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

// FP64 y-implicit half-step in FP32 pairs (the arithmetic of the FP64 solves,
// df_math.cuh): the FP64 kernel above is bound by the FP64 pipe (5 FP64
// instructions per unknown).  Same ring and shuffles; each value is split
// into a pair as it leaves the ring and its pair goes to the neighbouring
// lanes; the fused stencil f = e0 c + e1 (left + right) is formed with pair
// products and TwoSums, the forward and backward recurrences with
// df::rec_step, the forward values go to `out` as 8-byte pairs and the
// result as FP64 (exactly widened parts, one FP64 addition).  Coefficients
// per row, staged once per CTA as FP32 pairs (fl32(c), fl32(c - fl32(c))):
// (e0, e1) and (l1, l2) forward, (u1, u2) backward.  Range: the plan's sweep
// gains are bounded (SweepPlan::df_ok), |e0|, |e1| < 2^8 (else the CTA runs
// FP64), and inputs zero or in [2^-72, 2^91), so that every intermediate stays
// inside FP32; a warp that meets any other input redoes its 32 columns with
// FP64 arithmetic (u is not overwritten), so every result depends only on
// the data.  (Forming the stencil in FP64 instead -- 3 FP64 instructions
// and one split per unknown -- made the FP64 pipe the bound again: 198
// against 172 us.)
constexpr int kAdiDfThreadsMax = 512;

__device__ __forceinline__ float2 adi_split_coef(double c) {
  const float h = __double2float_rn(c);
  return make_float2(h, __double2float_rn(c - (double)h));
}
// zero or 2^-100 <= |c| < 2^8
__device__ __forceinline__ bool adi_coef_ok(double c) {
  const uint32_t hw = (uint32_t)__double2hiint(c) & 0x7fffffffu;
  return hw - ((1023u - 100u) << 20) < (108u << 20) || c == 0.0;
}
// the pair of an input value, or bad: zero or 2^-72 <= |v| < 2^91
__device__ __forceinline__ df::Pair adi_pair(double v, bool& bad) {
  df::Pair y;
  const uint32_t hw = (uint32_t)__double2hiint(v) & 0x7fffffffu;
  if (!df::split_fast(v, y)) y = df::Pair{0.f, 0.f};
  bad |= !(hw - (951u << 20) < (163u << 20) || (hw | (uint32_t)__double2loint(v)) == 0u);
  return y;
}
// c * v, unnormalised: TwoProduct of the high parts plus both cross terms
__device__ __forceinline__ df::Pair adi_prod(float ch, float cl, df::Pair v) {
  const float p = df::mul(ch, v.h);
  float e = df::fma_(ch, v.h, -p);
  e = df::fma_(ch, v.l, e);
  e = df::fma_(cl, v.h, e);
  return df::Pair{p, e};
}
__device__ __forceinline__ df::Pair adi_add(df::Pair a, df::Pair b) {
  float s, t;
  df::two_sum(a.h, b.h, s, t);
  return df::Pair{s, df::add(df::add(a.l, b.l), t)};
}

template <int BW, int D>
__global__ void __launch_bounds__(kAdiDfThreadsMax)
k_adi_il2_df(Coefs<double> cf_g, int N, const double* __restrict__ u, double* __restrict__ out, int64_t M,
             double r, int L) {
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
  float4* ra = reinterpret_cast<float4*>(smem_raw);  // (e0, e1)
  float4* rb = ra + N;                                // (l1, l2)
  float4* rc = rb + N;                                // (u1, u2)
  bool cbad = false;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double s = cf_g.s[i];
    const double e0 = s * (1.0 - 2.0 * r), e1 = s * r;
    const double l1 = cf_g.l1[i], l2 = BW == 2 ? cf_g.l2[i] : 0.0;
    const double u1 = cf_g.u1[i], u2 = BW == 2 ? cf_g.u2[i] : 0.0;
    cbad |= !(adi_coef_ok(e0) && adi_coef_ok(e1));
    const float2 a = adi_split_coef(e0), b = adi_split_coef(e1), c1 = adi_split_coef(l1), c2 = adi_split_coef(l2),
                 d1 = adi_split_coef(u1), d2 = adi_split_coef(u2);
    ra[i] = make_float4(a.x, a.y, b.x, b.y);
    rb[i] = make_float4(c1.x, c1.y, c2.x, c2.y);
    rc[i] = make_float4(d1.x, d1.y, d2.x, d2.y);
  }
  const bool cta_f64 = __syncthreads_or(cbad) != 0;
  const int lane = threadIdx.x & 31;
  constexpr int kSlot = 16;  // [own value | outer neighbour], 8 bytes each
  unsigned char* ring = smem_raw + (size_t)N * 3 * sizeof(float4) + (size_t)threadIdx.x * kSlot;
  const uint32_t ring_s = smem_u32(ring);
  const uint32_t pitch = blockDim.x * kSlot;
  const int64_t nwarps_total = (int64_t)gridDim.x * (blockDim.x / 32);
  const int64_t ngroups = (M + 31) / 32;
  for (int64_t wg = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); wg < ngroups; wg += nwarps_total) {
    const int64_t j = wg * 32 + lane;
    const bool valid = j < M;
    const int64_t jn = lane == 0 ? j - 1 : (lane == 31 ? j + 1 : -1);
    const bool has_n = (lane == 0 || lane == 31) && jn >= 0 && jn < M;
    const double* pu = u + (valid ? j : 0);
    const double* pn = u + (has_n ? jn : 0);
    double* po = out + (valid ? j : 0);
    auto request = [&](int slot, int row) {
      if (valid) cp_async8(ring_s + slot * pitch, pu + (int64_t)row * M);
      if (has_n) cp_async8(ring_s + slot * pitch + 8, pn + (int64_t)row * M);
    };
    // one pass over the group's columns: PAIRS, or FP64 (coefficients from
    // global memory, the row scale folded as in fuse_explicit)
    auto pass = [&](auto pairs_tag) -> bool {
      constexpr bool PAIRS = decltype(pairs_tag)::value;
      bool bad = false;
#pragma unroll 1
      for (int q = 0; q < D; q++) {
        if (q < N) request(q, q);
        cp_commit();
      }
      df::Pair w1{0.f, 0.f}, w2{0.f, 0.f};
      double d1 = 0.0, d2 = 0.0;
#pragma unroll 1
      for (int i0 = 0; i0 < N; i0 += U) {
        cp_wait<D - U>();
        __syncwarp();
        const int n = (N - i0) < U ? (N - i0) : U;
        const int s0 = i0 % D;
        double c[U], outer[U];
#pragma unroll
        for (int q = 0; q < U; q++) {
          const double* sl = reinterpret_cast<const double*>(ring + (size_t)(s0 + q) * pitch);
          c[q] = valid ? sl[0] : 0.0;
          outer[q] = has_n ? sl[1] : 0.0;
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < U; q++) {
          if (q < n && i0 + q + D < N) request(s0 + q, i0 + q + D);
          cp_commit();
        }
#pragma unroll
        for (int q = 0; q < U; q++) {
          const int i = i0 + q;
          if constexpr (PAIRS) {
            const df::Pair cp = adi_pair(c[q], bad);
            const df::Pair op = adi_pair(outer[q], bad);
            df::Pair lf{__shfl_up_sync(0xffffffffu, cp.h, 1), __shfl_up_sync(0xffffffffu, cp.l, 1)};
            df::Pair rt{__shfl_down_sync(0xffffffffu, cp.h, 1), __shfl_down_sync(0xffffffffu, cp.l, 1)};
            if (lane == 0) lf = op;
            if (lane == 31) rt = op;
            if (q < n && valid) {
              const float4 ea = ra[i], lb = rb[i];
              const df::Pair nb = adi_add(lf, rt);
              const df::Pair f = adi_add(adi_prod(ea.x, ea.y, cp), adi_prod(ea.z, ea.w, nb));
              const df::Pair w = df::rec_step<false, BW>(df::Pair{1.f, 0.f}, f, df::Pair{lb.x, lb.y}, w1,
                                                         df::Pair{lb.z, lb.w}, w2);
              w2 = w1;
              w1 = w;
              *reinterpret_cast<uint2*>(po + (int64_t)i * M) = make_uint2(__float_as_uint(w.h), __float_as_uint(w.l));
            }
          } else {
            double lf = __shfl_up_sync(0xffffffffu, c[q], 1);
            double rt = __shfl_down_sync(0xffffffffu, c[q], 1);
            if (lane == 0) lf = outer[q];
            if (lane == 31) rt = outer[q];
            if (q < n && valid) {
              const double s = cf_g.s[i];
              double w = fma(s * r, lf + rt, s * (1.0 - 2.0 * r) * c[q]);
              if (BW == 2) w = fma(-cf_g.l2[i], d2, w);
              w = fma(-cf_g.l1[i], d1, w);
              d2 = d1;
              d1 = w;
              po[(int64_t)i * M] = w;
            }
          }
        }
      }
      cp_wait<0>();
      __syncwarp();
      // backward: the forward values come back through the ring
#pragma unroll 1
      for (int q = 0; q < D; q++) {
        const int row = N - 1 - q;
        if (row >= 0 && valid) cp_async8(ring_s + q * pitch, po + (int64_t)row * M);
        cp_commit();
      }
      df::Pair x1{0.f, 0.f}, x2{0.f, 0.f};
      double y1 = 0.0, y2 = 0.0;
#pragma unroll 1
      for (int top = N - 1; top >= 0; top -= U) {
        cp_wait<D - U>();
        const int n = (top + 1) < U ? (top + 1) : U;
        const int s0 = (N - 1 - top) % D;
        uint2 wv[U];
#pragma unroll
        for (int q = 0; q < U; q++) wv[q] = *reinterpret_cast<const uint2*>(ring + (size_t)(s0 + q) * pitch);
#pragma unroll
        for (int q = 0; q < U; q++) {
          const int row = top - q - D;
          if (q < n && row >= 0 && valid) cp_async8(ring_s + (s0 + q) * pitch, po + (int64_t)row * M);
          cp_commit();
        }
        if (valid) {
#pragma unroll
          for (int q = 0; q < U; q++) {
            if (q >= n) break;
            const int i = top - q;
            if constexpr (PAIRS) {
              const float4 cu = rc[i];
              const df::Pair w{__uint_as_float(wv[q].x), __uint_as_float(wv[q].y)};
              const df::Pair x = df::rec_step<false, BW>(df::Pair{1.f, 0.f}, w, df::Pair{cu.x, cu.y}, x1,
                                                         df::Pair{cu.z, cu.w}, x2);
              x2 = x1;
              x1 = x;
              po[(int64_t)i * M] = df::combine_ok(x.h) ? df::combine_fast(x.h, x.l) : df::combine(x.h, x.l);
            } else {
              double x = __hiloint2double((int)wv[q].y, (int)wv[q].x);
              if (BW == 2) x = fma(-cf_g.u2[i], y2, x);
              x = fma(-cf_g.u1[i], y1, x);
              y2 = y1;
              y1 = x;
              po[(int64_t)i * M] = x;
            }
          }
        }
      }
      cp_wait<0>();
      __syncwarp();
      return bad;
    };
    if (cta_f64 || __any_sync(0xffffffffu, pass(std::true_type{}))) pass(std::false_type{});
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
    if constexpr (sizeof(C) == 8 && !ADJ) {
      // FP64 in FP32 pairs where the plan admits them and the records fit
      constexpr int D = 16;
      const size_t rec = (size_t)L * 3 * sizeof(float4);
      if (p.df_ok && option(BS_OPT_F64_PAIRS) != 1 && rec + 64 * D * 16 + 1024 <= (size_t)device_info().smem_optin) {
        auto k = k_adi_il2_df<BW, D>;
        const int64_t threads = ((M + 31) / 32) * 32;
        const StagedShape sh = staged_shape(threads * P, rec, (size_t)D * 16, kernel_regs((const void*)k),
                                            kAdiDfThreadsMax, true, 128);
        if (sh.threads > 0 && sh.staged) {
          const size_t bytes = rec + (size_t)sh.threads * D * 16;
          cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
          if (e != cudaSuccess) return e;
          k<<<dim3((sh.grid + P - 1) / P, P), sh.threads, bytes, st>>>(cf, N, u, out, M, r, L);
          return cudaGetLastError();
        }
      }
    }
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
