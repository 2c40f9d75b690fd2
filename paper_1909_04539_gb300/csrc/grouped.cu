// Grouped persistent solve: one launch runs every request of a serving batch.
// Each warp takes 32-system tiles from the work list (static stride over all
// warps of the grid) and runs, lane by lane, exactly the per-system arithmetic
// of the standalone solves (the same sweep, pair-arithmetic and refinement
// helpers), so a system's result does not depend on what else is in the
// batch.  The work list (count included) is read from device memory, so one
// captured CUDA graph (work-list copy + this launch) serves every batch.
#include "df_sweep.cuh"
#include "refine_math.cuh"
#include "serve.h"

namespace bs {

constexpr int kGroupThreads = 128;
constexpr int kGroupU = 8;

template <int BW>
__device__ void lane_solve_f64(const GReq& q, int64_t j) {
  const Coefs<double> cf = coefs_of<double>(q.c64, q.N);
  double* x = static_cast<double*>(q.B) + j;
  const int N = q.N;
  const int64_t M = q.M;
  double r1[1] = {0.0}, r2[1] = {0.0};
#pragma unroll 1
  for (int i0 = 0; i0 < N; i0 += kGroupU) {
    double f[kGroupU][1];
#pragma unroll
    for (int u = 0; u < kGroupU; u++)
      if (i0 + u < N) f[u][0] = x[(int64_t)(i0 + u) * M];
#pragma unroll
    for (int u = 0; u < kGroupU; u++)
      if (i0 + u < N) {
        fwd_step<BW, false, double, 1>(cf, i0 + u, f[u], r1, r2);
        x[(int64_t)(i0 + u) * M] = f[u][0];
      }
  }
  r1[0] = r2[0] = 0.0;
#pragma unroll 1
  for (int top = N - 1; top >= 0; top -= kGroupU) {
    double f[kGroupU][1];
#pragma unroll
    for (int u = 0; u < kGroupU; u++)
      if (top - u >= 0) f[u][0] = x[(int64_t)(top - u) * M];
#pragma unroll
    for (int u = 0; u < kGroupU; u++)
      if (top - u >= 0) {
        bwd_step<BW, false, double, 1>(cf, top - u, f[u], r1, r2);
        x[(int64_t)(top - u) * M] = f[u][0];
      }
  }
}

// FP64 data in FP32 pairs: the row groups of the two-sweep kernel
// (df_sweep.cuh), the forward values kept in place in B
template <int BW>
__device__ void lane_solve_pairs(const GReq& q, int64_t j) {
  constexpr int U = 4;  // the block of the standalone kernel: the same switch rows
  const DfRecs rc = df_recs_of(q.dfrec, q.N);
  const Coefs<double> c64 = coefs_of<double>(q.c64, q.N);
  double* x = static_cast<double*>(q.B) + j;
  const int N = q.N;
  const int64_t M = q.M;
  DfState<1> st;
  st.reset_values();
  st.f64 = false;
  st.rsw = N;
#pragma unroll 1
  for (int i0 = 0; i0 < N; i0 += U) {
    const int n = (N - i0) < U ? (N - i0) : U;
    double f[U][1];
    uint2 w[U][1];
#pragma unroll
    for (int u = 0; u < U; u++) f[u][0] = (u < n) ? x[(int64_t)(i0 + u) * M] : 0.0;
    df_fwd_group<BW, false, 1, U, false>(rc, c64, i0, n, f, w, st);
#pragma unroll
    for (int u = 0; u < U; u++)
      if (u < n) *reinterpret_cast<uint2*>(x + (int64_t)(i0 + u) * M) = w[u][0];
  }
  st.reset_values();
#pragma unroll 1
  for (int top = N - 1; top >= 0; top -= U) {
    const int n = (top + 1) < U ? (top + 1) : U;
    uint2 w[U][1];
    double xo[U][1];
#pragma unroll
    for (int u = 0; u < U; u++)
      w[u][0] = (u < n) ? *reinterpret_cast<const uint2*>(x + (int64_t)(top - u) * M) : make_uint2(0u, 0u);
    df_bwd_group<BW, false, 1, U, false>(rc, c64, top, n, w, xo, st);
#pragma unroll
    for (int u = 0; u < U; u++)
      if (u < n) x[(int64_t)(top - u) * M] = xo[u][0];
  }
}

template <int BW>
__device__ void lane_solve_refine(const GReq& q, int64_t j) {
  constexpr int U = 4;  // the block of the standalone kernel: same arithmetic
  const FRefineCoefs<BW> cf = make_frefine_coefs<BW>(q.lu_hi, q.lu_lo, q.N);
  const int N = q.N;
  const int64_t M = q.M;
  const float* pb = static_cast<const float*>(q.B) + j;
  double* px = q.X + j;
  float2* ps = reinterpret_cast<float2*>(q.X) + j;
  {
    float w1 = 0.f, w2 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll 1
    for (int i0 = 0; i0 < N; i0 += U) {
      const int n = (N - i0) < U ? (N - i0) : U;
      float b[U], w[U], d[U];
#pragma unroll
      for (int u = 0; u < U; u++) b[u] = (u < n) ? pb[(int64_t)(i0 + u) * M] : 0.f;
      frefine_pass1<BW, U>(cf, i0, n, b, w, d, w1, w2, d1, d2);
#pragma unroll
      for (int u = 0; u < U; u++)
        if (u < n) ps[(int64_t)(i0 + u) * M] = make_float2(w[u], d[u]);
    }
  }
  {
    float x1 = 0.f, x2 = 0.f, e1 = 0.f, e2 = 0.f;
#pragma unroll 1
    for (int top = N - 1; top >= 0; top -= U) {
      const int n = (top + 1) < U ? (top + 1) : U;
      float w[U], dl[U];
      double xo[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const float2 v = (u < n) ? ps[(int64_t)(top - u) * M] : make_float2(0.f, 0.f);
        w[u] = v.x;
        dl[u] = v.y;
      }
      frefine_pass2<BW, U>(cf, top, n, w, dl, xo, x1, x2, e1, e2);
#pragma unroll
      for (int u = 0; u < U; u++)
        if (u < n) px[(int64_t)(top - u) * M] = xo[u];
    }
  }
}

__global__ void __launch_bounds__(kGroupThreads) k_grouped(const unsigned char* __restrict__ work) {
  const GHeader* hdr = reinterpret_cast<const GHeader*>(work);
  const GReq* reqs = reinterpret_cast<const GReq*>(work + kGroupReqOff);
  const GTile* tiles = reinterpret_cast<const GTile*>(work + kGroupTileOff);
  const int n_tiles = hdr->n_tiles;
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x / 32);
  for (int t = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); t < n_tiles; t += warps) {
    const GTile tile = tiles[t];
    const GReq q = reqs[tile.req];
    const int64_t j = (int64_t)tile.j0 + lane;
    if (j >= q.M) continue;
    if (q.mode == SERVE_F64 && q.pairs) {
      if (q.width == 3)
        lane_solve_pairs<1>(q, j);
      else
        lane_solve_pairs<2>(q, j);
    } else if (q.mode == SERVE_F64) {
      if (q.width == 3)
        lane_solve_f64<1>(q, j);
      else
        lane_solve_f64<2>(q, j);
    } else {
      if (q.width == 3)
        lane_solve_refine<1>(q, j);
      else
        lane_solve_refine<2>(q, j);
    }
  }
}

int grouped_grid() { return device_info().sms * 4; }

cudaError_t launch_grouped(const unsigned char* d_work, int grid, cudaStream_t st) {
  k_grouped<<<grid, kGroupThreads, 0, st>>>(d_work);
  return cudaGetLastError();
}

}  // namespace bs
