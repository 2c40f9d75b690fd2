// Grouped persistent solve: one launch runs every request of a serving batch.
// Each warp takes 32-system tiles from the work list (static stride over all
// warps of the grid) and runs, lane by lane, exactly the per-system arithmetic
// of the standalone solves (the same sweep and refinement helpers), so a
// system's result does not depend on what else is in the batch.  The work
// list (count included) is read from device memory, so one captured CUDA
// graph (work-list copy + this launch) serves every batch.
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

template <int BW>
__device__ void lane_solve_refine(const GReq& q, int64_t j) {
  constexpr int W = 2 * BW + 1;
  const RefineCoefs<BW> cf = make_refine_coefs<BW>(q.c32, q.ul32, q.bhi, q.blo, q.N);
  const int N = q.N;
  const int64_t M = q.M;
  const float* pb = static_cast<const float*>(q.B) + j;
  double* px = q.X + j;
  float2* ps = reinterpret_cast<float2*>(q.X) + j;
  {  // pass 1
    float w1 = 0.f, w2 = 0.f;
#pragma unroll 1
    for (int i0 = 0; i0 < N; i0 += kGroupU) {
      float b[kGroupU];
#pragma unroll
      for (int u = 0; u < kGroupU; u++)
        if (i0 + u < N) b[u] = pb[(int64_t)(i0 + u) * M];
#pragma unroll
      for (int u = 0; u < kGroupU; u++)
        if (i0 + u < N) ps[(int64_t)(i0 + u) * M] = make_float2(refine_fwd<BW>(cf, i0 + u, b[u], w1, w2), b[u]);
    }
  }
  {  // pass 2
    float xw[W], bw[BW + 1];
#pragma unroll
    for (int k = 0; k < W; k++) xw[k] = 0.f;
#pragma unroll
    for (int k = 0; k <= BW; k++) bw[k] = 0.f;
    float z1 = 0.f, z2 = 0.f;
#pragma unroll 1
    for (int i = N - 1; i >= -BW; i--) {
      float x0 = 0.f, b = 0.f;
      if (i >= 0) {
        const float2 wb = ps[(int64_t)i * M];
        x0 = refine_bwd<BW>(cf, i, wb.x, xw);
        b = wb.y;
      }
#pragma unroll
      for (int k = W - 1; k > 0; k--) xw[k] = xw[k - 1];
      xw[0] = x0;
#pragma unroll
      for (int k = BW; k > 0; k--) bw[k] = bw[k - 1];
      bw[0] = b;
      const int qrow = i + BW;
      if (qrow < N) {
        const float z = refine_resid_z<BW>(cf, qrow, bw[BW], xw, z1, z2);
        ps[(int64_t)qrow * M] = make_float2(xw[BW], z);
      }
    }
  }
  {  // pass 3
    float d1 = 0.f, d2 = 0.f;
#pragma unroll 1
    for (int i0 = 0; i0 < N; i0 += kGroupU) {
      float2 xz[kGroupU];
#pragma unroll
      for (int u = 0; u < kGroupU; u++)
        if (i0 + u < N) xz[u] = ps[(int64_t)(i0 + u) * M];
#pragma unroll
      for (int u = 0; u < kGroupU; u++)
        if (i0 + u < N) px[(int64_t)(i0 + u) * M] = refine_out<BW>(cf, i0 + u, xz[u].x, xz[u].y, d1, d2);
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
    if (q.mode == SERVE_F64) {
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
