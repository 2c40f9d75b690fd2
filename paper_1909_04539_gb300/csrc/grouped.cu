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
constexpr int kGroupD = 16;  // rows in flight per lane (the standalone kernels' ring depth)

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

__global__ void __launch_bounds__(kGroupThreads) k_grouped(const unsigned char* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* ring = smem_raw + (size_t)threadIdx.x * 8;  // the lane's ring of kGroupD 8-byte slots
  const uint32_t ring_s = smem_u32(ring);
  const uint32_t pitch = blockDim.x * 8;
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
      // the standalone pair solve's lane body, records read from global memory
      const DfRecs rc = df_recs_of(q.dfrec, q.N);
      const Coefs<double> c64 = coefs_of<double>(q.c64, q.N);
      double* x = static_cast<double*>(q.B) + j;
      if (q.width == 3)
        df_sweep_systems<1, false, 1, kGroupD>(rc, c64, q.N, x, q.M, ring, ring_s, pitch);
      else
        df_sweep_systems<2, false, 1, kGroupD>(rc, c64, q.N, x, q.M, ring, ring_s, pitch);
    } else if (q.mode == SERVE_F64) {
      if (q.width == 3)
        lane_solve_f64<1>(q, j);
      else
        lane_solve_f64<2>(q, j);
    } else {
      // the standalone mixed-precision kernel's lane body, coefficients read
      // from global memory
      const float* B = static_cast<const float*>(q.B);
      if (q.width == 3)
        refine_factor_system<1, kGroupD>(make_frefine_coefs<1>(q.lu_hi, q.lu_lo, q.N), q.N, B, q.X, q.M, j, ring,
                                         ring_s, pitch);
      else
        refine_factor_system<2, kGroupD>(make_frefine_coefs<2>(q.lu_hi, q.lu_lo, q.N), q.N, B, q.X, q.M, j, ring,
                                         ring_s, pitch);
    }
  }
}

// One wave: the CTAs that fit on the device at once (registers and the
// rings' shared memory decide how many per SM).
int grouped_grid() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_grouped, kGroupThreads,
                                                    (size_t)kGroupThreads * kGroupD * 8) != cudaSuccess ||
      n < 1)
    n = 1;
  return device_info().sms * n;
}

cudaError_t launch_grouped(const unsigned char* d_work, int grid, cudaStream_t st) {
  k_grouped<<<grid, kGroupThreads, (size_t)kGroupThreads * kGroupD * 8, st>>>(d_work);
  return cudaGetLastError();
}

}  // namespace bs
