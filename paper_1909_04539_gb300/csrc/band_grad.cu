// Band-gradient reduction over the batch.
//
// For a scalar loss L with dL/dX given, X = A^{-1} B and GB = A^{-T} dL/dX,
// dL/dA = -GB X^T; the entries on the bands are
//   dbands[k*N + i] = -sum_j GB[i, j] * X[i + k - h, j],   h = width / 2.
// Each CTA owns kGradRows consecutive rows and reduces them over all M
// systems: threads stride over the systems accumulating in FP64, then a
// fixed-order warp-shuffle and shared-memory tree combines the threads.  The
// grid depends on N only, so the result is bitwise reproducible.
#include "sweep_kernels.cuh"

namespace bs {

constexpr int kGradThreads = 256;
constexpr int kGradRows = 4;

template <typename T, int W>
__global__ void __launch_bounds__(kGradThreads)
k_band_grad(int N, int64_t M, const T* __restrict__ GB, const T* __restrict__ X, int64_t rs, int64_t ss,
            double* __restrict__ dbands) {
  constexpr int H = W / 2;
  constexpr int NX = kGradRows + 2 * H;
  __shared__ double red[kGradThreads / 32][kGradRows * W];
  const int i0 = blockIdx.x * kGradRows;
  double acc[kGradRows][W];
#pragma unroll
  for (int r = 0; r < kGradRows; r++)
#pragma unroll
    for (int k = 0; k < W; k++) acc[r][k] = 0.0;

  for (int64_t j = threadIdx.x; j < M; j += kGradThreads) {
    double x[NX], g[kGradRows];
#pragma unroll
    for (int q = 0; q < NX; q++) {
      const int row = i0 - H + q;
      x[q] = (row >= 0 && row < N) ? (double)X[row * rs + j * ss] : 0.0;
    }
#pragma unroll
    for (int r = 0; r < kGradRows; r++) {
      const int row = i0 + r;
      g[r] = (row < N) ? (double)GB[row * rs + j * ss] : 0.0;
    }
#pragma unroll
    for (int r = 0; r < kGradRows; r++)
#pragma unroll
      for (int k = 0; k < W; k++) acc[r][k] = fma(g[r], x[r + k], acc[r][k]);
  }

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < kGradRows; r++)
#pragma unroll
    for (int k = 0; k < W; k++) {
      double v = acc[r][k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][r * W + k] = v;
    }
  __syncthreads();
  if (threadIdx.x < kGradRows * W) {
    const int r = threadIdx.x / W, k = threadIdx.x % W;
    double s = 0.0;
    for (int w = 0; w < kGradThreads / 32; w++) s += red[w][threadIdx.x];
    const int row = i0 + r, col = row + k - H;
    if (row < N) dbands[(int64_t)k * N + row] = (col >= 0 && col < N) ? -s : 0.0;
  }
}

bs_status launch_band_grad(bs_handle h, const void* GB, const void* X, bs_dtype t, bs_layout layout, int64_t M,
                           double* dbands, cudaStream_t st) {
  const int N = (int)h->N;
  const int64_t rs = layout == BS_INTERLEAVED ? M : 1;
  const int64_t ss = layout == BS_INTERLEAVED ? 1 : N;
  const int grid = (N + kGradRows - 1) / kGradRows;
  if (t == BS_F64) {
    if (h->width == 3)
      k_band_grad<double, 3><<<grid, kGradThreads, 0, st>>>(N, M, (const double*)GB, (const double*)X, rs, ss, dbands);
    else
      k_band_grad<double, 5><<<grid, kGradThreads, 0, st>>>(N, M, (const double*)GB, (const double*)X, rs, ss, dbands);
  } else {
    if (h->width == 3)
      k_band_grad<float, 3><<<grid, kGradThreads, 0, st>>>(N, M, (const float*)GB, (const float*)X, rs, ss, dbands);
    else
      k_band_grad<float, 5><<<grid, kGradThreads, 0, st>>>(N, M, (const float*)GB, (const float*)X, rs, ss, dbands);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "band gradient launch");
  return BS_OK;
}

}  // namespace bs
