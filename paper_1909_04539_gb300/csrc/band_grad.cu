// Band-gradient reduction over the batch.
//
// For a scalar loss L with dL/dX given, X = A^{-1} B and GB = A^{-T} dL/dX,
// dL/dA = -GB X^T; the entries on the bands are
//   dbands[k*N + i] = -sum_j GB[i, j] * X[i + k - h, j],   h = width / 2.
// Two levels, fixed order, no atomics:
//   1. a 2D grid of CTAs, each owning kGradRows rows and one chunk of the
//      systems, accumulates its products in FP64 (threads stride over the
//      chunk's systems; warp shuffles and a shared-memory tree combine the
//      threads) and writes one partial per (chunk, band, row) to scratch;
//   2. one thread per (band, row) adds the chunks' partials in chunk order.
// The grid shape is a function of N and M only, so the result is bitwise
// reproducible.  Work per unknown: `width` FP64 FMAs (the kernel is bound by
// the FP64 pipe on GB300), 16 bytes of compulsory reads (GB and X; the X
// halo of 2h rows per block of kGradRows comes mostly from L2).
#include <mutex>
#include <string>

#include "sweep_kernels.cuh"

namespace bs {

constexpr int kGradThreads = 256;
constexpr int kGradRows = 8;
constexpr int kGradTargetCtas = 512;
constexpr int64_t kGradMinChunk = 1024;  // systems per chunk at least

struct GradShape {
  int row_blocks;
  int chunks;
  int64_t chunk;  // systems per chunk (multiple of 2)
};

GradShape grad_shape(int N, int64_t M) {
  GradShape g{};
  g.row_blocks = (N + kGradRows - 1) / kGradRows;
  int64_t c = (kGradTargetCtas + g.row_blocks - 1) / g.row_blocks;
  const int64_t cmax = (M + kGradMinChunk - 1) / kGradMinChunk;
  if (c > cmax) c = cmax;
  if (c < 1) c = 1;
  int64_t chunk = (M + c - 1) / c;
  chunk = (chunk + 1) / 2 * 2;
  g.chunks = (int)((M + chunk - 1) / chunk);
  g.chunk = chunk;
  return g;
}

size_t band_grad_scratch_bytes(int width, int N, int64_t M) {
  const GradShape g = grad_shape(N, M);
  return (size_t)g.chunks * width * N * sizeof(double);
}

// Level 1.  blockIdx.x = row block, blockIdx.y = chunk.  partial layout:
// [chunk][band][row].  PER: periodic matrix, X rows taken modulo N.
template <typename T, int W, bool PER>
__global__ void __launch_bounds__(kGradThreads)
k_band_grad_partial(int N, int64_t M, int64_t chunk, const T* __restrict__ GB, const T* __restrict__ X, int64_t rs,
                    int64_t ss, double* __restrict__ partial) {
  constexpr int H = W / 2;
  constexpr int NX = kGradRows + 2 * H;
  __shared__ double red[kGradThreads / 32][kGradRows * W];
  const int i0 = blockIdx.x * kGradRows;
  const int64_t jlo = (int64_t)blockIdx.y * chunk;
  const int64_t jhi = (jlo + chunk) < M ? (jlo + chunk) : M;
  double acc[kGradRows][W];
#pragma unroll
  for (int r = 0; r < kGradRows; r++)
#pragma unroll
    for (int k = 0; k < W; k++) acc[r][k] = 0.0;

  for (int64_t j = jlo + threadIdx.x; j < jhi; j += kGradThreads) {
    double x[NX], g[kGradRows];
#pragma unroll
    for (int q = 0; q < NX; q++) {
      const int row = i0 - H + q;
      if constexpr (PER) {
        const int pr = ((row % N) + N) % N;
        x[q] = (double)X[pr * rs + j * ss];
      } else {
        x[q] = (row >= 0 && row < N) ? (double)X[row * rs + j * ss] : 0.0;
      }
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
    const int row = i0 + r;
    if (row < N) partial[((int64_t)blockIdx.y * W + k) * N + row] = s;
  }
}

// Level 2: dbands[k*N + i] = -(sum over chunks, in order); 0 outside the
// matrix (a periodic matrix has no entries outside).
__global__ void k_band_grad_finish(int W, int N, int chunks, int periodic, const double* __restrict__ partial,
                                   double* __restrict__ dbands) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)W * N) return;
  const int k = (int)(t / N), i = (int)(t % N);
  const int col = i + k - W / 2;
  double s = 0.0;
  for (int c = 0; c < chunks; c++) s += partial[(int64_t)c * W * N + t];
  dbands[t] = (periodic || (col >= 0 && col < N)) ? -s : 0.0;
}

// Both levels with caller-provided scratch of band_grad_scratch_bytes().
cudaError_t band_grad_with_scratch(int width, int N, bool periodic, const void* GB, const void* X, bs_dtype t,
                                   bs_layout layout, int64_t M, double* dbands, double* scratch, cudaStream_t st) {
  const int64_t rs = layout == BS_INTERLEAVED ? M : 1;
  const int64_t ss = layout == BS_INTERLEAVED ? 1 : N;
  const GradShape g = grad_shape(N, M);
  const dim3 grid(g.row_blocks, g.chunks);
  if (periodic) {  // width 3 only
    if (t == BS_F64)
      k_band_grad_partial<double, 3, true><<<grid, kGradThreads, 0, st>>>(N, M, g.chunk, (const double*)GB,
                                                                           (const double*)X, rs, ss, scratch);
    else
      k_band_grad_partial<float, 3, true><<<grid, kGradThreads, 0, st>>>(N, M, g.chunk, (const float*)GB,
                                                                          (const float*)X, rs, ss, scratch);
  } else if (t == BS_F64) {
    if (width == 3)
      k_band_grad_partial<double, 3, false><<<grid, kGradThreads, 0, st>>>(N, M, g.chunk, (const double*)GB,
                                                                     (const double*)X, rs, ss, scratch);
    else
      k_band_grad_partial<double, 5, false><<<grid, kGradThreads, 0, st>>>(N, M, g.chunk, (const double*)GB,
                                                                     (const double*)X, rs, ss, scratch);
  } else {
    if (width == 3)
      k_band_grad_partial<float, 3, false><<<grid, kGradThreads, 0, st>>>(N, M, g.chunk, (const float*)GB,
                                                                    (const float*)X, rs, ss, scratch);
    else
      k_band_grad_partial<float, 5, false><<<grid, kGradThreads, 0, st>>>(N, M, g.chunk, (const float*)GB,
                                                                    (const float*)X, rs, ss, scratch);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t n = (int64_t)width * N;
  k_band_grad_finish<<<(int)((n + 255) / 256), 256, 0, st>>>(width, N, g.chunks, periodic ? 1 : 0, scratch,
                                                             dbands);
  return cudaGetLastError();
}

bs_status launch_band_grad(bs_handle h, const void* GB, const void* X, bs_dtype t, bs_layout layout, int64_t M,
                           double* dbands, cudaStream_t st) {
  const int N = (int)h->N;
  double* scratch = nullptr;
  const size_t bytes = band_grad_scratch_bytes(h->width, N, M);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), bytes, st);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? set_error(BS_ENOMEM, "band gradient: scratch")
                                                              : cuda_error(e, "band gradient scratch");
  e = band_grad_with_scratch(h->width, N, h->periodic, GB, X, t, layout, M, dbands, scratch, st);
  const cudaError_t e2 = cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) return cuda_error(e, "band gradient launch");
  if (e2 != cudaSuccess) return cuda_error(e2, "band gradient scratch release");
  return BS_OK;
}

// ------------------------------------------------- no-allocation variant
//
// bs_band_grad_noalloc runs the same two levels as bs_band_grad, but keeps the
// per-chunk partials in this fixed device array instead of memory allocated
// per call, for callers that must not allocate device memory while they run
// (see include/bsolve.h).  Every GPU that loads the library holds the array
// (2 MiB) until the process exits.  The name below is only a host-side
// stand-in for the device array: host code must pass the device address that
// cudaGetSymbolAddress returns, looked up once per device.
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 18;
static __device__ __align__(256) double g_band_grad_scratch[kNoAllocScratchDoubles];

// Device address of g_band_grad_scratch on the current device, looked up on
// the first call for that device (the device must be current).
static cudaError_t noalloc_scratch(double** out) {
  static std::mutex mu;
  static double* ptr[64] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (!ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_band_grad_scratch);
    if (e != cudaSuccess) return e;
    ptr[dev] = static_cast<double*>(p);
  }
  *out = ptr[dev];
  return cudaSuccess;
}

}  // namespace bs

extern "C" bs_status bs_band_grad_noalloc(bs_handle h, const void* GB, const void* X, bs_dtype dtype,
                                          bs_layout layout, int64_t M, double* dbands, bs_stream stream) {
  using namespace bs;
  if (!valid_handle(h)) return set_error(BS_EINVAL, "bs_band_grad_noalloc: unknown handle");
  if (!GB || !X || !dbands) return set_error(BS_EINVAL, "bs_band_grad_noalloc: null data pointer");
  if (M < 1) return set_error(BS_EINVAL, "bs_band_grad_noalloc: M must be >= 1");
  if (layout != BS_INTERLEAVED && layout != BS_STRIDED)
    return set_error(BS_EINVAL, "bs_band_grad_noalloc: bad layout");
  if (dtype != BS_F64 && dtype != BS_F32)
    return set_error(BS_EINVAL, "bs_band_grad_noalloc: dtype must be BS_F64 or BS_F32");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) return set_error(BS_EINVAL, "bs_band_grad_noalloc: handle belongs to another device");
  const int N = (int)h->N;
  const size_t need = band_grad_scratch_bytes(h->width, N, M) / sizeof(double);
  if (need > kNoAllocScratchDoubles)
    return set_error(BS_EINVAL, "bs_band_grad_noalloc: this size needs " + std::to_string(need) +
                                    " doubles of scratch, more than the " +
                                    std::to_string(kNoAllocScratchDoubles) +
                                    " the fixed array holds; use bs_band_grad");
  double* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return cuda_error(e, "bs_band_grad_noalloc: scratch address");
  e = band_grad_with_scratch(h->width, N, h->periodic, GB, X, dtype, layout, M, dbands, scratch,
                             reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "bs_band_grad_noalloc launch");
  return BS_OK;
}

