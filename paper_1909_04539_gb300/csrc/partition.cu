// Row-partitioned banded solves for batches too small to fill the GPU with
// one thread per system (e.g. the 4096 lines of an ADI half-step, where each
// SM would hold less than one warp and the FP64 pipes of most SM
// sub-partitions would idle).
//
// The rows are cut into P blocks of L rows.  Step 1 is the ordinary sweep
// kernel run on the block-diagonal matrix A_blk (A without its entries that
// couple different blocks) with grid.y = P, one thread per (system, block):
// y = A_blk^{-1} d.  Since A = A_blk + (couplings), inside block k
//   x = y - sum_m V_m x_{top(k)-m} - sum_m W_m x_{bot(k)+m},   m = 1 .. h,
// with the spikes V_m, W_m (one copy for all systems: the LHS is shared).
// Step 2 (k_part_reduced) solves, per system, the banded reduced system for
// the 2h values at each block edge (rows bot(b)-h+1 .. bot(b), top(b+1) ..
// top(b+1)+h-1), whose LU is computed once with the handle.  Step 3
// (k_part_fix) applies the correction to the rows where a spike is non-zero:
// the first kv and the last kw rows of each block (spike entries below 2^-60
// of their maximum are zero, which changes no result above rounding).
#include "sweep_kernels.cuh"

namespace bs {

constexpr int kPartThreads = 256;

// Largest bandwidth of the reduced system's LU for half-width H: the unknowns
// of one block edge couple to those of the neighbouring edges, at most
// 3H - 1 positions away (2 for tridiagonal, 5 for pentadiagonal matrices).
template <int H>
__host__ __device__ constexpr int part_band() {
  return 3 * H - 1;
}

__device__ __forceinline__ int part_top(int b, int L) { return b * L; }
__device__ __forceinline__ int part_bot(int b, int L, int N) { return ((b + 1) * L < N ? (b + 1) * L : N) - 1; }

// Matrix row of reduced unknown zi.
template <int H>
__device__ __forceinline__ int part_zrow(int zi, int L, int N) {
  const int b = zi / (2 * H), t = zi % (2 * H);
  return t < H ? part_bot(b, L, N) - H + 1 + t : part_top(b + 1, L) + (t - H);
}

// Step 2: one thread per system.  bt (R x M, unknown i of the reduced system
// at bt[i * M + j]) receives the forward values, then the solution.  Rows are
// taken in groups of 8 whose loads are all issued before the group's
// recurrence runs, so a thread waits for memory once per group.
template <typename C, int H>
__global__ void __launch_bounds__(kPartThreads)
k_part_reduced(const C* __restrict__ lu, int R, int p, int q, int L, int N, const C* __restrict__ X, int64_t rs,
               int64_t ss, int64_t M, C* __restrict__ bt) {
  constexpr int G = 8;
  constexpr int kPartBand = part_band<H>();
  const C* dinv = lu + (int64_t)p * R;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
    C win[kPartBand];  // win[k] = the value k + 1 rows back
#pragma unroll
    for (int k = 0; k < kPartBand; k++) win[k] = C(0);
    for (int i0 = 0; i0 < R; i0 += G) {
      C z[G];
#pragma unroll
      for (int u = 0; u < G; u++) {
        const int i = i0 + u;
        z[u] = i < R ? X[part_zrow<H>(i, L, N) * rs + j * ss] : C(0);
      }
#pragma unroll
      for (int u = 0; u < G; u++) {
        const int i = i0 + u;
        if (i < R) {
          C v = z[u];
#pragma unroll
          for (int k = 0; k < kPartBand; k++)
            if (k < p) v = fma(-lu[(int64_t)k * R + i], win[k], v);
#pragma unroll
          for (int k = kPartBand - 1; k > 0; k--) win[k] = win[k - 1];
          win[0] = v;
          bt[i * M + j] = v;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kPartBand; k++) win[k] = C(0);
    for (int i0 = R - 1; i0 >= 0; i0 -= G) {
      C z[G];
#pragma unroll
      for (int u = 0; u < G; u++) z[u] = (i0 - u >= 0) ? bt[(i0 - u) * M + j] : C(0);
#pragma unroll
      for (int u = 0; u < G; u++) {
        const int i = i0 - u;
        if (i >= 0) {
          C v = z[u];
#pragma unroll
          for (int k = 0; k < kPartBand; k++)
            if (k < q) v = fma(-lu[(int64_t)(p + 1 + k) * R + i], win[k], v);
          v *= dinv[i];
#pragma unroll
          for (int k = kPartBand - 1; k > 0; k--) win[k] = win[k - 1];
          win[0] = v;
          bt[i * M + j] = v;
        }
      }
    }
  }
}

// Step 3: x = y - sum_m V_m beta_m - sum_m W_m tau_m on the corrected rows of
// every block, beta_m = x_{top(k)-m} = z_{2h(k-1)+h-m}, tau_m = x_{bot(k)+m} =
// z_{2hk+h+m-1}.  Work item (k, q, j): q < kv is row top(k) + q, q >= kv is
// row bot(k) - (q - kv).  Interleaved layout: j varies fastest (coalesced);
// strided: q does.
template <typename C, int H, bool STRIDED>
__global__ void __launch_bounds__(kPartThreads)
k_part_fix(const C* __restrict__ spk, int P, int L, int N, int kv, int kw, C* __restrict__ X, int64_t rs,
           int64_t ss, int64_t M, const C* __restrict__ bt) {
  const int Q = kv + kw;
  const int64_t total = (int64_t)P * Q * M;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int k, q;
    int64_t j;
    if (STRIDED) {
      q = (int)(t % Q);
      const int64_t rest = t / Q;
      k = (int)(rest % P);
      j = rest / P;
    } else {
      j = t % M;
      const int64_t rest = t / M;
      q = (int)(rest % Q);
      k = (int)(rest / Q);
    }
    const int top = part_top(k, L), bot = part_bot(k, L, N);
    const int top_end = k > 0 ? top + kv : top;  // rows [top, top_end) form the top range
    int row;
    if (q < kv) {
      if (k == 0) continue;  // no block above
      row = top + q;
      if (row > bot) continue;
    } else {
      if (k == P - 1) continue;  // no block below
      row = bot - (q - kv);
      if (row < top_end) continue;  // already in the top range
    }
    C* px = X + row * rs + j * ss;
    C x = *px;
#pragma unroll
    for (int m = 1; m <= H; m++) {
      if (k > 0) x = fma(-spk[(int64_t)(m - 1) * N + row], bt[(int64_t)(2 * H * (k - 1) + H - m) * M + j], x);
      if (k < P - 1) x = fma(-spk[(int64_t)(H + m - 1) * N + row], bt[(int64_t)(2 * H * k + H + m - 1) * M + j], x);
    }
    *px = x;
  }
}

template <typename C, int H>
static cudaError_t part_correct_t(const PartPlan& pp, int N, C* X, bs_layout layout, int64_t M, C* bt,
                                  cudaStream_t st) {
  const int64_t rs = layout == BS_INTERLEAVED ? M : 1;
  const int64_t ss = layout == BS_INTERLEAVED ? 1 : N;
  const C* lu;
  const C* spk;
  if constexpr (sizeof(C) == 8) {
    lu = reinterpret_cast<const C*>(pp.red64);
    spk = reinterpret_cast<const C*>(pp.spk64);
  } else {
    lu = reinterpret_cast<const C*>(pp.red32);
    spk = reinterpret_cast<const C*>(pp.spk32);
  }
  const int sms = device_info().sms;
  int64_t g = (M + kPartThreads - 1) / kPartThreads;
  k_part_reduced<C, H><<<(int)(g < 1 ? 1 : g), kPartThreads, 0, st>>>(lu, pp.R, pp.p, pp.q, pp.L, N, X, rs, ss,
                                                                       M, bt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)pp.P * (pp.kv + pp.kw) * M;
  if (total == 0) return cudaSuccess;
  g = (total + kPartThreads - 1) / kPartThreads;
  const int64_t cap = (int64_t)sms * 8;
  if (g > cap) g = cap;
  if (layout == BS_STRIDED)
    k_part_fix<C, H, true><<<(int)g, kPartThreads, 0, st>>>(spk, pp.P, pp.L, N, pp.kv, pp.kw, X, rs, ss, M, bt);
  else
    k_part_fix<C, H, false><<<(int)g, kPartThreads, 0, st>>>(spk, pp.P, pp.L, N, pp.kv, pp.kw, X, rs, ss, M, bt);
  return cudaGetLastError();
}

template <typename C>
static cudaError_t part_correct_c(const PartPlan& pp, int N, C* X, bs_layout layout, int64_t M, C* bt,
                                  cudaStream_t st) {
  return pp.h == 1 ? part_correct_t<C, 1>(pp, N, X, layout, M, bt, st)
                   : part_correct_t<C, 2>(pp, N, X, layout, M, bt, st);
}

// Steps 2 and 3 on X (FP64 or FP32 values), with stream-ordered scratch for
// the reduced systems.
bs_status part_correct(const PartPlan& pp, int N, void* X, bs_dtype t, bs_layout layout, int64_t M,
                       cudaStream_t st) {
  const size_t es = t == BS_F64 ? sizeof(double) : sizeof(float);
  void* bt = nullptr;
  cudaError_t e = cudaMallocAsync(&bt, (size_t)pp.R * (size_t)M * es, st);
  if (e != cudaSuccess)
    return e == cudaErrorMemoryAllocation ? set_error(BS_ENOMEM, "partitioned solve: scratch")
                                          : cuda_error(e, "partitioned solve scratch");
  if (t == BS_F64)
    e = part_correct_c<double>(pp, N, static_cast<double*>(X), layout, M, static_cast<double*>(bt), st);
  else
    e = part_correct_c<float>(pp, N, static_cast<float*>(X), layout, M, static_cast<float*>(bt), st);
  const cudaError_t e2 = cudaFreeAsync(bt, st);
  if (e != cudaSuccess) return cuda_error(e, "partitioned solve correction");
  if (e2 != cudaSuccess) return cuda_error(e2, "partitioned solve scratch release");
  return BS_OK;
}

}  // namespace bs
