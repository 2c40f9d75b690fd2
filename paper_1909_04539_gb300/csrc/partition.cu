// Row-partitioned tridiagonal solves for batches too small to fill the GPU
// with one thread per system (e.g. the 4096 lines of an ADI half-step, where
// each SM would hold less than one warp and the FP64 pipes of most SM
// sub-partitions would idle).
//
// The rows are cut into P blocks of L rows.  Step 1 is the ordinary sweep
// kernel run on the block-diagonal matrix A_blk (A without the couplings
// across block edges) with grid.y = P, one thread per (system, block):
// y = A_blk^{-1} d.  Since A = A_blk + (couplings), inside block k
//   x = y - V x_{top(k)-1} - W x_{bot(k)+1},
// with the spikes V = A_k^{-1} (a_top e_1), W = A_k^{-1} (c_bot e_L), one copy
// for all systems because the LHS is shared.  Step 2 (k_part_reduced) solves,
// per system, the pentadiagonal reduced system for the values at the block
// edges, z = (x_bot(0), x_top(1), x_bot(1), x_top(2), ...), whose
// factorisation is computed once with the handle.  Step 3 (k_part_fix)
// applies the correction to the rows where a spike is non-zero: the first kv
// and the last kw rows of each block (spike entries below 2^-60 of their
// maximum are zero, which changes no result above rounding).
#include "sweep_kernels.cuh"

namespace bs {

constexpr int kPartThreads = 256;

__device__ __forceinline__ int part_top(int b, int L) { return b * L; }
__device__ __forceinline__ int part_bot(int b, int L, int N) { return ((b + 1) * L < N ? (b + 1) * L : N) - 1; }

// Step 2: one thread per system.  bt (R x M, row q of the reduced system at
// bt[q * M + j]) receives the forward values, then the solution.  Rows are
// taken in groups of 8 whose loads are all issued before the group's
// recurrence runs, so a thread waits for memory once per group.
template <typename C>
__global__ void __launch_bounds__(kPartThreads)
k_part_reduced(Coefs<C> rc, int R, int L, int N, const C* __restrict__ X, int64_t rs, int64_t ss, int64_t M,
               C* __restrict__ bt) {
  constexpr int G = 8;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
    C w1 = C(0), w2 = C(0);
    for (int q0 = 0; q0 < R; q0 += G) {
      C z[G];
#pragma unroll
      for (int u = 0; u < G; u++) {
        const int q = q0 + u;
        const int row = (q & 1) ? part_top(q / 2 + 1, L) : part_bot(q / 2, L, N);
        z[u] = q < R ? X[row * rs + j * ss] : C(0);
      }
#pragma unroll
      for (int u = 0; u < G; u++) {
        const int q = q0 + u;
        if (q < R) {
          C w = rc.s[q] * z[u];
          w = fma(-rc.l2[q], w2, w);
          w = fma(-rc.l1[q], w1, w);
          w2 = w1;
          w1 = w;
          bt[q * M + j] = w;
        }
      }
    }
    C x1 = C(0), x2 = C(0);
    for (int q0 = R - 1; q0 >= 0; q0 -= G) {
      C z[G];
#pragma unroll
      for (int u = 0; u < G; u++) z[u] = (q0 - u >= 0) ? bt[(q0 - u) * M + j] : C(0);
#pragma unroll
      for (int u = 0; u < G; u++) {
        const int q = q0 - u;
        if (q >= 0) {
          C x = z[u];
          x = fma(-rc.u2[q], x2, x);
          x = fma(-rc.u1[q], x1, x);
          x2 = x1;
          x1 = x;
          bt[q * M + j] = x;
        }
      }
    }
  }
}

// Step 3: x = y - V beta - W tau on the corrected rows of every block, with
// beta = x_bot(k-1) = z_{2(k-1)} and tau = x_top(k+1) = z_{2k+1}.  Work item
// (k, q, j): q < kv is row top(k) + q, q >= kv is row bot(k) - (q - kv).
// Interleaved layout: j varies fastest (coalesced); strided: q does.
template <typename C, bool STRIDED>
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
    const C beta = k > 0 ? bt[(int64_t)(2 * (k - 1)) * M + j] : C(0);
    const C tau = k < P - 1 ? bt[(int64_t)(2 * k + 1) * M + j] : C(0);
    C* px = X + row * rs + j * ss;
    C x = fma(-spk[row], beta, *px);
    *px = fma(-spk[N + row], tau, x);
  }
}

template <typename C>
static cudaError_t part_correct_t(const PartPlan& pp, int N, C* X, bs_layout layout, int64_t M, C* bt,
                                  cudaStream_t st) {
  const int64_t rs = layout == BS_INTERLEAVED ? M : 1;
  const int64_t ss = layout == BS_INTERLEAVED ? 1 : N;
  const C* rbase;
  const C* spk;
  if constexpr (sizeof(C) == 8) {
    rbase = reinterpret_cast<const C*>(pp.red.c64);
    spk = reinterpret_cast<const C*>(pp.spk64);
  } else {
    rbase = reinterpret_cast<const C*>(pp.red.c32);
    spk = reinterpret_cast<const C*>(pp.spk32);
  }
  const Coefs<C> rc = coefs_of<C>(rbase, pp.R);
  const int sms = device_info().sms;
  int64_t g = (M + kPartThreads - 1) / kPartThreads;
  k_part_reduced<C><<<(int)(g < 1 ? 1 : g), kPartThreads, 0, st>>>(rc, pp.R, pp.L, N, X, rs, ss, M, bt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)pp.P * (pp.kv + pp.kw) * M;
  if (total == 0) return cudaSuccess;
  g = (total + kPartThreads - 1) / kPartThreads;
  const int64_t cap = (int64_t)sms * 8;
  if (g > cap) g = cap;
  if (layout == BS_STRIDED)
    k_part_fix<C, true><<<(int)g, kPartThreads, 0, st>>>(spk, pp.P, pp.L, N, pp.kv, pp.kw, X, rs, ss, M, bt);
  else
    k_part_fix<C, false><<<(int)g, kPartThreads, 0, st>>>(spk, pp.P, pp.L, N, pp.kv, pp.kw, X, rs, ss, M, bt);
  return cudaGetLastError();
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
    e = part_correct_t<double>(pp, N, static_cast<double*>(X), layout, M, static_cast<double*>(bt), st);
  else
    e = part_correct_t<float>(pp, N, static_cast<float*>(X), layout, M, static_cast<float*>(bt), st);
  const cudaError_t e2 = cudaFreeAsync(bt, st);
  if (e != cudaSuccess) return cuda_error(e, "partitioned solve correction");
  if (e2 != cudaSuccess) return cuda_error(e2, "partitioned solve scratch release");
  return BS_OK;
}

}  // namespace bs
