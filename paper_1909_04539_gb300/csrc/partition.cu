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
// (k_part_fix_il / k_part_fix_st for the two layouts) applies the correction
// to the rows where a spike is non-zero:
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

// Step 2: one-warp CTAs, one thread per system.  Each lane first copies its
// system's R block-edge values into its column of a shared R x 32 tile with
// cp.async (all R copies in flight at once), and the LU factors of the
// reduced matrix are staged beside it; the two recurrences then run from
// shared memory, and only the solution goes out, to bt (R x M, unknown i of
// system j at bt[i * M + j]).  In each row the terms of the older values are
// added first, so only the last FMA waits for the previous row's result.
constexpr int kPartRedThreads = 32;

template <typename C>
__device__ __forceinline__ void part_cp(uint32_t dst, const C* src) {
  if constexpr (sizeof(C) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}

template <typename C, int H>
__global__ void __launch_bounds__(kPartRedThreads)
k_part_reduced(const C* __restrict__ lu_g, int R, int p, int q, int L, int N, const C* __restrict__ X, int64_t rs,
               int64_t ss, int64_t M, C* __restrict__ bt) {
  constexpr int kPartBand = part_band<H>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* lu = reinterpret_cast<C*>(smem_raw);  // (p + q + 1) x R
  C* zt = lu + (size_t)(p + q + 1) * R;    // R x 32: value i of lane t at zt[i * 32 + t]
  const int lane = threadIdx.x;
  for (int e = lane; e < (p + q + 1) * R; e += kPartRedThreads) lu[e] = lu_g[e];
  const C* dinv = lu + (size_t)p * R;
  for (int64_t j0 = (int64_t)blockIdx.x * kPartRedThreads; j0 < M; j0 += (int64_t)gridDim.x * kPartRedThreads) {
    const int64_t j = j0 + lane;
    const bool valid = j < M;
    if (valid)
      for (int i = 0; i < R; i++)
        part_cp(smem_u32(zt + i * kPartRedThreads + lane), X + part_zrow<H>(i, L, N) * rs + j * ss);
    cp_commit();
    cp_wait<0>();
    __syncwarp();  // also orders the lu staging before its first use
    if (valid) {
      C win[kPartBand];  // win[k] = the value k + 1 rows back
#pragma unroll
      for (int k = 0; k < kPartBand; k++) win[k] = C(0);
      for (int i = 0; i < R; i++) {
        C v = zt[i * kPartRedThreads + lane];
#pragma unroll
        for (int k = kPartBand - 1; k >= 0; k--)
          if (k < p) v = fma(-lu[(size_t)k * R + i], win[k], v);
#pragma unroll
        for (int k = kPartBand - 1; k > 0; k--) win[k] = win[k - 1];
        win[0] = v;
        zt[i * kPartRedThreads + lane] = v;
      }
#pragma unroll
      for (int k = 0; k < kPartBand; k++) win[k] = C(0);
      for (int i = R - 1; i >= 0; i--) {
        C v = zt[i * kPartRedThreads + lane];
#pragma unroll
        for (int k = kPartBand - 1; k >= 0; k--)
          if (k < q) v = fma(-lu[(size_t)(p + 1 + k) * R + i], win[k], v);
        v *= dinv[i];
#pragma unroll
        for (int k = kPartBand - 1; k > 0; k--) win[k] = win[k - 1];
        win[0] = v;
        bt[i * M + j] = v;
      }
    }
    __syncwarp();  // the tile is reused by the next group of systems
  }
}

// Step 3: x = y - sum_m V_m beta_m - sum_m W_m tau_m on the corrected rows of
// every block, beta_m = x_{top(k)-m} = z_{2h(k-1)+h-m}, tau_m = x_{bot(k)+m} =
// z_{2hk+h+m-1}.  Corrected row q of block k: q < kv is row top(k) + q,
// q >= kv is row bot(k) - (q - kv).
__device__ __forceinline__ int part_fix_row(int k, int q, int P, int L, int N, int kv) {
  const int top = part_top(k, L), bot = part_bot(k, L, N);
  const int top_end = k > 0 ? top + kv : top;  // rows [top, top_end) form the top range
  if (q < kv) {
    if (k == 0) return -1;  // no block above
    const int row = top + q;
    return row > bot ? -1 : row;
  }
  if (k == P - 1) return -1;  // no block below
  const int row = bot - (q - kv);
  return row < top_end ? -1 : row;  // already in the top range
}

template <typename C, int H>
__device__ __forceinline__ C part_fix_one(C x, const C* __restrict__ spk, int k, int P, int N, int row, int64_t M,
                                          int64_t j, const C* __restrict__ bt) {
#pragma unroll
  for (int m = 1; m <= H; m++) {
    if (k > 0) x = fma(-spk[(int64_t)(m - 1) * N + row], bt[(int64_t)(2 * H * (k - 1) + H - m) * M + j], x);
    if (k < P - 1) x = fma(-spk[(int64_t)(H + m - 1) * N + row], bt[(int64_t)(2 * H * k + H + m - 1) * M + j], x);
  }
  return x;
}

// Interleaved layout: blockIdx.y is the block k, blockIdx.z a group of G of
// its corrected rows; the threads take consecutive systems (coalesced).  The
// rows and their spike entries are the same for the whole CTA and stay in
// registers, each thread reads its system's 2h edge values once, and the G
// rows' loads are all issued before their arithmetic (G = 8 rows for
// tridiagonal matrices, 4 for pentadiagonal ones, whose spike entries take
// twice the registers).
template <int H>
__host__ __device__ constexpr int part_fix_rows() {
  return H == 1 ? 8 : 4;
}

template <typename C, int H>
__global__ void __launch_bounds__(kPartThreads)
k_part_fix_il(const C* __restrict__ spk, int P, int L, int N, int kv, int kw, C* __restrict__ X, int64_t M,
              const C* __restrict__ bt) {
  constexpr int G = part_fix_rows<H>();
  const int Q = kv + kw;
  const int k = blockIdx.y;
  int row[G];
  C sv[G][H], sw[G][H];
#pragma unroll
  for (int g = 0; g < G; g++) {
    const int q = blockIdx.z * G + g;
    row[g] = q < Q ? part_fix_row(k, q, P, L, N, kv) : -1;
    const int rr = row[g] < 0 ? 0 : row[g];
#pragma unroll
    for (int m = 0; m < H; m++) {
      sv[g][m] = k > 0 ? spk[(int64_t)m * N + rr] : C(0);
      sw[g][m] = k < P - 1 ? spk[(int64_t)(H + m) * N + rr] : C(0);
    }
  }
  for (int64_t j = (int64_t)blockIdx.x * kPartThreads + threadIdx.x; j < M; j += (int64_t)gridDim.x * kPartThreads) {
    // beta_m = x_{top(k)-m} = z_{2h(k-1)+h-m}, tau_m = x_{bot(k)+m} = z_{2hk+h+m-1}
    C beta[H], tau[H], xv[G];
#pragma unroll
    for (int m = 0; m < H; m++) {
      beta[m] = k > 0 ? bt[(int64_t)(2 * H * (k - 1) + H - 1 - m) * M + j] : C(0);
      tau[m] = k < P - 1 ? bt[(int64_t)(2 * H * k + H + m) * M + j] : C(0);
    }
#pragma unroll
    for (int g = 0; g < G; g++) xv[g] = row[g] >= 0 ? X[(int64_t)row[g] * M + j] : C(0);
#pragma unroll
    for (int g = 0; g < G; g++) {
      if (row[g] >= 0) {
        C x = xv[g];
#pragma unroll
        for (int m = 0; m < H; m++) {
          if (k > 0) x = fma(-sv[g][m], beta[m], x);
          if (k < P - 1) x = fma(-sw[g][m], tau[m], x);
        }
        X[(int64_t)row[g] * M + j] = x;
      }
    }
  }
}

// Strided layout: threadIdx.x walks the corrected rows of a system
// (consecutive addresses within each of the two ranges), each warp S
// systems at once (their edge values and rows loaded before the arithmetic),
// blockIdx.y the blocks.
constexpr int kPartFixWarps = kPartThreads / 32;
constexpr int kPartFixSys = 4;  // systems per warp

template <typename C, int H>
__global__ void __launch_bounds__(kPartThreads)
k_part_fix_st(const C* __restrict__ spk, int P, int L, int N, int kv, int kw, C* __restrict__ X, int64_t M,
              const C* __restrict__ bt) {
  constexpr int S = kPartFixSys;
  const int Q = kv + kw;
  const int k = blockIdx.y;
  const int64_t step = (int64_t)gridDim.x * kPartFixWarps * S;
  for (int64_t j0 = ((int64_t)blockIdx.x * kPartFixWarps + threadIdx.y) * S; j0 < M; j0 += step) {
    // beta_m = x_{top(k)-m} = z_{2h(k-1)+h-m}, tau_m = x_{bot(k)+m} = z_{2hk+h+m-1}
    C beta[S][H], tau[S][H];
#pragma unroll
    for (int s = 0; s < S; s++) {
      const int64_t j = j0 + s < M ? j0 + s : j0;
#pragma unroll
      for (int m = 0; m < H; m++) {
        beta[s][m] = k > 0 ? bt[(int64_t)(2 * H * (k - 1) + H - 1 - m) * M + j] : C(0);
        tau[s][m] = k < P - 1 ? bt[(int64_t)(2 * H * k + H + m) * M + j] : C(0);
      }
    }
    for (int q = threadIdx.x; q < Q; q += 32) {
      const int row = part_fix_row(k, q, P, L, N, kv);
      if (row < 0) continue;
      C sv[H], sw[H], xv[S];
#pragma unroll
      for (int m = 0; m < H; m++) {
        sv[m] = k > 0 ? spk[(int64_t)m * N + row] : C(0);
        sw[m] = k < P - 1 ? spk[(int64_t)(H + m) * N + row] : C(0);
      }
#pragma unroll
      for (int s = 0; s < S; s++) xv[s] = j0 + s < M ? X[(j0 + s) * N + row] : C(0);
#pragma unroll
      for (int s = 0; s < S; s++) {
        if (j0 + s < M) {
          C x = xv[s];
#pragma unroll
          for (int m = 0; m < H; m++) {
            if (k > 0) x = fma(-sv[m], beta[s][m], x);
            if (k < P - 1) x = fma(-sw[m], tau[s][m], x);
          }
          X[(j0 + s) * N + row] = x;
        }
      }
    }
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
  const size_t red_smem = ((size_t)(pp.p + pp.q + 1) * pp.R + (size_t)pp.R * kPartRedThreads) * sizeof(C);
  auto kr = k_part_reduced<C, H>;
  cudaError_t e = cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)red_smem);
  if (e != cudaSuccess) return e;
  int64_t g = (M + kPartRedThreads - 1) / kPartRedThreads;
  if (g > 65535) g = 65535;
  kr<<<(int)(g < 1 ? 1 : g), kPartRedThreads, red_smem, st>>>(lu, pp.R, pp.p, pp.q, pp.L, N, X, rs, ss, M, bt);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int Q = pp.kv + pp.kw;
  if (Q == 0 || pp.P < 2) return cudaSuccess;
  if (layout == BS_STRIDED) {
    int64_t gx = (M + kPartFixWarps * kPartFixSys - 1) / (kPartFixWarps * kPartFixSys);
    if (gx > 65535) gx = 65535;
    k_part_fix_st<C, H><<<dim3((unsigned)gx, (unsigned)pp.P), dim3(32, kPartFixWarps), 0, st>>>(
        spk, pp.P, pp.L, N, pp.kv, pp.kw, X, M, bt);
  } else {
    int64_t gx = (M + kPartThreads - 1) / kPartThreads;
    if (gx > 65535) gx = 65535;
    const int gz = (Q + part_fix_rows<H>() - 1) / part_fix_rows<H>();  // Q <= L / 2 <= N / 2, P <= 32
    k_part_fix_il<C, H><<<dim3((unsigned)gx, (unsigned)pp.P, (unsigned)gz), kPartThreads, 0, st>>>(
        spk, pp.P, pp.L, N, pp.kv, pp.kw, X, M, bt);
  }
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
