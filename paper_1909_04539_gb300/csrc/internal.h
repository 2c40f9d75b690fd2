// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/bsolve.h"

#ifdef __CUDACC__
#define BS_HD __host__ __device__
#else
#define BS_HD
#endif

namespace bs {

// Coefficients of one sweep pair, each an array of N values.  Every solve of
// the library (primal and adjoint, tri and penta) has the form
//   forward : w_i = s_i f_i - l1_i w_{i-1} - l2_i w_{i-2}          (i = 0..N-1)
//   backward: x_i = t_i w_i - u1_i x_{i+1} - u2_i x_{i+2}          (i = N-1..0)
// with s == 1 or t == 1 where the flags say so, l2 == u2 == 0 for width 3,
// and every coefficient that would reach outside the matrix stored as 0.
// A periodic (cyclic tridiagonal) plan adds the Sherman-Morrison rank-one
// correction (Sec. 3.3) in the same two passes: the forward pass also sums
// sigma = sum_i pw_i f_i over the raw right-hand side, and the backward pass
// writes x_i - sigma pc_i while the recurrence carries the uncorrected x_i.
enum { C_S = 0, C_L1, C_L2, C_T, C_U1, C_U2, C_PW, C_PC, C_COUNT };

template <typename C>
struct Coefs {
  const C* s;
  const C* l1;
  const C* l2;
  const C* t;
  const C* u1;
  const C* u2;
  const C* pw;  // periodic plans only
  const C* pc;
  int per_lo;   // rows per_lo <= i < per_hi have pw_i == pc_i == 0, so a
  int per_hi;   // block of rows inside that range skips the correction
  C eps;        // uniform pentadiagonal plans: the outermost sub-diagonal entry
};

struct SweepPlan {
  int bw;          // band half-width: 1 (tri) or 2 (penta)
  bool fwd_scale;  // s present
  bool bwd_scale;  // t present
  bool periodic;   // pw / pc present (Sherman-Morrison correction)
  int per_lo, per_hi;  // rows without correction terms (see Coefs)
  bool uniform;    // pentadiagonal with every a_i (i >= 3, 1-based) equal to eps
  double eps;
  double* c64;     // device, C_COUNT * N
  float* c32;      // device, C_COUNT * N
  // FP32-pair sweeps (sweep_df.cu) of primal and adjoint plans: per row the
  // coefficient pairs of each sweep packed as float4 + float2 (device, 48 N
  // bytes: forward float4 x N, backward float4 x N, forward float2 x N,
  // backward float2 x N); df_ok: the plan's sweep gains keep pair arithmetic
  // inside the FP32 range for inputs below 2^101 (see make_df_records)
  float* dfrec;
  bool df_ok;
  // periodic plans: per row the correction weights (pw', pc') = (2^k pw,
  // 2^-k pc) as FP32 pairs, (pw' hi, pw' lo, pc' hi, pc' lo) as float4 x N
  // (device; null otherwise); dfper_unscale = 2^-k (sigma = 2^-k sigma')
  float* dfper;
  double dfper_unscale;
  // Windowed sweeps (sweep_win.cu): FP32 records, per row forward
  // (s, l1, l2, 0) and backward (t, u1, u2, 0) as float4 (device, 32 N
  // bytes); win32 / win_df: rows after which a backward sweep started from
  // zero is within 2^-28 / 2^-50 of the true one (0: not windowed)
  float* rec32;
  int win32, win_df;
};

template <typename C>
BS_HD inline Coefs<C> coefs_of(const C* base, int64_t N) {
  return Coefs<C>{base + C_S * N,  base + C_L1 * N, base + C_L2 * N, base + C_T * N,
                  base + C_U1 * N, base + C_U2 * N, base + C_PW * N, base + C_PC * N, 0, 0};
}

}  // namespace bs

namespace bs {
// Row-partitioned solve of a banded matrix (half-width h = 1 or 2) for
// batches too small to fill the GPU one thread per system (e.g. the 4096
// lines of an ADI half-step).  Rows are cut into P blocks of L rows (the last
// may be shorter).  With A_blk = A without its entries that couple different
// blocks, y = A_blk^{-1} d is solved with one thread per (system, block);
// then inside block k
//   x = y - sum_m V_m x_{top-m} - sum_m W_m x_{bot+m}     (m = 1 .. h),
// V_m, W_m the block's spikes (one copy: the LHS is shared).  The 2h values
// at each block edge, z = (x_{bot(0)-h+1} .. x_{bot(0)}, x_{top(1)} ..
// x_{top(1)+h-1}, ...), R = 2h (P - 1) of them, solve a banded reduced system
// factorised once (LU without pivoting, lower bandwidth p, upper q), and the
// correction touches only the first kv and last kw rows of a block (spike
// entries below 2^-60 of their maximum are zero).
struct PartPlan {
  int P, L, R, kv, kw, h, p, q;
  SweepPlan blk;   // block-diagonal plan, C_COUNT x N
  double* spk64;   // 2h x N: V_1 .. V_h, then W_1 .. W_h
  float* spk32;
  double* red64;   // (p + q + 1) x R: row i of the LU at [k * R + i]: k < p the
  float* red32;    // multiplier of column i-1-k, k = p 1 / U_ii, k > p U_{i, i+k-p}
};
}  // namespace bs

namespace bs {
// Two-ended sweeps (small batches): the even lane of a pair eliminates rows
// 0 .. k-1 top-down with `top` (A = L U / L R), the odd lane rows N-1 .. k+h
// bottom-up with `bot` (A = U' L', coefficients in original row order), h
// the band half-width; the meeting rows k .. k+h-1 follow from their last
// forward values w_{k-1}, w_{k-2} and z_{k+h}, z_{k+h+1} with the weights m:
//   h = 1: x_k = (f_k + m0 w_{k-1} + m1 z_{k+1}) m2
//          (m0 = -a_k, m1 = -c_k, m2 = 1 / (b_k - a_k chat_{k-1} - c_k chat'_{k+1}))
//   h = 2: r0 = f_k + m0 w_{k-2} + m1 w_{k-1} + m2 z_{k+2},
//          r1 = f_{k+1} + m3 w_{k-1} + m4 z_{k+2} + m5 z_{k+3},
//          (x_k, x_{k+1}) = (m6 r0 + m7 r1, m8 r0 + m9 r1).
struct TwistPlan {
  bool ok;
  int k;
  double m[10];
  const SweepPlan* top;
  const SweepPlan* bot;
};
}  // namespace bs

struct bs_factor_s {
  int width;
  int64_t N;
  int device;
  bs::SweepPlan plan[3];   // [0] primal A^{-1} (A = L U), [1] adjoint A^{-T},
                           // [2] primal through the reversed factorisation A = U' L'
                           //     (first sweep runs over decreasing rows)
  double* bands64;         // device, width * N, entries outside the matrix zeroed
  float* bands_hi;         // device, width * N: FP32 rounding of the bands
  float* bands_lo;         // device, width * N: FP32 rounding of (band - hi)
  // The primal sweep coefficients of plan[0] as FP64 values split into FP32
  // high and low parts, 5 * N each: [0] s, [1] l1, [2] l2 (0 for tri),
  // [3] u1, [4] u2 (0 for tri); the high parts equal plan[0].c32.
  float* lu_hi;
  float* lu_lo;
  size_t device_bytes;
  bool has_ul;             // plan[2] is valid (reversed elimination met no bad pivot)
  bool has_part;           // part[] valid (N large enough, spikes decay)
  bs::PartPlan part[2];    // [0] for A, [1] for A^T
  bool periodic;           // cyclic tridiagonal (bs_factor_periodic): bands64 holds the
                           // corner entries a_1 (band 0, row 0) and c_N (band 2, row N-1)
  bool cn_pairs;           // the explicit side 2I - A of a Crank-Nicolson step may run in
                           // FP32 pairs: every band entry 0 or in [2^-20, 2^20] and every
                           // row's sum of |2I - A| entries at most 16 (cn.cu)
  bs::TwistPlan twist[2];  // two-ended tridiagonal sweeps: [0] for A (plan[0], plan[2]),
                           // [1] for A^T (tplan[])
  bs::SweepPlan tplan[2];  // A^T = L U and A^T = U' L' (primal form, original row order)
  int64_t server_refs;     // server requests naming this handle that have not finished
                           // (guarded by the handle registry's lock; bs_destroy refuses > 0)
};

namespace bs {

bs_status set_error(bs_status s, const std::string& msg);
bs_status cuda_error(cudaError_t e, const char* what);
bool valid_handle(bs_handle h);
// Pin / unpin a handle for a server request (false: unknown handle).
bool handle_ref(bs_handle h);
void handle_unref(bs_handle h);

struct DeviceInfo {
  int sms;
  int l2_bytes;
  int smem_optin;
};
const DeviceInfo& device_info();
int64_t option(int o);

// Launchers
bs_status launch_sweep(const SweepPlan& p, int64_t N, const void* in, void* out, bs_dtype in_t,
                       bs_dtype out_t, bs_layout layout, int64_t M, cudaStream_t st);
bs_status launch_refine(bs_handle h, const void* B, bs_dtype b_t, double* X, int64_t M, int steps, int mode,
                        cudaStream_t st);
bs_status launch_band_grad(bs_handle h, const void* GB, const void* X, bs_dtype t, bs_layout layout,
                           int64_t M, double* dbands, cudaStream_t st);
bool df_eligible(const SweepPlan& p, bs_layout layout);
// Launch shape of a persistent one-thread-per-group sweep whose CTAs stage
// rec_bytes of coefficient records in shared memory (if they fit) and use
// per_thread shared bytes per thread: grid, CTA size, whether staged.
struct StagedShape {
  int grid, threads;
  bool staged;
  double cost;  // busiest-SM warp shares summed over the grid's passes
};
StagedShape staged_shape(int64_t groups, size_t rec_bytes, size_t per_thread, int regs, int max_threads,
                         bool any_size, int prefer);
// registers per thread of a kernel (0 if unknown)
int kernel_regs(const void* kernel);
cudaError_t sweep_df(const SweepPlan& p, bool adjoint, int N, double* X, int64_t M, cudaStream_t st);
cudaError_t sweep_win_df(const SweepPlan& p, bool adjoint, int N, double* X, int64_t M, cudaStream_t st);
template <typename Sin>
cudaError_t sweep_win32(const SweepPlan& p, bool adjoint, int N, const Sin* in, float* out, int64_t M,
                        cudaStream_t st);
int win_rows(bool pairs);

}  // namespace bs
