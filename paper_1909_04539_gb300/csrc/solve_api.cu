// C-ABI entry points of the solves and the launch-shape policy.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <string>

#include "sweep_kernels.cuh"

namespace bs {

// L, P: row blocks of a partitioned solve (0, 1: none)
cudaError_t sweep_f64(const SweepPlan&, bool, int, const void*, void*, bs_layout, int64_t, cudaStream_t, int L = 0,
                      int P = 1);
cudaError_t sweep_f32(const SweepPlan&, bool, int, const void*, void*, bs_layout, int64_t, cudaStream_t, int L = 0,
                      int P = 1);
cudaError_t sweep_bf16(const SweepPlan&, bool, int, const void*, void*, bs_layout, int64_t, cudaStream_t, int L = 0,
                       int P = 1);

static int64_t g_opt[BS_OPT_COUNT] = {0};

int64_t option(int o) { return (o >= 0 && o < BS_OPT_COUNT) ? g_opt[o] : 0; }

// The shape of one launch for a given CTA size.
static LaunchShape shape_for(int bw, int N, int64_t threads_needed, size_t coef_elem, size_t spill_elem,
                             int per_thread_systems, size_t extra_smem_per_thread, size_t extra_smem_fixed, int tpb,
                             int extra_coef_arrays) {
  const DeviceInfo& d = device_info();
  LaunchShape sh{};
  sh.threads = tpb;
  const size_t coef_bytes = align_up((size_t)(1 + 2 * bw + extra_coef_arrays) * N * coef_elem, 16);
  const size_t extra = extra_smem_fixed + extra_smem_per_thread * (size_t)tpb;
  const size_t limit = (size_t)(d.smem_optin > 0 ? d.smem_optin : 48 * 1024) - 1024;
  sh.smem_coefs = coef_bytes + extra <= limit;
  sh.smem = sh.smem_coefs ? coef_bytes : 0;
  const int64_t blocks_needed = (threads_needed + tpb - 1) / tpb;
  const size_t per_block_smem = sh.smem + extra + 1024;
  int by_smem = (int)((228 * 1024) / per_block_smem);
  int by_threads = 2048 / tpb;
  int per_sm = (int)(option(BS_OPT_BLOCKS_PER_SM) > 0 ? option(BS_OPT_BLOCKS_PER_SM) : 32);
  if (per_sm > by_smem) per_sm = by_smem;
  if (per_sm > by_threads) per_sm = by_threads;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)d.sms * per_sm;
  // Optional bound on the forward values in flight (each thread keeps N rows
  // of its systems between the sweeps); off by default.
  const int64_t budget = option(BS_OPT_INFLIGHT_BYTES);
  if (budget > 0) {
    const int64_t per_block = (int64_t)tpb * per_thread_systems * N * (int64_t)spill_elem;
    int64_t cap = per_block > 0 ? budget / per_block : grid;
    if (cap < d.sms) cap = d.sms;
    if (grid > cap) grid = cap;
  }
  if (grid > blocks_needed) grid = blocks_needed;
  if (grid < 1) grid = 1;
  sh.grid = (int)grid;
  return sh;
}

// Estimated time of an FP64 sweep launch, in units of one warp's share of
// the FP64 pipe, on its busiest SM.  CTAs go to SMs in turn and each takes
// groups of systems c, c + grid, ... of the persistent loop, so the busiest
// SM runs its ceil(grid / sms) CTAs for q = blocks / grid rounds and its
// share of the rem = blocks % grid remainder in one more.  A round with k
// warps on the SM costs max(k, kLone): below ~5.5 warps the FP64 pipe is no
// longer the bound and a round costs what a nearly lone warp's dependent
// chain takes (fitted to the penta N = 512, M = 65536 solve, the 4096-line
// ADI half-step and the partitioned tri N = 4096, M = 4096 solve at 32, 64
// and 128 threads: the short second rounds of a grid that holds only part of
// the batch were 9-20 % slower, one round with 7 warps per SM instead of
// 3-4 CTAs of 4 was 5-8 % faster).
static double fp64_round_cost(const LaunchShape& sh, int64_t threads_needed, int sms) {
  constexpr double kLone = 5.5;
  const int64_t blocks = (threads_needed + sh.threads - 1) / sh.threads;
  const int64_t grid = sh.grid;
  const double w = sh.threads / 32.0;
  const int64_t q = blocks / grid, rem = blocks % grid;
  auto round = [&](int64_t ctas) { return std::max((double)ctas * w, kLone); };
  double c = (double)q * round((grid + sms - 1) / sms);
  if (rem > 0) c += round((rem + sms - 1) / sms);
  return c;
}

LaunchShape sweep_shape(int bw, int N, int64_t threads_needed, size_t coef_elem, size_t spill_elem,
                        int per_thread_systems, size_t extra_smem_per_thread, size_t extra_smem_fixed, int tpb,
                        int extra_coef_arrays, bool balance) {
  const DeviceInfo& d = device_info();
  auto shape = [&](int t) {
    return shape_for(bw, N, threads_needed, coef_elem, spill_elem, per_thread_systems, extra_smem_per_thread,
                     extra_smem_fixed, t, extra_coef_arrays);
  };
  if (tpb > 0) return shape(tpb);
  if (option(BS_OPT_CTA_THREADS) > 0) return shape((int)std::min<int64_t>(option(BS_OPT_CTA_THREADS), 128));
  // Policy: 128 threads, halved while the batch would give fewer than two
  // CTAs per SM.  With `balance` (row-partitioned ADI half-steps), FP64 sweeps,
  // bound by the FP64 pipe, then take the CTA size whose rounds load the
  // busiest SM least (fp64_round_cost), if it is strictly better; the larger
  // CTA on a tie (4096^2 FP64 y-implicit half-step: 0.231 -> 0.215 ms).
  // Solves keep the plain policy: on the penta N = 512, M = 65536 batch
  // 32-thread CTAs made the FP64 solve 5 % faster alone, but they fill every
  // SM's shared memory, and a mixed-precision solve on another stream could
  // no longer run beside it (that step: 1.107 -> 1.235 ms); partitioned
  // solves (tri N = 4096, M = 4096: 0.145 -> 0.138 ms alone) share the
  // server's streams the same way.
  tpb = 128;
  while (tpb > 32 && threads_needed < (int64_t)2 * d.sms * tpb) tpb /= 2;
  LaunchShape best = shape(tpb);
  if (balance && coef_elem == 8 && spill_elem == 8) {
    double best_cost = fp64_round_cost(best, threads_needed, d.sms);
    for (int t = 128; t >= 32; t /= 2) {
      if (t == tpb) continue;
      const LaunchShape sh = shape(t);
      const double c = fp64_round_cost(sh, threads_needed, d.sms);
      if (c < best_cost * 0.97) {
        best = sh;
        best_cost = c;
      }
    }
  }
  return best;
}

int kernel_regs(const void* kernel) {
  cudaFuncAttributes a{};
  return cudaFuncGetAttributes(&a, kernel) == cudaSuccess ? a.numRegs : 0;
}

// Candidates: every multiple of 64 up to max_threads (any_size = false: only
// 64, 128 and 256) with staged records, 32 too without, or the CTA size
// BS_OPT_CTA_THREADS forces (32-thread CTAs that each stage the records were
// slower in every measured case).  CTAs per SM follow from shared memory (records
// once per CTA) and registers; a pass of the persistent grid costs its
// busiest SM's warps, at least 4 (below ~4 warps per SM the dependent chains,
// not issue, set the time); the cheapest shape wins, on a tie the CTA size
// nearest `prefer` (the larger of two as near).  Staged records are preferred
// whenever some CTA size fits them.
StagedShape staged_shape(int64_t groups, size_t rec_bytes, size_t per_thread, int regs, int max_threads,
                         bool any_size, int prefer) {
  const DeviceInfo& d = device_info();
  const size_t sm_bytes = 228 * 1024, limit = (size_t)(d.smem_optin > 0 ? d.smem_optin : 48 * 1024) - 1024;
  const int reg_alloc = regs > 0 ? (regs + 7) / 8 * 8 : 0;
  StagedShape best{0, 0, false, 1e300};
  const int forced = (int)option(BS_OPT_CTA_THREADS);
  for (int staged = 1; staged >= 0 && best.threads == 0; staged--) {
    for (int t = 32; t <= max_threads; t = (t < 64 ? 64 : t + 64)) {
      if (forced > 0 && t != forced) continue;
      if (!forced && staged && (t == 32 || (!any_size && t != 64 && t != 128 && t != 256))) continue;
      const size_t cta = (staged ? rec_bytes : 0) + (size_t)t * per_thread;
      if (cta > limit) continue;
      int c = (int)(sm_bytes / (cta + 1024));
      c = std::min(c, 2048 / t);
      if (reg_alloc > 0) c = std::min(c, 65536 / (reg_alloc * t));
      if (c < 1) continue;
      const int64_t blocks = (groups + t - 1) / t;
      const int64_t grid = std::min<int64_t>((int64_t)d.sms * c, blocks);
      const int64_t per_pass = grid * t;
      double cost = 0.0;
      for (int64_t done = 0; done < groups; done += per_pass) {
        const int64_t active = std::min<int64_t>(grid, (groups - done + t - 1) / t);
        const int64_t busy = (active + d.sms - 1) / d.sms;
        cost += std::max(busy * t / 32.0, 4.0);
      }
      const bool nearer = std::abs(t - prefer) < std::abs(best.threads - prefer) ||
                          (std::abs(t - prefer) == std::abs(best.threads - prefer) && t > best.threads);
      if (cost < best.cost - 1e-9 || (cost < best.cost + 1e-9 && nearer))
        best = StagedShape{(int)std::max<int64_t>(grid, 1), t, staged != 0, cost};
    }
  }
  return best;
}

bs_status part_correct(const PartPlan& pp, int N, void* X, bs_dtype t, bs_layout layout, int64_t M,
                       cudaStream_t st);
bool use_twisted(bs_handle h, int which, bs_layout layout, int64_t M);
cudaError_t sweep_twisted(bs_handle h, int which, const void* in, void* out, bs_dtype t, int64_t M,
                          cudaStream_t st);

// The two-ended sweep also beats a partition into two blocks (measured
// N = 400, 512: 1.1-1.3x); from four blocks on the partition is faster.
static bool take_twisted(bs_handle h, int which, bs_layout layout, int64_t M, bool part) {
  return use_twisted(h, which, layout, M) &&
         (!part || (h->part[which].P <= 2 && option(BS_OPT_PARTITION) != 2));
}

// Whether a solve of M systems runs row-partitioned: by default when the
// batch has fewer than 256 systems per SM (measured: 65536 systems of N = 512
// already keep every SM busy, 4096 lines of an ADI step do not).
bool use_partition(bs_handle h, int64_t M) {
  if (!h->has_part || h->periodic) return false;
  const int64_t o = option(BS_OPT_PARTITION);
  if (o == 1) return false;
  if (o == 2) return true;
  return M < (int64_t)device_info().sms * 256;
}

// One-thread-per-system interleaved solve of plan p (primal or adjoint) on
// the windowed or pair sweeps where they apply; returns false if neither
// applies (the caller runs the streaming kernels).
static bool fast_sweep(const SweepPlan& p, bool adjoint, int N, void* B, bs_dtype dtype, bs_layout layout,
                       int64_t M, cudaStream_t st, cudaError_t* e) {
  if (layout != BS_INTERLEAVED) return false;
  const bool win = option(BS_OPT_WINDOW) != 1;
  if (dtype == BS_F64 && df_eligible(p, layout)) {  // periodic plans too (no windows)
    // pairs: the two-sweep kernel unless windows are asked for (the pair
    // arithmetic is bound by instruction issue, and the windowed sweep's extra
    // backward steps cost more than the forward values' round trip through
    // memory: penta N = 512, M = 65536 0.256 - 0.31 ms against 0.19 ms)
    *e = (option(BS_OPT_WINDOW) == 2 && p.win_df > 0) ? sweep_win_df(p, adjoint, N, static_cast<double*>(B), M, st)
                                                       : sweep_df(p, adjoint, N, static_cast<double*>(B), M, st);
    return true;
  }
  if (p.periodic) return false;
  // (the scalar-eps sweeps of a uniform pentadiagonal matrix, on request,
  // run in the streaming kernels)
  const bool uni = p.uniform && p.bw == 2 && option(BS_OPT_UNIFORM) == 2;
  if (dtype == BS_F32 && win && !uni && p.win32 > 0 && p.rec32) {
    *e = sweep_win32<float>(p, adjoint, N, static_cast<const float*>(B), static_cast<float*>(B), M, st);
    return true;
  }
  return false;
}

static bs_status check_common(bs_handle h, const void* B, bs_layout layout, int64_t M, const char* fn) {
  if (!valid_handle(h)) return set_error(BS_EINVAL, std::string(fn) + ": unknown handle");
  if (!B) return set_error(BS_EINVAL, std::string(fn) + ": null data pointer");
  if (M < 1) return set_error(BS_EINVAL, std::string(fn) + ": M must be >= 1");
  if (layout != BS_INTERLEAVED && layout != BS_STRIDED)
    return set_error(BS_EINVAL, std::string(fn) + ": bad layout");
  if (M > INT64_MAX / 16 / h->N) return set_error(BS_EINVAL, std::string(fn) + ": N*M too large");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device)
    return set_error(BS_EINVAL, std::string(fn) + ": handle belongs to device " + std::to_string(h->device) +
                                    ", current device is " + std::to_string(dev));
  return BS_OK;
}

}  // namespace bs

using namespace bs;

extern "C" {

bs_status bs_set_option(int opt, int64_t value) {
  if (opt < 0 || opt >= BS_OPT_COUNT) return set_error(BS_EINVAL, "bs_set_option: unknown option");
  if (value < 0) return set_error(BS_EINVAL, "bs_set_option: negative value");
  if (opt == BS_OPT_CTA_THREADS && value != 0 && value != 32 && !(value % 64 == 0 && value <= 512))
    return set_error(BS_EINVAL, "bs_set_option: BS_OPT_CTA_THREADS must be 0, 32 or a multiple of 64 up to 512");
  if (opt == BS_OPT_F64_PAIRS && value > 3) return set_error(BS_EINVAL, "bs_set_option: BS_OPT_F64_PAIRS must be 0..3");
  if (opt == BS_OPT_WINDOW && value > 2) return set_error(BS_EINVAL, "bs_set_option: BS_OPT_WINDOW must be 0, 1 or 2");
  g_opt[opt] = value;
  return BS_OK;
}

bs_status bs_solve(bs_handle h, void* B, bs_dtype dtype, bs_layout layout, int64_t M, bs_stream stream) {
  bs_status s = check_common(h, B, layout, M, "bs_solve");
  if (s != BS_OK) return s;
  cudaError_t e;
  const int N = (int)h->N;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (dtype != BS_F64 && dtype != BS_F32)
    return set_error(BS_EINVAL, "bs_solve: dtype must be BS_F64 or BS_F32 (BF16 input: bs_solve_bf16)");
  const bool part = use_partition(h, M);
  if (take_twisted(h, 0, layout, M, part)) {
    e = sweep_twisted(h, 0, B, B, dtype, M, st);
    if (e != cudaSuccess) return cuda_error(e, "bs_solve launch");
    return BS_OK;
  }
  const SweepPlan& p = part ? h->part[0].blk : h->plan[0];
  const int L = part ? h->part[0].L : 0, P = part ? h->part[0].P : 1;
  if (!part && fast_sweep(p, false, N, B, dtype, layout, M, st, &e))
    ;
  else if (dtype == BS_F64)
    e = sweep_f64(p, false, N, B, B, layout, M, st, L, P);
  else
    e = sweep_f32(p, false, N, B, B, layout, M, st, L, P);
  if (e != cudaSuccess) return cuda_error(e, "bs_solve launch");
  if (part) return part_correct(h->part[0], N, B, dtype, layout, M, st);
  return BS_OK;
}

bs_status bs_solve_bf16(bs_handle h, const void* B, float* X, bs_layout layout, int64_t M, bs_stream stream) {
  bs_status s = check_common(h, B, layout, M, "bs_solve_bf16");
  if (s != BS_OK) return s;
  if (!X) return set_error(BS_EINVAL, "bs_solve_bf16: X is NULL");
  const char* b0 = static_cast<const char*>(B);
  const char* x0 = reinterpret_cast<const char*>(X);
  const size_t nm = (size_t)h->N * (size_t)M;
  if (b0 < x0 + nm * 4 && x0 < b0 + nm * 2) return set_error(BS_EINVAL, "bs_solve_bf16: B and X overlap");
  const bool part = use_partition(h, M);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (take_twisted(h, 0, layout, M, part)) {
    const cudaError_t e = sweep_twisted(h, 0, B, X, BS_BF16, M, st);
    if (e != cudaSuccess) return cuda_error(e, "bs_solve_bf16 launch");
    return BS_OK;
  }
  const SweepPlan& p = part ? h->part[0].blk : h->plan[0];
  cudaError_t e;
  if (!part && layout == BS_INTERLEAVED && !p.periodic && option(BS_OPT_WINDOW) != 1 && p.win32 > 0 && p.rec32 &&
      !(p.uniform && p.bw == 2 && option(BS_OPT_UNIFORM) == 2) &&
      M % 2 == 0 && reinterpret_cast<uintptr_t>(B) % 4 == 0 && reinterpret_cast<uintptr_t>(X) % 8 == 0)
    e = sweep_win32<__nv_bfloat16>(p, false, (int)h->N, static_cast<const __nv_bfloat16*>(B), X, M, st);
  else
    e = sweep_bf16(p, false, (int)h->N, B, X, layout, M, st, part ? h->part[0].L : 0, part ? h->part[0].P : 1);
  if (e != cudaSuccess) return cuda_error(e, "bs_solve_bf16 launch");
  if (part) return part_correct(h->part[0], (int)h->N, X, BS_F32, layout, M, st);
  return BS_OK;
}

bs_status bs_solve_adjoint(bs_handle h, void* G, bs_dtype dtype, bs_layout layout, int64_t M, const void* X,
                           double* dbands, bs_stream stream) {
  bs_status s = check_common(h, G, layout, M, "bs_solve_adjoint");
  if (s != BS_OK) return s;
  if ((X == nullptr) != (dbands == nullptr))
    return set_error(BS_EINVAL, "bs_solve_adjoint: X and dbands must both be given or both be NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  const int N = (int)h->N;
  if (dtype != BS_F64 && dtype != BS_F32) return set_error(BS_EINVAL, "bs_solve_adjoint: dtype must be BS_F64 or BS_F32");
  // partitioned: the primal-form plan of A^T's block-diagonal part
  const bool part = use_partition(h, M);
  if (take_twisted(h, 1, layout, M, part)) {
    e = sweep_twisted(h, 1, G, G, dtype, M, st);
    if (e != cudaSuccess) return cuda_error(e, "bs_solve_adjoint launch");
    if (X) return launch_band_grad(h, G, X, dtype, layout, M, dbands, st);
    return BS_OK;
  }
  const SweepPlan& p = part ? h->part[1].blk : h->plan[1];
  const int L = part ? h->part[1].L : 0, P = part ? h->part[1].P : 1;
  if (!part && fast_sweep(p, true, N, G, dtype, layout, M, st, &e))
    ;
  else if (dtype == BS_F64)
    e = sweep_f64(p, !part, N, G, G, layout, M, st, L, P);
  else
    e = sweep_f32(p, !part, N, G, G, layout, M, st, L, P);
  if (e != cudaSuccess) return cuda_error(e, "bs_solve_adjoint launch");
  if (part) {
    const bs_status ps = part_correct(h->part[1], N, G, dtype, layout, M, st);
    if (ps != BS_OK) return ps;
  }
  if (X) return launch_band_grad(h, G, X, dtype, layout, M, dbands, st);
  return BS_OK;
}

bs_status bs_band_grad(bs_handle h, const void* GB, const void* X, bs_dtype dtype, bs_layout layout, int64_t M,
                       double* dbands, bs_stream stream) {
  bs_status s = check_common(h, GB, layout, M, "bs_band_grad");
  if (s != BS_OK) return s;
  if (!X || !dbands) return set_error(BS_EINVAL, "bs_band_grad: X and dbands must be non-NULL");
  if (dtype != BS_F64 && dtype != BS_F32) return set_error(BS_EINVAL, "bs_band_grad: dtype must be BS_F64 or BS_F32");
  return launch_band_grad(h, GB, X, dtype, layout, M, dbands, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
