// Band-gradient reduction over the batch.
//
// For a scalar loss L with dL/dX given, X = A^{-1} B and GB = A^{-T} dL/dX,
// dL/dA = -GB X^T; the entries on the bands are
//   dbands[k*N + i] = -sum_j GB[i, j] * X[i + k - h, j],   h = width / 2.
// Two levels, fixed order, no atomics:
//   1. the work space (groups of kGradGroups row blocks of kGradRows rows) x
//      (systems), taken in group-major order, is cut into G equal contiguous
//      ranges, one per CTA of a grid that fills the device exactly once (G =
//      SMs x resident CTAs per SM, so no partial last wave).  A CTA walks its
//      range as at most a few segments (one per block group it touches); for
//      each segment the CTA's thread group g strides over the systems
//      accumulating the products of the group's row block g in FP64, a warp
//      reduce-scatter (shuffles) and a shared-memory pass across the group's
//      warps combine them, and one partial per (CTA, segment, row block,
//      band, row) goes to scratch;
//   2. one thread per (band, row) adds the partials of the CTAs that touched
//      its row block, in CTA order.
// The decomposition is a function of N, M and G only, so the result is
// bitwise reproducible on a given device.  16 bytes of compulsory reads per
// unknown (GB and X); the X halo of 2h rows per row block is shared with the
// neighbouring blocks of the group, which the same CTA sweeps at the same
// time.
//
// Arithmetic of level 1.  FP64 data: one FP64 FMA per product except for
// the products of the top X rows of a thread's window, which are summed in
// FP32 pairs (see kGradSplit5; the kernel is bound by the FP64 pipe).  FP32
// data: a thread's products for one (band, row) are summed in FP32 pairs
// over runs of kGradRun systems -- each product exact by an FMA-based
// TwoProduct, added with Knuth's TwoSum, the rounding errors collected in
// the low part -- and each run's pair is added, exactly widened, to an FP64
// sum: `width` products in FP32 arithmetic per unknown
// instead of `width` FP64 FMAs (the FP64 pipe of GB300 runs at 1/64 of the
// FP32 rate) and width / kGradRun FP64 additions.  A run of K products of
// typical size t carries an error of about sqrt(K) 2^-48 t, so a sum of M
// random-sign terms, of size sqrt(M) t, is off by about sqrt(K) 2^-48
// relative (K = 32: ~2e-14).  Values outside [2^-32, 2^48) (besides zero)
// could overflow or underflow the FP32 parts: a CTA that meets one in a
// segment recomputes that segment with FP64 FMAs, so the result depends only
// on the data.  (The same pairs for all products of FP64 data, each value
// split into two FP32 parts, measured slower than the FP64 FMAs: the splits
// cost about 20 integer instructions per value; penta N = 512, M = 65536:
// 0.33 - 0.48 ms against 0.32 ms.  So did a layout for interleaved data in which a warp
// reads one row of 32 systems and sums each row's products over its lanes
// with shuffles, in pairs: 0.44 ms (FP32 data 0.37 ms) -- the per-row
// butterfly costs ~250 warp instructions per 32 unknowns.)
#include <climits>
#include <mutex>
#include <string>

#include "df_math.cuh"
#include "refine_math.cuh"
#include "sweep_kernels.cuh"

namespace bs {

constexpr int kGradThreads = 256;
// Rows per block: 3 keeps a thread's accumulators and two register sets of
// rows small enough (<= 120 registers) for two 256-thread CTAs per SM, whose
// warps keep the FP64 pipe busier than one CTA of 8-row blocks (202
// registers): penta N = 512, M = 65536: 0.321 against 0.356 ms (4 rows:
// 0.327, 2 rows: 0.326).
constexpr int kGradRows = 3;
// Row blocks a CTA sweeps side by side: its threads form kGradGroups groups,
// group g taking row block kGradGroups * rg + g of the same systems, so that
// the X rows two neighbouring blocks share are loaded by two groups of one SM
// at about the same time (the second load hits L1) instead of by two CTAs at
// unrelated times (both from DRAM).
constexpr int kGradGroups = 4;
constexpr int kGradGroupThreads = kGradThreads / kGradGroups;
static_assert(kGradGroupThreads % 32 == 0, "a group is whole warps");

struct GradShape {
  int R;      // row blocks
  int RG;     // groups of kGradGroups row blocks
  int G;      // CTAs
  int S;      // most segments (block groups) one CTA can touch
  int64_t M;  // systems
};

// CTA c owns the positions [range_lo(c), range_lo(c + 1)) of the RG*M work
// space (position p = block group p / M, system p % M).
__host__ __device__ __forceinline__ int64_t range_lo(int64_t c, int64_t total, int64_t G) { return c * total / G; }

static int grad_ctas_per_sm();

GradShape grad_shape(int N, int64_t M) {
  GradShape g{};
  g.R = (N + kGradRows - 1) / kGradRows;
  g.RG = (g.R + kGradGroups - 1) / kGradGroups;
  g.M = M;
  g.G = device_info().sms * grad_ctas_per_sm();
  const int64_t total = (int64_t)g.RG * M;
  // a range of ceil(total / G) positions touches at most this many block groups
  const int64_t per = (total + g.G - 1) / g.G;
  g.S = (int)((per + M - 1) / M) + 1;
  if (g.S > g.RG) g.S = g.RG;
  return g;
}

size_t band_grad_scratch_bytes(int width, int N, int64_t M) {
  const GradShape g = grad_shape(N, M);
  return (size_t)g.G * g.S * kGradGroups * width * kGradRows * sizeof(double);
}

template <typename T>
__device__ __forceinline__ double to_wide(T v) {
  if constexpr (sizeof(T) == 8)
    return v;
  else
    return widen_exact(v);  // integer-only widening: keeps the FP64 pipe for the FMAs
}

// Products per (band, row) summed in pairs before one FP64 addition (FP32
// data; the pair bands of FP64 data).  Measured against runs of 16 (ms,
// penta N = 512, M = 65536): FP64 data 0.2443 against 0.2517, FP32 data
// 0.1898 against 0.2022 (fewer FP64 additions; results within 1.4e-14).
constexpr int kGradRun = 32;

// v is zero or 2^-32 <= |v| < 2^48 (the pair arithmetic's range here: the
// products stay within [2^-64, 2^96) and a run's sums far from overflow)
__device__ __forceinline__ bool grad_in_range(float v) {
  const uint32_t b = __float_as_uint(v) & 0x7fffffffu;
  return b - ((127u - 32u) << 23) < (80u << 23) || b == 0u;
}

// FP64 data: zero or 2^-32 <= |v| < 2^48, and v as a pair (|v - (h + l)| <=
// 2^-48 |v|)
__device__ __forceinline__ bool grad_in_range(double v) {
  const uint32_t hw = df::hiword(v) & 0x7fffffffu;
  return hw - ((1023u - 32u) << 20) < (80u << 20) || (hw | df::loword(v)) == 0u;
}
__device__ __forceinline__ df::Pair grad_pair(double v) {
  df::Pair y;
  if (!df::split_fast(v, y)) y = df::Pair{0.f, 0.f};  // in range: zero
  return y;
}

// FP64 data: the products g[r] x[r + k] whose X row lies at or above index
// kGradSplit of the thread's window of NX rows (r + k >= kGradSplit) are
// summed in FP32 pairs as for FP32 data -- each value they need split once,
// the product a TwoProduct plus the two cross terms -- and the others with
// FP64 FMAs, so that the FP32 and integer pipes take part of the work the
// FP64 pipe bounds; the X rows below the split are never converted.  The
// FP64 sums of the pair products' runs live in shared memory (one column per
// thread), which leaves the registers to the loads in flight.  Measured
// (penta N = 512, M = 65536, ms): all products in FP64 0.321; the top pair
// bands (k >= 5 - n) with the run sums in registers n = 1: 0.281, 2: 0.295,
// 3: 0.329; in shared memory 1: 0.278, 2: 0.258, 3: 0.298 (with the
// row-block groups and runs of 32: 2: 0.2415, 3: 0.288); by split row,
// kGradSplit = 4 (6 pair products, 6 values split): 0.2375, 3 (9, 7):
// 0.260, 2 (12, 8): 0.279 -- beyond six products the splits and the spilled
// registers cost more issue slots than the FP64 FMAs they replace (so did one
// warp in four or eight taking all products in pairs: 0.326 / 0.298 against
// 0.244 ms).  Tri N = 1024, M = 2^18: all FP64 1.435 ms, the top band in pairs
// 1.228, then 1.280 with the groups; kGradSplit = 3 (3 products, 5 values):
// 1.227, 2 (6, 6): 1.280.
constexpr bool kGradPairSmem = true;
constexpr int kGradSplit5 = 4;
constexpr int kGradSplit3 = 3;

// Position of the pair product (r, k), r + k >= S, among all of them in (k,
// r) order; their count for (r, k) = (-1, -1).
template <int W, int S>
__host__ __device__ constexpr int pair_slot(int r, int k) {
  int n = 0;
  for (int kk = 0; kk < W; kk++)
    for (int rr = 0; rr < kGradRows; rr++)
      if (rr + kk >= S) {
        if (rr == r && kk == k) return n;
        n++;
      }
  return n;
}

// a += g * x for pairs of FP64 values, not renormalised
__device__ __forceinline__ void grad_acc(df::Pair& a, df::Pair g, df::Pair x) {
  const float p = df::mul(g.h, x.h);
  float e = df::fma_(g.h, x.h, -p);
  e = df::fma_(g.h, x.l, e);
  e = df::fma_(g.l, x.h, e);
  float s, t;
  df::two_sum(a.h, p, s, t);
  a.h = s;
  a.l = df::add(a.l, df::add(t, e));
}

// a += g * x in pairs, not renormalised: a.h the running FP32 sum, a.l the
// rounding errors of its additions (the product g * x = p + e is exact)
__device__ __forceinline__ void grad_acc(df::Pair& a, float g, float x) {
  const float p = df::mul(g, x);
  const float e = df::fma_(g, x, -p);
  float s, t;
  df::two_sum(a.h, p, s, t);
  a.h = s;
  a.l = df::add(a.l, df::add(t, e));
}

// Level 1.  partial layout: [CTA][segment][group][band][row in block].
// PER: periodic matrix, X rows taken modulo N.
template <typename T, int W, bool PER>
__global__ void __launch_bounds__(kGradThreads, 2)
k_band_grad_partial(int N, int64_t M, int R, int RG, int S, const T* __restrict__ GB, const T* __restrict__ X,
                    int64_t rs, int64_t ss, double* __restrict__ partial) {
  constexpr int H = W / 2;
  constexpr int NX = kGradRows + 2 * H;
  constexpr int NV = kGradRows * W;  // accumulators per thread
  static_assert(NV <= 64, "reduce-scatter holds at most 64 values per lane");
  __shared__ double red[kGradThreads / 32][64];
  constexpr int SP = (sizeof(T) == 8) ? (W == 5 ? kGradSplit5 : kGradSplit3) : NX;
  constexpr int NP = pair_slot<W, SP>(-1, -1);  // pair products (FP64 data)
  constexpr int KPS = (kGradPairSmem && NP > 0) ? NP : 1;
  __shared__ double psum[KPS][kGradThreads];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = threadIdx.x / kGradGroupThreads, tg = threadIdx.x % kGradGroupThreads;
  const int64_t total = (int64_t)RG * M;
  const int64_t lo = range_lo(blockIdx.x, total, gridDim.x);
  const int64_t hi = range_lo(blockIdx.x + 1, total, gridDim.x);
  const int rg0 = (int)(lo / M);
  for (int64_t p = lo; p < hi;) {
    const int rg = (int)(p / M);
    const int64_t seg_end = hi < (int64_t)(rg + 1) * M ? hi : (int64_t)(rg + 1) * M;
    const int rb = rg * kGradGroups + grp;
    // a group past the last row block has no systems (its partials are not read)
    const int64_t jlo = p - (int64_t)rg * M, jhi = rb < R ? seg_end - (int64_t)rg * M : jlo;
    const int i0 = rb * kGradRows;
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) acc[v] = 0.0;
    // rows i0 - H .. i0 + kGradRows - 1 + H of X and i0 .. of GB for system
    // j; the next system's rows are requested before the current ones are
    // used (two register sets), so each thread keeps one load batch in flight
    // while its arithmetic runs
    auto fetch = [&](int64_t j, T (&x)[NX], T (&g)[kGradRows]) {
#pragma unroll
      for (int q = 0; q < NX; q++) {
        const int row = i0 - H + q;
        if constexpr (PER) {
          const int pr = ((row % N) + N) % N;
          x[q] = X[pr * rs + j * ss];
        } else {
          x[q] = (row >= 0 && row < N) ? X[row * rs + j * ss] : T(0);
        }
      }
#pragma unroll
      for (int r = 0; r < kGradRows; r++) {
        const int row = i0 + r;
        g[r] = (row < N) ? GB[row * rs + j * ss] : T(0);
      }
    };
    // the segment's systems in the order fetch / use, over both register sets
    auto sweep = [&](auto use) {
      T xa[NX], ga[kGradRows], xb[NX], gb[kGradRows];
      int64_t j = jlo + tg;
      if (j < jhi) fetch(j, xa, ga);
      for (; j < jhi; j += 2 * kGradGroupThreads) {
        const int64_t j1 = j + kGradGroupThreads;
        if (j1 < jhi) fetch(j1, xb, gb);
        use(xa, ga);
        if (j1 >= jhi) break;
        if (j1 + kGradGroupThreads < jhi) fetch(j1 + kGradGroupThreads, xa, ga);
        use(xb, gb);
      }
    };
    auto fp64 = [&]() {
#pragma unroll
      for (int v = 0; v < NV; v++) acc[v] = 0.0;
      sweep([&](const T (&x)[NX], const T (&g)[kGradRows]) {
#pragma unroll
        for (int r = 0; r < kGradRows; r++)
#pragma unroll
          for (int k = 0; k < W; k++)
            acc[k * kGradRows + r] = fma(to_wide(g[r]), to_wide(x[r + k]), acc[k * kGradRows + r]);
      });
    };
    if constexpr (sizeof(T) == 8 && NP == 0) {
      fp64();
    } else if constexpr (sizeof(T) == 8) {
      // products with r + k < SP with FP64 FMAs, the others in pairs (runs
      // of kGradRun systems, then FP64 sums of the runs)
      bool bad = false;
      df::Pair pa[NP];
#pragma unroll
      for (int v = 0; v < NP; v++) pa[v] = df::Pair{0.f, 0.f};
#pragma unroll
      for (int v = 0; v < NV; v++) acc[v] = 0.0;
      if constexpr (kGradPairSmem) {
#pragma unroll
        for (int v = 0; v < NP; v++) psum[v][threadIdx.x] = 0.0;
      }
      int run = 0;
      auto flush = [&]() {
#pragma unroll
        for (int k = 0; k < W; k++)
#pragma unroll
          for (int r = 0; r < kGradRows; r++)
            if (r + k >= SP) {
              const int v = pair_slot<W, SP>(r, k);
              if constexpr (kGradPairSmem)
                psum[v][threadIdx.x] += widen_exact(pa[v].h) + widen_exact(pa[v].l);
              else
                acc[k * kGradRows + r] += widen_exact(pa[v].h) + widen_exact(pa[v].l);
              pa[v] = df::Pair{0.f, 0.f};
            }
      };
      sweep([&](const T (&x)[NX], const T (&g)[kGradRows]) {
#pragma unroll
        for (int r = 0; r < kGradRows; r++)
#pragma unroll
          for (int k = 0; k < W; k++)
            if (r + k < SP) acc[k * kGradRows + r] = fma(g[r], x[r + k], acc[k * kGradRows + r]);
        df::Pair gp[kGradRows], xp[NX];
        bool in = true;
#pragma unroll
        for (int r = 0; r < kGradRows; r++) {
          in &= grad_in_range(g[r]);
          gp[r] = grad_pair(g[r]);
        }
#pragma unroll
        for (int q = SP; q < NX; q++) {
          in &= grad_in_range(x[q]);
          xp[q] = grad_pair(x[q]);
        }
        bad |= !in;
#pragma unroll
        for (int r = 0; r < kGradRows; r++)
#pragma unroll
          for (int k = 0; k < W; k++)
            if (r + k >= SP) grad_acc(pa[pair_slot<W, SP>(r, k)], gp[r], xp[r + k]);
        if (++run == kGradRun) {
          flush();
          run = 0;
        }
      });
      flush();
      if constexpr (kGradPairSmem) {
#pragma unroll
        for (int k = 0; k < W; k++)
#pragma unroll
          for (int r = 0; r < kGradRows; r++)
            if (r + k >= SP) acc[k * kGradRows + r] = psum[pair_slot<W, SP>(r, k)][threadIdx.x];
      }
      // a value outside the pairs' range anywhere in the segment: FP64 FMAs
      if (__syncthreads_or(bad)) fp64();
    } else {
      // pairs, runs of kGradRun systems
      bool bad = false;
      df::Pair pa[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) pa[v] = df::Pair{0.f, 0.f};
      int run = 0;
      auto flush = [&]() {
#pragma unroll
        for (int v = 0; v < NV; v++) {
          acc[v] += widen_exact(pa[v].h) + widen_exact(pa[v].l);
          pa[v] = df::Pair{0.f, 0.f};
        }
      };
      sweep([&](const T (&x)[NX], const T (&g)[kGradRows]) {
        bool in = true;
#pragma unroll
        for (int q = 0; q < NX; q++) in &= grad_in_range(x[q]);
#pragma unroll
        for (int r = 0; r < kGradRows; r++) in &= grad_in_range(g[r]);
        bad |= !in;
#pragma unroll
        for (int r = 0; r < kGradRows; r++)
#pragma unroll
          for (int k = 0; k < W; k++) grad_acc(pa[k * kGradRows + r], g[r], x[r + k]);
        if (++run == kGradRun) {
          flush();
          run = 0;
        }
      });
      flush();
      // a value outside the pairs' range anywhere in the segment: FP64 FMAs
      if (__syncthreads_or(bad)) fp64();
    }
    // Warp reduce-scatter over the NV values: at each level a lane keeps one
    // half, sends the other to its partner and adds what it receives.  Up to
    // 16 values (every use here): four halvings leave lane l with value
    // l / 2 summed over 16 lanes, and a last exchange with lane l ^ 1 makes
    // it the warp sum -- 16 FP64 additions per lane (63 when padded to 64).
    if constexpr (NV <= 16) {
      double w16[16];
#pragma unroll
      for (int i = 0; i < 16; i++) w16[i] = (i < NV) ? acc[i < NV ? i : 0] : 0.0;
#pragma unroll
      for (int o = 16, n = 8; o >= 2; o >>= 1, n >>= 1) {
#pragma unroll
        for (int i = 0; i < n; i++) {
          const bool up = lane & o;
          const double keep = up ? w16[i + n] : w16[i], send = up ? w16[i] : w16[i + n];
          w16[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      w16[0] += __shfl_xor_sync(0xffffffffu, w16[0], 1);
      if ((lane & 1) == 0) red[warp][lane >> 1] = w16[0];
    } else {  // padded to 64: lane l ends with the warp sums of values 2l, 2l + 1
      double w32[32];
#pragma unroll
      for (int i = 0; i < 32; i++) {
        const double a = (i < NV) ? acc[i < NV ? i : 0] : 0.0;
        const double b = (i + 32 < NV) ? acc[i + 32 < NV ? i + 32 : 0] : 0.0;
        const bool up = lane & 16;
        const double keep = up ? b : a, send = up ? a : b;
        w32[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
      }
#pragma unroll
      for (int o = 8, n = 16; o >= 1; o >>= 1, n >>= 1) {
#pragma unroll
        for (int i = 0; i < n; i++) {
          const bool up = lane & o;
          const double keep = up ? w32[i + n] : w32[i], send = up ? w32[i] : w32[i + n];
          w32[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      red[warp][2 * lane] = w32[0];
      red[warp][2 * lane + 1] = w32[1];
    }
    __syncthreads();
    if (threadIdx.x < NV * kGradGroups) {
      constexpr int WG = kGradGroupThreads / 32;  // warps per group
      const int g = threadIdx.x / NV, v = threadIdx.x % NV;
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < WG; w++) t += red[g * WG + w][v];
      partial[(((int64_t)blockIdx.x * S + (rg - rg0)) * kGradGroups + g) * NV + v] = t;
    }
    __syncthreads();
    p = seg_end;
  }
}

// Level 2: dbands[k*N + i] = -(sum of the partials of the CTAs that touched
// row block i / kGradRows); 0 outside the matrix (a periodic matrix has no
// entries outside).  One warp per (band, row): lane l takes the CTAs c0 + l,
// c0 + l + 32, .. in that order, and the lanes' sums are added in a fixed
// butterfly order (lane 0's result is stored), so the result stays bitwise
// reproducible.
__global__ void k_band_grad_finish(int W, int N, int64_t M, int RG, int G, int S, int periodic,
                                   const double* __restrict__ partial, double* __restrict__ dbands) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= (int64_t)W * N) return;  // whole warps
  const int k = (int)(t / N), i = (int)(t % N);
  const int rb = i / kGradRows, r = i % kGradRows;
  const int rg = rb / kGradGroups, grp = rb % kGradGroups;
  const int col = i + k - W / 2;
  const int64_t total = (int64_t)RG * M;
  const int64_t b_lo = (int64_t)rg * M, b_hi = b_lo + M;
  // the CTA whose range [c total / G, (c + 1) total / G) holds position p is
  // floor(((p + 1) G - 1) / total) (the last of equal starts: empty ranges hold none)
  const int64_t c0 = ((b_lo + 1) * G - 1) / total, c1 = (b_hi * G - 1) / total;
  double s = 0.0;
  for (int64_t c = c0 + lane; c <= c1; c += 32) {
    const int64_t lo = range_lo(c, total, G), hi = range_lo(c + 1, total, G);
    if (hi > lo) {  // a CTA starting inside the group has it as its first segment
      const int seg = lo >= b_lo ? 0 : rg - (int)(lo / M);
      s += partial[((c * S + seg) * kGradGroups + grp) * (int64_t)(W * kGradRows) + k * kGradRows + r];
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) dbands[t] = (periodic || (col >= 0 && col < N)) ? -s : 0.0;
}

template <typename T, int W, bool PER>
static int ctas_per_sm_of() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_band_grad_partial<T, W, PER>, kGradThreads, 0) !=
          cudaSuccess ||
      n < 1)
    n = 1;
  return n;
}

// Resident CTAs per SM of the partial kernel (the smallest over its
// instantiations, so that every variant uses the same decomposition).
static int grad_ctas_per_sm() {
  static std::mutex mu;
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  std::lock_guard<std::mutex> lk(mu);
  if (!cached[dev]) {
    int n = ctas_per_sm_of<double, 5, false>();
    const int m[] = {ctas_per_sm_of<double, 3, false>(), ctas_per_sm_of<double, 3, true>(),
                     ctas_per_sm_of<float, 5, false>(), ctas_per_sm_of<float, 3, false>(),
                     ctas_per_sm_of<float, 3, true>()};
    for (int v : m) n = v < n ? v : n;
    cached[dev] = n;
  }
  return cached[dev];
}

// Both levels with caller-provided scratch of band_grad_scratch_bytes().
cudaError_t band_grad_with_scratch(int width, int N, bool periodic, const void* GB, const void* X, bs_dtype t,
                                   bs_layout layout, int64_t M, double* dbands, double* scratch, cudaStream_t st) {
  const int64_t rs = layout == BS_INTERLEAVED ? M : 1;
  const int64_t ss = layout == BS_INTERLEAVED ? 1 : N;
  const GradShape g = grad_shape(N, M);
#define BS_GRAD(TT, WW, PP)                                                                         \
  k_band_grad_partial<TT, WW, PP><<<g.G, kGradThreads, 0, st>>>(N, M, g.R, g.RG, g.S, (const TT*)GB,       \
                                                                (const TT*)X, rs, ss, scratch)
  if (periodic) {  // width 3 only
    if (t == BS_F64)
      BS_GRAD(double, 3, true);
    else
      BS_GRAD(float, 3, true);
  } else if (t == BS_F64) {
    if (width == 3)
      BS_GRAD(double, 3, false);
    else
      BS_GRAD(double, 5, false);
  } else {
    if (width == 3)
      BS_GRAD(float, 3, false);
    else
      BS_GRAD(float, 5, false);
  }
#undef BS_GRAD
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t n = (int64_t)width * N * 32;  // one warp per output
  k_band_grad_finish<<<(int)((n + 255) / 256), 256, 0, st>>>(width, N, M, g.RG, g.G, g.S, periodic ? 1 : 0,
                                                             scratch, dbands);
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
// the first call for that device (the device must be current).  *first: the
// lookup is still to be done (the caller refuses that during stream capture).
static cudaError_t noalloc_scratch(double** out, cudaStream_t st, bool* capturing) {
  static std::mutex mu;
  static double* ptr[64] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  *capturing = false;
  if (!ptr[dev]) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone) {
      *capturing = true;
      return cudaSuccess;
    }
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
  if (M > INT64_MAX / 16 / h->N) return set_error(BS_EINVAL, "bs_band_grad_noalloc: N*M too large");
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
  bool capturing = false;
  cudaError_t e = noalloc_scratch(&scratch, reinterpret_cast<cudaStream_t>(stream), &capturing);
  if (e != cudaSuccess) return cuda_error(e, "bs_band_grad_noalloc: scratch address");
  if (capturing)
    return set_error(BS_EINVAL, "bs_band_grad_noalloc: the first call on a device looks up the array's address "
                                "and must not be made while its stream is being captured");
  e = band_grad_with_scratch(h->width, N, h->periodic, GB, X, dtype, layout, M, dbands, scratch,
                             reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_error(e, "bs_band_grad_noalloc launch");
  return BS_OK;
}

