// Two-ended ("twisted") tridiagonal solves for small batches.
//
// With one thread per system (Sec. 2) a batch too small to fill the GPU takes
// as long as one system's chain of 2N dependent steps (forward, then
// backward).  On GB300 a warp-wide FP64 instruction costs the same whatever
// the number of active lanes, so that time does not shrink with the batch:
// N = 64 takes ~14 us for 1 system as for 9728.  Here two threads share a
// system and the chain halves.  The even lane eliminates rows 0 .. k-1
// top-down with the factorisation A = L U of Sec. 3.1 (w_i = s_i f_i -
// l1_i w_{i-1}); the odd lane eliminates rows N-1 .. k+1 bottom-up with the
// factorisation of the row-reversed matrix, A = U' L' (z_i = s'_i f_i -
// l1'_i z_{i+1}).  At row k = N / 2 the two meet:
//   x_k = (f_k - a_k w_{k-1} - c_k z_{k+1}) / g_k,
//   g_k = b_k - a_k chat_{k-1} - c_k chat'_{k+1},
// (row k of A with x_{k-1} = w_{k-1} - chat_{k-1} x_k and x_{k+1} = z_{k+1} -
// chat'_{k+1} x_k substituted), and each lane back-substitutes its half
// outward: x_i = w_i - chat_i x_{i+1} above, x_i = z_i - chat'_i x_{i-1}
// below.  N + 1 dependent steps instead of 2N, the same FP64 operations per
// row as the one-thread sweeps.
#include "sweep_kernels.cuh"

namespace bs {

constexpr int kTwThreads = 64;

template <typename C>
struct TwistArgs {
  const C* s[2];   // [0] top half: plan of A = L U; [1] bottom half: plan of A = U' L'
  const C* l1[2];  // (each indexed by matrix row)
  const C* u1[2];
  int k;           // meeting row
  C a, c, g;       // a_k, c_k and 1 / g_k
};

// Even lane (h = 0): rows 0, 1, .., k-1 forward, then k-1, .., 0 backward.
// Odd lane (h = 1): rows N-1, .., k+1 forward, then k+1, .., N-1 backward.
template <typename C, int U>
__global__ void __launch_bounds__(kTwThreads)
k_sweep_tw(TwistArgs<C> ta, int N, const C* in, C* out, int64_t M) {  // in == out allowed
  const int h = threadIdx.x & 1;
  const int k = ta.k;
  const int n = h ? N - 1 - k : k;       // rows this lane eliminates
  const int r0 = h ? N - 1 : 0;          // its first row
  const int dr = h ? -1 : 1;             // row step of its forward sweep
  const C* __restrict__ S = h ? ta.s[1] : ta.s[0];  // selects, not a dynamic index into the parameters
  const C* __restrict__ L1 = h ? ta.l1[1] : ta.l1[0];
  const C* __restrict__ U1 = h ? ta.u1[1] : ta.u1[0];
  const int64_t pairs = ((int64_t)gridDim.x * blockDim.x) >> 1;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 1; j < M; j += pairs) {
    const int64_t dp = h ? -M : M;       // pointer step of the forward sweep
    // forward sweep over this lane's n rows, U rows per block, the next
    // block's inputs requested before the current block is computed
    C w = C(0);
    {
      const C* pin = in + (int64_t)r0 * M + j;
      C* pout = out + (int64_t)r0 * M + j;
      C fa[U], fb[U];
      auto load = [&](C (&f)[U], int q0) {
#pragma unroll
        for (int u = 0; u < U; u++)
          if (q0 + u < n) f[u] = pin[(int64_t)(q0 + u) * dp];
      };
      auto run = [&](C (&f)[U], int q0) {
        C sv[U], lv[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int i = r0 + dr * (q0 + u < n ? q0 + u : q0);
          sv[u] = __ldg(S + i);
          lv[u] = __ldg(L1 + i);
        }
#pragma unroll
        for (int u = 0; u < U; u++)
          if (q0 + u < n) {
            w = fma(-lv[u], w, f[u] * sv[u]);
            pout[(int64_t)(q0 + u) * dp] = w;
          }
      };
      if (n > 0) load(fa, 0);
      for (int q0 = 0; q0 < n; q0 += 2 * U) {
        if (q0 + U < n) load(fb, q0 + U);
        run(fa, q0);
        if (q0 + U >= n) break;
        if (q0 + 2 * U < n) load(fa, q0 + 2 * U);
        run(fb, q0 + U);
      }
    }
    // meeting row, read and written by the even lane only: it receives
    // z_{k+1} (0 when k = N - 1) from the odd lane and hands x_k back.  The
    // shuffles name exactly the two lanes of the pair, whose loops above may
    // have run different trip counts.
    const unsigned pair = 3u << ((threadIdx.x & 31) & ~1u);
    const C zk = __shfl_xor_sync(pair, w, 1);
    C x = C(0);
    if (!h) {
      x = fma(-ta.c, zk, fma(-ta.a, w, in[(int64_t)k * M + j])) * ta.g;
      out[(int64_t)k * M + j] = x;
    }
    const C xe = __shfl_xor_sync(pair, x, 1);
    if (h) x = xe;
    // backward sweep outward from row k over the same n rows
    {
      const int rb = k - dr;  // first row: k - 1 (even) or k + 1 (odd)
      C* pb = out + (int64_t)rb * M + j;
      C fa[U], fb[U];
      auto load = [&](C (&f)[U], int q0) {
#pragma unroll
        for (int u = 0; u < U; u++)
          if (q0 + u < n) f[u] = pb[-(int64_t)(q0 + u) * dp];
      };
      auto run = [&](C (&f)[U], int q0) {
        C uv[U];
#pragma unroll
        for (int u = 0; u < U; u++) uv[u] = __ldg(U1 + rb - dr * (q0 + u < n ? q0 + u : q0));
#pragma unroll
        for (int u = 0; u < U; u++)
          if (q0 + u < n) {
            x = fma(-uv[u], x, f[u]);
            pb[-(int64_t)(q0 + u) * dp] = x;
          }
      };
      if (n > 0) load(fa, 0);
      for (int q0 = 0; q0 < n; q0 += 2 * U) {
        if (q0 + U < n) load(fb, q0 + U);
        run(fa, q0);
        if (q0 + U >= n) break;
        if (q0 + 2 * U < n) load(fa, q0 + 2 * U);
        run(fb, q0 + U);
      }
    }
  }
}

template <typename C>
static cudaError_t launch_tw(const TwistPlan& tp, int N, const C* in, C* out, int64_t M, cudaStream_t st) {
  TwistArgs<C> ta{};
  for (int q = 0; q < 2; q++) {
    const SweepPlan& p = q == 0 ? *tp.top : *tp.bot;
    const C* base;
    if constexpr (sizeof(C) == 8)
      base = reinterpret_cast<const C*>(p.c64);
    else
      base = reinterpret_cast<const C*>(p.c32);
    const Coefs<C> cf = coefs_of<C>(base, N);
    ta.s[q] = cf.s;
    ta.l1[q] = cf.l1;
    ta.u1[q] = cf.u1;
  }
  ta.k = tp.k;
  ta.a = (C)tp.a;
  ta.c = (C)tp.c;
  ta.g = (C)tp.g;
  const int64_t threads = 2 * M;
  int64_t grid = (threads + kTwThreads - 1) / kTwThreads;
  const int64_t cap = (int64_t)device_info().sms * (2048 / kTwThreads);
  if (grid > cap) grid = cap;
  k_sweep_tw<C, 8><<<(int)grid, kTwThreads, 0, st>>>(ta, N, in, out, M);
  return cudaGetLastError();
}

// Whether a solve with A (which = 0) or A^T (which = 1) takes the two-ended
// sweep: tridiagonal, not periodic, the handle has a meeting row for that
// matrix, interleaved layout, and at most 128 systems per SM; BS_OPT_TWISTED
// 1 never, 2 whenever the handle allows.  Measured on GB300 (N = 64 .. 2048,
// FP64 and FP32): 1.8-2.3x faster than one thread per system up to 64
// systems per SM, 1.2-1.6x at 128, slower from 256 on, where the one-thread
// sweeps already keep the SMs busy.
bool use_twisted(bs_handle h, int which, bs_layout layout, int64_t M) {
  if (h->width != 3 || h->periodic || !h->twist[which].ok || layout != BS_INTERLEAVED) return false;
  const int64_t o = option(BS_OPT_TWISTED);
  if (o == 1) return false;
  if (o == 2) return true;
  return M <= (int64_t)device_info().sms * 128;
}

cudaError_t sweep_twisted(bs_handle h, int which, const void* in, void* out, bs_dtype t, int64_t M,
                          cudaStream_t st) {
  const int N = (int)h->N;
  const TwistPlan& tp = h->twist[which];
  if (t == BS_F64)
    return launch_tw<double>(tp, N, static_cast<const double*>(in), static_cast<double*>(out), M, st);
  return launch_tw<float>(tp, N, static_cast<const float*>(in), static_cast<float*>(out), M, st);
}

}  // namespace bs
