// Two-ended ("twisted") banded solves for small batches.
//
// With one thread per system (Sec. 2) a batch too small to fill the GPU takes
// as long as one system's chain of 2N dependent steps (forward, then
// backward).  On GB300 a warp-wide FP64 instruction costs the same whatever
// the number of active lanes, so that time does not shrink with the batch:
// N = 64 takes ~14 us for 1 system as for 9728.  Here two threads share a
// system and the chain halves.  The even lane eliminates rows 0 .. k-1
// top-down with the factorisation of Sec. 3.1 / 4.1 (A = L U, A = L R:
// w_i = s_i f_i - l1_i w_{i-1} - l2_i w_{i-2}); the odd lane eliminates rows
// N-1 .. k+h bottom-up with the factorisation of the row-reversed matrix,
// A = U' L' (z_i = s'_i f_i - l1'_i z_{i+1} - l2'_i z_{i+2}), h the band
// half-width.  The h meeting rows k .. k+h-1 are then solved from the two
// lanes' last forward values:
//   tridiagonal:   x_k = (f_k - a_k w_{k-1} - c_k z_{k+1}) / g_k,
//                  g_k = b_k - a_k chat_{k-1} - c_k chat'_{k+1}
//   (row k of A with x_{k-1} = w_{k-1} - chat_{k-1} x_k and x_{k+1} = z_{k+1}
//   - chat'_{k+1} x_k substituted);
//   pentadiagonal: rows k and k+1 with x_{k-2}, x_{k-1} (from the top lane's
//   back-substitution) and x_{k+2}, x_{k+3} (bottom lane) written as affine
//   functions of x_k, x_{k+1}: a 2x2 system whose inverse and right-hand
//   side weights are formed with the handle.
// Each lane then back-substitutes its part outward: x_i = w_i - u1_i x_{i+1}
// - u2_i x_{i+2} above, x_i = z_i - u1'_i x_{i-1} - u2'_i x_{i-2} below.
// About N + 2h dependent steps instead of 2N, and per row the same FP64
// operations as the one-thread sweeps.
#include "sweep_kernels.cuh"

namespace bs {

constexpr int kTwThreads = 64;

template <typename C>
struct TwistArgs {
  const C* s[2];   // [0] top part: plan of A = L U / L R; [1] bottom part: plan of A = U' L'
  const C* l1[2];  // (each indexed by matrix row)
  const C* l2[2];
  const C* u1[2];
  const C* u2[2];
  int k;           // first meeting row
  C m[10];         // meeting-row weights (TwistPlan::m)
};

// One input value widened to the compute type (BF16 storage: exact in FP32).
template <typename C, typename Sin>
__device__ __forceinline__ C tw_load(const Sin* p) {
  if constexpr (std::is_same<Sin, __nv_bfloat16>::value)
    return bf16_bits_to_float(*reinterpret_cast<const unsigned short*>(p));
  else
    return *p;
}

// Even lane (t = 0): rows 0, 1, .., k-1 forward, then k-1, .., 0 backward.
// Odd lane (t = 1): rows N-1, .., k+BW forward, then k+BW, .., N-1 backward.
template <typename C, typename Sin, int BW, int U>
__global__ void __launch_bounds__(kTwThreads)
k_sweep_tw(TwistArgs<C> ta, int N, const Sin* in, C* out, int64_t M) {  // in == out allowed
  const int t = threadIdx.x & 1;
  const int k = ta.k;
  const int n = t ? N - k - BW : k;      // rows this lane eliminates
  const int r0 = t ? N - 1 : 0;          // its first row
  const int dr = t ? -1 : 1;             // row step of its forward sweep
  // selects, not a dynamic index into the kernel parameters
  const C* __restrict__ S = t ? ta.s[1] : ta.s[0];
  const C* __restrict__ L1 = t ? ta.l1[1] : ta.l1[0];
  const C* __restrict__ L2 = t ? ta.l2[1] : ta.l2[0];
  const C* __restrict__ U1 = t ? ta.u1[1] : ta.u1[0];
  const C* __restrict__ U2 = t ? ta.u2[1] : ta.u2[0];
  const unsigned pair = 3u << ((threadIdx.x & 31) & ~1u);
  const int64_t pairs = ((int64_t)gridDim.x * blockDim.x) >> 1;
  for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 1; j < M; j += pairs) {
    const int64_t dp = t ? -M : M;       // pointer step of the forward sweep
    // forward sweep over this lane's n rows, U rows per block, the next
    // block's inputs requested before the current block is computed
    C w1 = C(0), w2 = C(0);  // the last and second-to-last forward values
    {
      const Sin* pin = in + (int64_t)r0 * M + j;
      C* pout = out + (int64_t)r0 * M + j;
      C fa[U], fb[U];
      auto load = [&](C (&f)[U], int q0) {
#pragma unroll
        for (int u = 0; u < U; u++)
          if (q0 + u < n) f[u] = tw_load<C>(pin + (int64_t)(q0 + u) * dp);
      };
      auto run = [&](C (&f)[U], int q0) {
        C sv[U], lv[U], lw[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int i = r0 + dr * (q0 + u < n ? q0 + u : q0);
          sv[u] = __ldg(S + i);
          lv[u] = __ldg(L1 + i);
          lw[u] = BW == 2 ? __ldg(L2 + i) : C(0);
        }
#pragma unroll
        for (int u = 0; u < U; u++)
          if (q0 + u < n) {
            C w = f[u] * sv[u];
            if (BW == 2) w = fma(-lw[u], w2, w);
            w = fma(-lv[u], w1, w);
            w2 = w1;
            w1 = w;
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
    // meeting rows, read and written by the even lane only: it receives the
    // odd lane's last forward values (0 where that lane has fewer rows) and
    // hands the meeting rows' solution back.  The shuffles name exactly the
    // two lanes of the pair, whose loops above may have run different trip
    // counts.
    const C z1 = __shfl_xor_sync(pair, w1, 1);
    const C z2 = __shfl_xor_sync(pair, w2, 1);
    C x1 = C(0), x2 = C(0);  // backward state: the nearest and next solved rows
    if (t == 0) {
      const C* m = ta.m;
      if constexpr (BW == 1) {
        x1 = fma(m[1], z1, fma(m[0], w1, tw_load<C>(in + (int64_t)k * M + j))) * m[2];
        out[(int64_t)k * M + j] = x1;
      } else {
        const C r0v = fma(m[2], z1, fma(m[1], w1, fma(m[0], w2, tw_load<C>(in + (int64_t)k * M + j))));
        const C r1v = fma(m[5], z2, fma(m[4], z1, fma(m[3], w1, tw_load<C>(in + (int64_t)(k + 1) * M + j))));
        x1 = fma(m[7], r1v, m[6] * r0v);  // x_k
        x2 = fma(m[9], r1v, m[8] * r0v);  // x_{k+1}
        out[(int64_t)k * M + j] = x1;
        out[(int64_t)(k + 1) * M + j] = x2;
      }
    }
    {
      const C e1 = __shfl_xor_sync(pair, x1, 1);
      const C e2 = __shfl_xor_sync(pair, x2, 1);
      if (t) {  // below the meeting rows the nearest solved row is the last one
        x1 = BW == 2 ? e2 : e1;
        x2 = BW == 2 ? e1 : C(0);
      }
    }
    // backward sweep outward from the meeting rows over the same n rows
    {
      const int rb = t ? k + BW : k - 1;  // first row
      C* pb = out + (int64_t)rb * M + j;
      C fa[U], fb[U];
      auto load = [&](C (&f)[U], int q0) {
#pragma unroll
        for (int u = 0; u < U; u++)
          if (q0 + u < n) f[u] = pb[-(int64_t)(q0 + u) * dp];
      };
      auto run = [&](C (&f)[U], int q0) {
        C uv[U], uw[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int i = rb - dr * (q0 + u < n ? q0 + u : q0);
          uv[u] = __ldg(U1 + i);
          uw[u] = BW == 2 ? __ldg(U2 + i) : C(0);
        }
#pragma unroll
        for (int u = 0; u < U; u++)
          if (q0 + u < n) {
            C x = f[u];
            if (BW == 2) x = fma(-uw[u], x2, x);
            x = fma(-uv[u], x1, x);
            x2 = x1;
            x1 = x;
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

template <typename C, typename Sin>
static cudaError_t launch_tw(const TwistPlan& tp, int bw, int N, const Sin* in, C* out, int64_t M, cudaStream_t st) {
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
    ta.l2[q] = cf.l2;
    ta.u1[q] = cf.u1;
    ta.u2[q] = cf.u2;
  }
  ta.k = tp.k;
  for (int q = 0; q < 10; q++) ta.m[q] = (C)tp.m[q];
  const int64_t threads = 2 * M;
  int64_t grid = (threads + kTwThreads - 1) / kTwThreads;
  const int64_t cap = (int64_t)device_info().sms * (2048 / kTwThreads);
  if (grid > cap) grid = cap;
  if (bw == 1)
    k_sweep_tw<C, Sin, 1, 8><<<(int)grid, kTwThreads, 0, st>>>(ta, N, in, out, M);
  else
    k_sweep_tw<C, Sin, 2, 8><<<(int)grid, kTwThreads, 0, st>>>(ta, N, in, out, M);
  return cudaGetLastError();
}

// Whether a solve with A (which = 0) or A^T (which = 1) takes the two-ended
// sweep: not periodic, the handle has meeting rows for that matrix,
// interleaved layout, and at most 128 systems per SM; BS_OPT_TWISTED 1
// never, 2 whenever the handle allows.  Measured on GB300 (tridiagonal,
// N = 64 .. 2048, FP64 and FP32): 1.8-2.3x faster than one thread per system
// up to 64 systems per SM, 1.2-1.6x at 128, slower from 256 on, where the
// one-thread sweeps already keep the SMs busy.
bool use_twisted(bs_handle h, int which, bs_layout layout, int64_t M) {
  if (h->periodic || !h->twist[which].ok || layout != BS_INTERLEAVED) return false;
  const int64_t o = option(BS_OPT_TWISTED);
  if (o == 1) return false;
  if (o == 2) return true;
  return M <= (int64_t)device_info().sms * 128;
}

// t: storage type of `in` (BS_BF16: FP32 arithmetic and output).
cudaError_t sweep_twisted(bs_handle h, int which, const void* in, void* out, bs_dtype t, int64_t M,
                          cudaStream_t st) {
  const int N = (int)h->N;
  const int bw = h->width / 2;
  const TwistPlan& tp = h->twist[which];
  if (t == BS_F64)
    return launch_tw<double>(tp, bw, N, static_cast<const double*>(in), static_cast<double*>(out), M, st);
  if (t == BS_BF16)
    return launch_tw<float>(tp, bw, N, static_cast<const __nv_bfloat16*>(in), static_cast<float*>(out), M, st);
  return launch_tw<float>(tp, bw, N, static_cast<const float*>(in), static_cast<float*>(out), M, st);
}

}  // namespace bs
