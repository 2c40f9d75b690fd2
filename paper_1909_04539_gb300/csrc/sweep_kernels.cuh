// Batched shared-LHS sweep kernels (sm_103a).
//
// One thread owns V neighbouring systems (V = one 128-bit load of the input
// type, or 1 for ragged M) and runs, for each of them, the forward sweep over
// rows 0..N-1 and then the backward sweep over rows N-1..0 (Sec. 2: "each
// thread handles a particular system ... forward sweep followed by a backward
// sweep").  The LHS coefficients are one shared copy (Sec. 2, Fig. 1), staged
// once per CTA into shared memory and read as warp-wide broadcasts.  The
// forward-sweep values are kept in the output buffer between the sweeps, as
// the paper overwrites the RHS in place (Sec. 3.1); the launcher bounds the
// number of systems in flight so that these values are still in L2 when the
// backward sweep reads them back.
//
// Both the primal solve (A^{-1}) and the adjoint solve (A^{-T}) of both band
// widths use the same recurrence pair
//   forward : w_i = s_i f_i - l1_i w_{i-1} - l2_i w_{i-2}
//   backward: x_i = t_i w_i - u1_i x_{i+1} - u2_i x_{i+2}
// where the primal has t == 1 and the adjoint s == 1 (ADJ).  Each step's
// dependency on the previous row goes through a single FMA.
//
// Uniform pentadiagonal matrices (every entry of the outermost sub-diagonal
// equal, Sec. 4.1's cuPentUniformBatch) keep that entry as one scalar eps
// (UNI): the primal forward step is w_i = s_i (f_i - eps w_{i-2}) - l1_i
// w_{i-1} and the adjoint backward step x_i = t_i (w_i - eps x_{i+2}) - u1_i
// x_{i+1}, so one coefficient array fewer is staged and read per row.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "internal.h"

namespace bs {

constexpr int kSweepThreads = 128;

// ------------------------------------------------------------------ I/O

template <typename S, typename C, int V>
struct IO;

template <>
struct IO<double, double, 2> {
  static __device__ __forceinline__ void load(const double* p, double (&o)[2]) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    o[0] = t.x;
    o[1] = t.y;
  }
  static __device__ __forceinline__ void store(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};
template <>
struct IO<double, double, 1> {
  static __device__ __forceinline__ void load(const double* p, double (&o)[1]) { o[0] = *p; }
  static __device__ __forceinline__ void store(double* p, const double (&v)[1]) { *p = v[0]; }
};
template <>
struct IO<float, float, 4> {
  static __device__ __forceinline__ void load(const float* p, float (&o)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = t.x;
    o[1] = t.y;
    o[2] = t.z;
    o[3] = t.w;
  }
  static __device__ __forceinline__ void store(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct IO<float, float, 2> {
  static __device__ __forceinline__ void load(const float* p, float (&o)[2]) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    o[0] = t.x;
    o[1] = t.y;
  }
  static __device__ __forceinline__ void store(float* p, const float (&v)[2]) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  }
};
template <>
struct IO<float, float, 1> {
  static __device__ __forceinline__ void load(const float* p, float (&o)[1]) { o[0] = *p; }
  static __device__ __forceinline__ void store(float* p, const float (&v)[1]) { *p = v[0]; }
};
// bf16 storage is widened exactly to FP32 (bf16 is the top half of an FP32).
__device__ __forceinline__ float bf16_bits_to_float(uint32_t h) { return __uint_as_float(h << 16); }
template <>
struct IO<__nv_bfloat16, float, 4> {
  static __device__ __forceinline__ void load(const __nv_bfloat16* p, float (&o)[4]) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    o[0] = bf16_bits_to_float(t.x & 0xffffu);
    o[1] = bf16_bits_to_float(t.x >> 16);
    o[2] = bf16_bits_to_float(t.y & 0xffffu);
    o[3] = bf16_bits_to_float(t.y >> 16);
  }
};
template <>
struct IO<__nv_bfloat16, float, 1> {
  static __device__ __forceinline__ void load(const __nv_bfloat16* p, float (&o)[1]) {
    o[0] = bf16_bits_to_float(*reinterpret_cast<const unsigned short*>(p));
  }
};

// ------------------------------------------------------- coefficient staging

// Copies the coefficient arrays a sweep of kind (BW, ADJ, PER) uses into
// shared memory (when SMEM) and returns pointers to wherever they live.
template <int BW, bool ADJ, bool SMEM, typename C, bool PER = false, bool UNI = false>
__device__ __forceinline__ Coefs<C> stage_coefs(Coefs<C> cf, int N, C* sm) {
  if (SMEM) {
    int off = 0;
    auto stage = [&](const C*& p) {
      C* dst = sm + off;
      for (int i = threadIdx.x; i < N; i += blockDim.x) dst[i] = p[i];
      p = dst;
      off += N;
    };
    if (!ADJ) stage(cf.s);
    stage(cf.l1);
    if (BW == 2 && !(UNI && !ADJ)) stage(cf.l2);
    if (ADJ) stage(cf.t);
    stage(cf.u1);
    if (BW == 2 && !(UNI && ADJ)) stage(cf.u2);
    if (PER) {
      stage(cf.pw);
      stage(cf.pc);
    }
    __syncthreads();
  }
  return cf;
}

template <int BW, bool PER = false, bool UNI = false>
__host__ __device__ constexpr int coef_arrays() {
  // scale + BW lower + BW upper (+ pw, pc) (- the scalar eps's array)
  return 1 + 2 * BW + (PER ? 2 : 0) - ((UNI && BW == 2) ? 1 : 0);
}

// Coefficients of rows r0, r0 + 1, ... (the row block of a partitioned
// launch) as a plan of its own.
template <typename C>
__host__ __device__ __forceinline__ Coefs<C> shift_coefs(Coefs<C> c, int r0) {
  c.s += r0;
  c.l1 += r0;
  c.l2 += r0;
  c.t += r0;
  c.u1 += r0;
  c.u2 += r0;
  c.pw += r0;
  c.pc += r0;
  c.per_lo -= r0;
  c.per_hi -= r0;
  return c;
}

// Periodic correction terms (Sherman-Morrison, Sec. 3.3) of one block of U
// rows: before the forward block, sig += pw_i f_i over the raw inputs; after
// the backward block, f_i -= sig pc_i (the recurrence state keeps the
// uncorrected values).  Callers skip blocks that lie entirely inside
// [per_lo, per_hi), where both arrays are zero.
template <typename C, int V, int U>
__device__ __forceinline__ void per_dot(const Coefs<C>& cf, int i0, int n, const C (&f)[U][V], C (&sig)[V]) {
  C pw[U];
#pragma unroll
  for (int u = 0; u < U; u++) pw[u] = cf.pw[(u < n) ? i0 + u : i0];
#pragma unroll
  for (int u = 0; u < U; u++)
    if (u < n)
#pragma unroll
      for (int v = 0; v < V; v++) sig[v] = fma(pw[u], f[u][v], sig[v]);
}
template <typename C, int V, int U>
__device__ __forceinline__ void per_fix(const Coefs<C>& cf, int top, int n, C (&f)[U][V], const C (&sig)[V]) {
  C pc[U];
#pragma unroll
  for (int u = 0; u < U; u++) pc[u] = cf.pc[(u < n) ? top - u : top];
#pragma unroll
  for (int u = 0; u < U; u++)
    if (u < n)
#pragma unroll
      for (int v = 0; v < V; v++) f[u][v] = fma(-sig[v], pc[u], f[u][v]);
}

// One forward step for V systems at row i (f holds the input on entry and
// the forward value on exit).
template <int BW, bool ADJ, typename C, int V, bool UNI = false>
__device__ __forceinline__ void fwd_step(const Coefs<C>& cf, int i, C (&f)[V], C (&w1)[V], C (&w2)[V]) {
  constexpr bool kUni = UNI && !ADJ && BW == 2;
  const C l1 = cf.l1[i];
  C s = C(1), l2 = C(0);
  if (!ADJ) s = cf.s[i];
  if (BW == 2 && !kUni) l2 = cf.l2[i];
#pragma unroll
  for (int v = 0; v < V; v++) {
    C w;
    if (kUni) {
      w = fma(-cf.eps, w2[v], f[v]) * s;
    } else {
      w = ADJ ? f[v] : f[v] * s;
      if (BW == 2) w = fma(-l2, w2[v], w);
    }
    w = fma(-l1, w1[v], w);
    if (BW == 2) w2[v] = w1[v];
    w1[v] = w;
    f[v] = w;
  }
}

// One backward step for V systems at row i (f holds w_i on entry, x_i on exit).
template <int BW, bool ADJ, typename C, int V, bool UNI = false>
__device__ __forceinline__ void bwd_step(const Coefs<C>& cf, int i, C (&f)[V], C (&x1)[V], C (&x2)[V]) {
  constexpr bool kUni = UNI && ADJ && BW == 2;
  const C u1 = cf.u1[i];
  C t = C(1), u2 = C(0);
  if (ADJ) t = cf.t[i];
  if (BW == 2 && !kUni) u2 = cf.u2[i];
#pragma unroll
  for (int v = 0; v < V; v++) {
    C x;
    if (kUni) {
      x = fma(-cf.eps, x2[v], f[v]) * t;
    } else {
      x = ADJ ? f[v] * t : f[v];
      if (BW == 2) x = fma(-u2, x2[v], x);
    }
    x = fma(-u1, x1[v], x);
    if (BW == 2) x2[v] = x1[v];
    x1[v] = x;
    f[v] = x;
  }
}

// Block versions of the two steps: U consecutive rows (n of them valid).
// All coefficient loads of the block are issued before any arithmetic, so
// they do not wait behind the caller's stores of the previous block (which
// the compiler must assume may alias them).  Per row and system the
// arithmetic is exactly that of fwd_step / bwd_step.
template <int BW, bool ADJ, typename C, int V, int U, bool UNI = false>
__device__ __forceinline__ void fwd_block(const Coefs<C>& cf, int i0, int n, C (&f)[U][V], C (&w1)[V],
                                          C (&w2)[V]) {
  constexpr bool kUni = UNI && !ADJ && BW == 2;
  C s[U], l1[U], l2[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    const int i = (u < n) ? i0 + u : i0;
    l1[u] = cf.l1[i];
    s[u] = ADJ ? C(1) : cf.s[i];
    l2[u] = (BW == 2 && !kUni) ? cf.l2[i] : C(0);
  }
#pragma unroll
  for (int u = 0; u < U; u++) {
    if (u < n) {
#pragma unroll
      for (int v = 0; v < V; v++) {
        C w;
        if (kUni) {
          w = fma(-cf.eps, w2[v], f[u][v]) * s[u];
        } else {
          w = ADJ ? f[u][v] : f[u][v] * s[u];
          if (BW == 2) w = fma(-l2[u], w2[v], w);
        }
        w = fma(-l1[u], w1[v], w);
        if (BW == 2) w2[v] = w1[v];
        w1[v] = w;
        f[u][v] = w;
      }
    }
  }
}

// Backward block: rows top, top-1, ..., top-n+1 held in f[0..n-1].
template <int BW, bool ADJ, typename C, int V, int U, bool UNI = false>
__device__ __forceinline__ void bwd_block(const Coefs<C>& cf, int top, int n, C (&f)[U][V], C (&x1)[V],
                                          C (&x2)[V]) {
  constexpr bool kUni = UNI && ADJ && BW == 2;
  C t[U], u1[U], u2[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    const int i = (u < n) ? top - u : top;
    u1[u] = cf.u1[i];
    t[u] = ADJ ? cf.t[i] : C(1);
    u2[u] = (BW == 2 && !kUni) ? cf.u2[i] : C(0);
  }
#pragma unroll
  for (int u = 0; u < U; u++) {
    if (u < n) {
#pragma unroll
      for (int v = 0; v < V; v++) {
        C x;
        if (kUni) {
          x = fma(-cf.eps, x2[v], f[u][v]) * t[u];
        } else {
          x = ADJ ? f[u][v] * t[u] : f[u][v];
          if (BW == 2) x = fma(-u2[u], x2[v], x);
        }
        x = fma(-u1[u], x1[v], x);
        if (BW == 2) x2[v] = x1[v];
        x1[v] = x;
        f[u][v] = x;
      }
    }
  }
}

// FP32 sweeps whose coefficients are staged in shared memory keep each row's
// forward (s, l1, l2) and backward (t, u1, u2) coefficients in one 16-byte
// record each: one 128-bit shared load per row and sweep instead of one load
// per coefficient array (the FP32 sweeps are bound by instruction issue).
// The arithmetic is that of fwd_block / bwd_block.
template <int BW, bool ADJ, bool UNI>
__device__ __forceinline__ void stage_records(const Coefs<float>& cf, int N, float4* fr, float4* br) {
  constexpr bool kUniF = UNI && !ADJ && BW == 2, kUniB = UNI && ADJ && BW == 2;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    fr[i] = make_float4(ADJ ? 1.f : cf.s[i], cf.l1[i], (BW == 2 && !kUniF) ? cf.l2[i] : 0.f, 0.f);
    br[i] = make_float4(ADJ ? cf.t[i] : 1.f, cf.u1[i], (BW == 2 && !kUniB) ? cf.u2[i] : 0.f, 0.f);
  }
  __syncthreads();
}

template <int BW, bool ADJ, int V, int U, bool UNI>
__device__ __forceinline__ void fwd_block_rec(const float4* fr, float eps, int i0, int n, float (&f)[U][V],
                                              float (&w1)[V], float (&w2)[V]) {
  constexpr bool kUni = UNI && !ADJ && BW == 2;
  float4 r[U];
#pragma unroll
  for (int u = 0; u < U; u++) r[u] = fr[(u < n) ? i0 + u : i0];
#pragma unroll
  for (int u = 0; u < U; u++) {
    if (u < n) {
#pragma unroll
      for (int v = 0; v < V; v++) {
        float w;
        if (kUni) {
          w = fmaf(-eps, w2[v], f[u][v]) * r[u].x;
        } else {
          w = ADJ ? f[u][v] : f[u][v] * r[u].x;
          if (BW == 2) w = fmaf(-r[u].z, w2[v], w);
        }
        w = fmaf(-r[u].y, w1[v], w);
        if (BW == 2) w2[v] = w1[v];
        w1[v] = w;
        f[u][v] = w;
      }
    }
  }
}

template <int BW, bool ADJ, int V, int U, bool UNI>
__device__ __forceinline__ void bwd_block_rec(const float4* br, float eps, int top, int n, float (&f)[U][V],
                                              float (&x1)[V], float (&x2)[V]) {
  constexpr bool kUni = UNI && ADJ && BW == 2;
  float4 r[U];
#pragma unroll
  for (int u = 0; u < U; u++) r[u] = br[(u < n) ? top - u : top];
#pragma unroll
  for (int u = 0; u < U; u++) {
    if (u < n) {
#pragma unroll
      for (int v = 0; v < V; v++) {
        float x;
        if (kUni) {
          x = fmaf(-eps, x2[v], f[u][v]) * r[u].x;
        } else {
          x = ADJ ? f[u][v] * r[u].x : f[u][v];
          if (BW == 2) x = fmaf(-r[u].z, x2[v], x);
        }
        x = fmaf(-r[u].y, x1[v], x);
        if (BW == 2) x2[v] = x1[v];
        x1[v] = x;
        f[u][v] = x;
      }
    }
  }
}

// ------------------------------------------------------ async row copies

// Per-lane rings of rows in shared memory, filled with cp.async.  Each lane
// copies and later reads only its own bytes, so no barrier is needed: a lane
// waits for its own copy groups (cp.async.wait_group), which complete in
// order.  Slot r of lane t sits at ring + (r * blockDim.x + t) * SLOT, so a
// warp reads 32 * SLOT contiguous bytes.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// 16 bytes through L2 only (.cg): also safe for data this thread stored
// earlier in the same kernel.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
// 8 bytes through L1 (.ca); used only for inputs the kernel never writes.
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
// 4 bytes through L1 (.ca), likewise.
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

// One lane-row copy of V elements of S (V * sizeof(S) is 8, 16 or 32 bytes).
template <typename S, int V>
__device__ __forceinline__ void copy_row(uint32_t dst, const S* src) {
  constexpr int bytes = V * (int)sizeof(S);
  static_assert(bytes == 8 || bytes == 16 || bytes == 32, "lane row must be 8, 16 or 32 bytes");
  if constexpr (bytes == 8) {
    cp_async8(dst, src);
  } else if constexpr (bytes == 16) {
    cp_async16(dst, src);
  } else {
    cp_async16(dst, src);
    cp_async16(dst + 16, reinterpret_cast<const unsigned char*>(src) + 16);
  }
}

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------- interleaved layout

// Row i of system j at [i*M + j].  Thread g owns systems [g*V, g*V + V).
// Rows are moved in blocks of U with a two-block register pipeline: the loads
// of the next block are issued before the current block is computed, so each
// thread keeps up to 2*U*V loads in flight.
template <int BW, bool ADJ, bool SMEM, typename C, typename Sin, typename Sout, int V, int U, bool PER, bool UNI>
__global__ void __launch_bounds__(kSweepThreads)
k_sweep_il(Coefs<C> cf_g, int N, const Sin* in, Sout* out, int64_t M, int L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  {  // row block of a partitioned launch (blockIdx.y; L = N otherwise)
    const int r0 = blockIdx.y * L;
    N = (N - r0) < L ? (N - r0) : L;
    cf_g = shift_coefs(cf_g, r0);
    in += (int64_t)r0 * M;
    out += (int64_t)r0 * M;
  }
  const Coefs<C> cf = stage_coefs<BW, ADJ, SMEM, C, PER, UNI>(cf_g, N, reinterpret_cast<C*>(smem_raw));
  const int64_t ngroups = M / V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
    const Sin* pin = in + g * V;
    Sout* pout = out + g * V;
    C a[U][V], b[U][V];
    C r1[V], r2[V], sig[V];
#pragma unroll
    for (int v = 0; v < V; v++) sig[v] = C(0);

    auto load_fwd = [&](C (&blk)[U][V], int i0) {
#pragma unroll
      for (int u = 0; u < U; u++)
        if (i0 + u < N) IO<Sin, C, V>::load(pin + (int64_t)(i0 + u) * M, blk[u]);
    };
    auto run_fwd = [&](C (&blk)[U][V], int i0) {
      const int n = (N - i0) < U ? (N - i0) : U;
      if constexpr (PER)
        if (i0 < cf.per_lo || i0 + n > cf.per_hi) per_dot<C, V, U>(cf, i0, n, blk, sig);
      fwd_block<BW, ADJ, C, V, U, UNI>(cf, i0, n, blk, r1, r2);
#pragma unroll
      for (int u = 0; u < U; u++)
        if (u < n) IO<Sout, C, V>::store(pout + (int64_t)(i0 + u) * M, blk[u]);
    };
    auto load_bwd = [&](C (&blk)[U][V], int top) {
#pragma unroll
      for (int u = 0; u < U; u++)
        if (top - u >= 0) IO<Sout, C, V>::load(pout + (int64_t)(top - u) * M, blk[u]);
    };
    auto run_bwd = [&](C (&blk)[U][V], int top) {
      const int n = (top + 1) < U ? (top + 1) : U;
      bwd_block<BW, ADJ, C, V, U, UNI>(cf, top, n, blk, r1, r2);
      if constexpr (PER)
        if (top + 1 - n < cf.per_lo || top + 1 > cf.per_hi) per_fix<C, V, U>(cf, top, n, blk, sig);
#pragma unroll
      for (int u = 0; u < U; u++)
        if (u < n) IO<Sout, C, V>::store(pout + (int64_t)(top - u) * M, blk[u]);
    };

    // forward sweep
#pragma unroll
    for (int v = 0; v < V; v++) r1[v] = r2[v] = C(0);
    load_fwd(a, 0);
    for (int i0 = 0; i0 < N; i0 += 2 * U) {
      if (i0 + U < N) load_fwd(b, i0 + U);
      run_fwd(a, i0);
      if (i0 + U >= N) break;
      if (i0 + 2 * U < N) load_fwd(a, i0 + 2 * U);
      run_fwd(b, i0 + U);
    }
    // backward sweep
#pragma unroll
    for (int v = 0; v < V; v++) r1[v] = r2[v] = C(0);
    load_bwd(a, N - 1);
    for (int top = N - 1; top >= 0; top -= 2 * U) {
      if (top - U >= 0) load_bwd(b, top - U);
      run_bwd(a, top);
      if (top - U < 0) break;
      if (top - 2 * U >= 0) load_bwd(a, top - 2 * U);
      run_bwd(b, top - U);
    }
  }
}


// Interleaved layout, deep-pipelined variant for V > 1.  Each lane streams
// its rows through a private ring of D slots (16 bytes each): D rows of
// input are in flight per lane while the recurrence runs.  The forward values
// of the last D rows stay in the ring, so the backward sweep starts without
// reloading them; the earlier ones go to the output buffer and are streamed
// back through the same ring.
template <int BW, bool ADJ, bool SMEM, typename C, typename Sin, typename Sout, int V, int D, bool PER, bool UNI>
__global__ void __launch_bounds__(kSweepThreads)
k_sweep_il2(Coefs<C> cf_g, int N, const Sin* in, Sout* out, int64_t M, int L) {
  static_assert(V * sizeof(Sout) == 16 || V * sizeof(Sout) == 8, "output lane row must be 8 or 16 bytes");
  constexpr int U = 4;  // rows per block; D is a multiple of U
  static_assert(D % U == 0, "ring depth must be a multiple of the block");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  {  // row block of a partitioned launch (blockIdx.y; L = N otherwise)
    const int r0 = blockIdx.y * L;
    N = (N - r0) < L ? (N - r0) : L;
    cf_g = shift_coefs(cf_g, r0);
    in += (int64_t)r0 * M;
    out += (int64_t)r0 * M;
  }
  // FP32 with staged coefficients: per-row records (stage_records)
  constexpr bool REC = SMEM && std::is_same<C, float>::value && !PER;
  const float4* fr = reinterpret_cast<const float4*>(smem_raw);
  const float4* br = fr + N;
  Coefs<C> cf = cf_g;
  size_t coef_bytes;
  if constexpr (REC) {
    stage_records<BW, ADJ, UNI>(cf_g, N, reinterpret_cast<float4*>(smem_raw), reinterpret_cast<float4*>(smem_raw) + N);
    coef_bytes = (size_t)N * 2 * sizeof(float4);
  } else {
    cf = stage_coefs<BW, ADJ, SMEM, C, PER, UNI>(cf_g, N, reinterpret_cast<C*>(smem_raw));
    coef_bytes = SMEM ? align_up((size_t)coef_arrays<BW, PER, UNI>() * N * sizeof(C), 16) : 0;
  }
  unsigned char* ring = smem_raw + coef_bytes + (size_t)threadIdx.x * 16;
  const uint32_t ring_s = smem_u32(ring);
  const uint32_t pitch = blockDim.x * 16;
  const int64_t ngroups = M / V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
    const Sin* pin = in + g * V;
    Sout* pout = out + g * V;
    C r1[V], r2[V], sig[V];
#pragma unroll
    for (int v = 0; v < V; v++) r1[v] = r2[v] = sig[v] = C(0);
    // forward sweep: rows 0..D-1 requested up front (one copy group per
    // block of U rows), then each block is consumed and its slots refilled
    // with one new group; the group a block waits for was committed D / U
    // groups earlier
    const Sin* pnext = pin;  // next row to request
#pragma unroll 1
    for (int r = 0; r < D; r++) {
      if (r < N) copy_row<Sin, V>(ring_s + r * pitch, pnext);
      pnext += M;
      if ((r + 1) % U == 0) cp_commit();
    }
    Sout* prow = pout;  // output row i0
    // one block of U rows; FULL: all U rows exist and each refills its slot
    // (no per-row guards), otherwise the guarded general case
    auto fwd = [&](auto full_tag, int i0) {
      constexpr bool FULL = decltype(full_tag)::value;
      cp_wait<D / U - 1>();
      const int n = FULL ? U : ((N - i0) < U ? (N - i0) : U);
      const int s0 = i0 % D;
      C f[U][V];
#pragma unroll
      for (int u = 0; u < U; u++)
        if (FULL || u < n) IO<Sin, C, V>::load(reinterpret_cast<const Sin*>(ring + (size_t)(s0 + u) * pitch), f[u]);
      if constexpr (PER)
        if (i0 < cf.per_lo || i0 + n > cf.per_hi) per_dot<C, V, U>(cf, i0, n, f, sig);
      if constexpr (REC)
        fwd_block_rec<BW, ADJ, V, U, UNI>(fr, cf.eps, i0, n, f, r1, r2);
      else
        fwd_block<BW, ADJ, C, V, U, UNI>(cf, i0, n, f, r1, r2);
#pragma unroll
      for (int u = 0; u < U; u++) {
        if constexpr (FULL) {
          IO<Sout, C, V>::store(prow, f[u]);
          copy_row<Sin, V>(ring_s + (s0 + u) * pitch, pnext);
        } else {
          const int i = i0 + u;
          if (u < n) {
            if (i + D < N) {
              IO<Sout, C, V>::store(prow, f[u]);
              copy_row<Sin, V>(ring_s + (s0 + u) * pitch, pnext);
            } else {
              IO<Sout, C, V>::store(reinterpret_cast<Sout*>(ring + (size_t)(s0 + u) * pitch), f[u]);  // tail on chip
            }
          }
        }
        prow += M;
        pnext += M;
      }
      cp_commit();
    };
    // (periodic plans keep the one guarded loop: a second, unguarded copy of
    // their body raised the FP64 kernel from 80 to 92 registers and made the
    // periodic spline solve 25 % slower)
    int i0 = 0;
    if constexpr (!PER) {
#pragma unroll 1
      for (; i0 + U + D <= N; i0 += U) fwd(std::true_type{}, i0);
    }
#pragma unroll 1
    for (; i0 < N; i0 += U) fwd(std::false_type{}, i0);
    // backward sweep: rows N-1 .. N-D are in the ring; row i - D is requested
    // into the slot row i frees (one group per block, as above; blocks are
    // aligned to N - 1 and D is a multiple of U, so the rows a block needs
    // were requested together, D / U blocks earlier)
#pragma unroll
    for (int v = 0; v < V; v++) r1[v] = r2[v] = C(0);
    const int tail = N - D;
    prow = pout + (int64_t)(N - 1) * M;               // output row `top`
    const Sout* pback = pout + (int64_t)(N - 1 - D) * M;  // row top - D, requested next
    // FULL: all U rows exist and each requests row i - D.  Its wait is also
    // taken on the first blocks, whose rows are on chip: fewer than D / U
    // groups are pending then, so it does not block.
    auto bwd = [&](auto full_tag, int top) {
      constexpr bool FULL = decltype(full_tag)::value;
      const int n = FULL ? U : ((top + 1) < U ? (top + 1) : U);
      if (FULL || top - (n - 1) < tail) cp_wait<D / U - 1>();
      C f[U][V];
#pragma unroll
      for (int u = 0; u < U; u++)
        if (FULL || u < n)
          IO<Sout, C, V>::load(reinterpret_cast<const Sout*>(ring + (size_t)((top - u) % D) * pitch), f[u]);
      if constexpr (REC)
        bwd_block_rec<BW, ADJ, V, U, UNI>(br, cf.eps, top, n, f, r1, r2);
      else
        bwd_block<BW, ADJ, C, V, U, UNI>(cf, top, n, f, r1, r2);
      if constexpr (PER)
        if (top + 1 - n < cf.per_lo || top + 1 > cf.per_hi) per_fix<C, V, U>(cf, top, n, f, sig);
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int i = top - u;
        if constexpr (FULL) {
          IO<Sout, C, V>::store(prow, f[u]);
          copy_row<Sout, V>(ring_s + (i % D) * pitch, pback);
        } else {
          if (u < n) {
            IO<Sout, C, V>::store(prow, f[u]);
            if (i - D >= 0) copy_row<Sout, V>(ring_s + (i % D) * pitch, pback);
          }
        }
        prow -= M;
        pback -= M;
      }
      cp_commit();
    };
    int top = N - 1;
    if constexpr (!PER) {
#pragma unroll 1
      for (; top >= D + U - 1; top -= U) bwd(std::true_type{}, top);
    }
#pragma unroll 1
    for (; top >= 0; top -= U) bwd(std::false_type{}, top);
    cp_wait<0>();
  }
}

// ------------------------------------------------------ strided layout

// Row i of system j at [j*N + i] (system-contiguous).  Each warp owns 32
// systems, one per lane, and moves rows in chunks of 32 through a private
// shared-memory tile: for each system the 32 lanes load 32 consecutive rows
// (one coalesced segment) into a tile column, then each lane sweeps its own
// system down the tile, then the tile goes back the same way.
constexpr int kStRows = 32;
constexpr int kStPad = 33;

template <int BW, bool ADJ, bool SMEM, typename C, typename Sin, typename Sout, bool PER, bool UNI>
__global__ void __launch_bounds__(kSweepThreads)
k_sweep_st(Coefs<C> cf_g, int N, const Sin* in, Sout* out, int64_t M, int64_t ld, int L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  {  // row block of a partitioned launch (blockIdx.y; L = N otherwise); ld = system stride
    const int r0 = blockIdx.y * L;
    N = (N - r0) < L ? (N - r0) : L;
    cf_g = shift_coefs(cf_g, r0);
    in += r0;
    out += r0;
  }
  C* smc = reinterpret_cast<C*>(smem_raw);
  const Coefs<C> cf = stage_coefs<BW, ADJ, SMEM, C, PER, UNI>(cf_g, N, smc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kWarps = kSweepThreads / 32;
  C* tile = smc + (SMEM ? coef_arrays<BW, PER, UNI>() * N : 0) + warp * kStRows * kStPad;
  const int64_t nwg = (M + 31) / 32;
  for (int64_t wg = (int64_t)blockIdx.x * kWarps + warp; wg < nwg; wg += (int64_t)gridDim.x * kWarps) {
    const int64_t j0 = wg * 32;
    const int nsys = (int)((M - j0) < 32 ? (M - j0) : 32);
    const bool mine = lane < nsys;
    C r1[1] = {C(0)}, r2[1] = {C(0)}, sig[1] = {C(0)};
    // forward sweep, chunks of rows in increasing order
    for (int c0 = 0; c0 < N; c0 += kStRows) {
      const int rows = (N - c0) < kStRows ? (N - c0) : kStRows;
      if (lane < rows)
        for (int s = 0; s < nsys; s++) {
          C v[1];
          IO<Sin, C, 1>::load(in + (j0 + s) * ld + c0 + lane, v);
          tile[lane * kStPad + s] = v[0];
        }
      __syncwarp();
      if (mine)
        for (int r = 0; r < rows; r++) {
          C f[1] = {tile[r * kStPad + lane]};
          if constexpr (PER)
            if (c0 + r < cf.per_lo || c0 + r >= cf.per_hi) sig[0] = fma(cf.pw[c0 + r], f[0], sig[0]);
          fwd_step<BW, ADJ, C, 1, UNI>(cf, c0 + r, f, r1, r2);
          tile[r * kStPad + lane] = f[0];
        }
      __syncwarp();
      if (lane < rows)
        for (int s = 0; s < nsys; s++) {
          const C v[1] = {tile[lane * kStPad + s]};
          IO<Sout, C, 1>::store(out + (j0 + s) * ld + c0 + lane, v);
        }
      __syncwarp();
    }
    // backward sweep, chunks in decreasing order
    r1[0] = r2[0] = C(0);
    const int last = ((N - 1) / kStRows) * kStRows;
    for (int c0 = last; c0 >= 0; c0 -= kStRows) {
      const int rows = (N - c0) < kStRows ? (N - c0) : kStRows;
      if (lane < rows)
        for (int s = 0; s < nsys; s++) {
          C v[1];
          IO<Sout, C, 1>::load(out + (j0 + s) * ld + c0 + lane, v);
          tile[lane * kStPad + s] = v[0];
        }
      __syncwarp();
      if (mine)
        for (int r = rows - 1; r >= 0; r--) {
          C f[1] = {tile[r * kStPad + lane]};
          bwd_step<BW, ADJ, C, 1, UNI>(cf, c0 + r, f, r1, r2);
          if constexpr (PER)
            if (c0 + r < cf.per_lo || c0 + r >= cf.per_hi) f[0] = fma(-sig[0], cf.pc[c0 + r], f[0]);
          tile[r * kStPad + lane] = f[0];
        }
      __syncwarp();
      if (lane < rows)
        for (int s = 0; s < nsys; s++) {
          const C v[1] = {tile[lane * kStPad + s]};
          IO<Sout, C, 1>::store(out + (j0 + s) * ld + c0 + lane, v);
        }
      __syncwarp();
    }
  }
}

// --------------------------------------------------------------- launcher

struct LaunchShape {
  int grid;
  int threads;     // per CTA
  size_t smem;     // coefficient bytes staged in shared memory (0 if read from global)
  bool smem_coefs;
};

// Chooses the grid and shared memory of one sweep launch.  The grid is
// persistent (each thread loops over groups of systems); it is capped so that
// the forward values of all systems in flight take at most half of L2.
// extra_smem_per_thread: shared bytes each thread needs beyond the
// coefficients (ring slots); extra_smem_fixed: per CTA (transpose tiles).
// tpb = 0 lets the policy pick 32, 64 or 128 threads per CTA so that small
// batches still spread over every SM.
// extra_coef_arrays: coefficient arrays staged beyond the 1 + 2 bw of a plain
// sweep (2 for the periodic correction).  balance: pick the CTA size of an
// FP64 launch by the load of the busiest SM (the row-partitioned ADI
// half-steps; solves keep the plain policy, since concurrent solves on other
// streams lose the SMs whose shared memory a balanced grid fills).
LaunchShape sweep_shape(int bw, int N, int64_t threads_needed, size_t coef_elem, size_t spill_elem,
                        int per_thread_systems, size_t extra_smem_per_thread, size_t extra_smem_fixed, int tpb,
                        int extra_coef_arrays = 0, bool balance = false);

// L, P: rows per block and blocks of a partitioned launch (L = N, P = 1
// otherwise); grid.y = P.
template <int BW, bool ADJ, bool PER, bool UNI, typename C, typename Sin, typename Sout, int V>
cudaError_t launch_il(Coefs<C> cf, int N, const Sin* in, Sout* out, int64_t M, int L, int P, cudaStream_t st) {
  constexpr int U = 8;
  constexpr int kExtra = coef_arrays<BW, PER, UNI>() - coef_arrays<BW>();  // arrays beyond 1 + 2 BW
  const int64_t groups = M / V;
  if constexpr (V > 1 || sizeof(Sout) == 8) {
    // pipelined kernel: ring of D 16-byte slots per lane; the FP32 sweeps are
    // bound by memory latency, so they keep twice the rows in flight -- but a
    // partitioned launch has the threads, and shallow rings let more CTAs fit
    // FP32 without the periodic terms stages 8 values per row (two records)
    constexpr int kExtra2 = (sizeof(C) == 4 && !PER) ? 8 - coef_arrays<BW>() : kExtra;
    auto go = [&](auto dtag) -> cudaError_t {
      constexpr int D = decltype(dtag)::value;
      const LaunchShape sh = sweep_shape(BW, L, groups * P, sizeof(C), sizeof(Sout), V, D * 16, 0, 0, kExtra2);
      const size_t bytes = sh.smem + (size_t)sh.threads * D * 16;
      const dim3 grid((sh.grid + P - 1) / P, P);
      auto k = sh.smem_coefs ? k_sweep_il2<BW, ADJ, true, C, Sin, Sout, V, D, PER, UNI>
                             : k_sweep_il2<BW, ADJ, false, C, Sin, Sout, V, D, PER, UNI>;
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
      k<<<grid, sh.threads, bytes, st>>>(cf, N, in, out, M, L);
      return cudaGetLastError();
    };
    if constexpr (sizeof(C) == 4) {
      if (P == 1) return go(std::integral_constant<int, 32>{});
    }
    return go(std::integral_constant<int, 16>{});
  } else {
    const LaunchShape sh = sweep_shape(BW, L, groups * P, sizeof(C), sizeof(Sout), V, 0, 0, 0, kExtra);
    const dim3 grid((sh.grid + P - 1) / P, P);
    if (sh.smem_coefs) {
      auto k = k_sweep_il<BW, ADJ, true, C, Sin, Sout, V, U, PER, UNI>;
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
      if (e != cudaSuccess) return e;
      k<<<grid, sh.threads, sh.smem, st>>>(cf, N, in, out, M, L);
    } else {
      k_sweep_il<BW, ADJ, false, C, Sin, Sout, V, U, PER, UNI><<<grid, sh.threads, 0, st>>>(cf, N, in, out, M, L);
    }
    return cudaGetLastError();
  }
}

template <int BW, bool ADJ, bool PER, bool UNI, typename C, typename Sin, typename Sout>
cudaError_t launch_st(Coefs<C> cf, int N, const Sin* in, Sout* out, int64_t M, int L, int P, cudaStream_t st) {
  constexpr int kExtra = coef_arrays<BW, PER, UNI>() - coef_arrays<BW>();
  const int64_t threads = ((M + 31) / 32) * 32;
  const size_t tiles = (size_t)(kSweepThreads / 32) * kStRows * kStPad * sizeof(C);
  LaunchShape sh = sweep_shape(BW, L, threads * P, sizeof(C), sizeof(Sout), 1, 0, tiles, kSweepThreads, kExtra);
  const dim3 grid((sh.grid + P - 1) / P, P);
  if (sh.smem_coefs) {
    auto k = k_sweep_st<BW, ADJ, true, C, Sin, Sout, PER, UNI>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sh.smem + tiles));
    if (e != cudaSuccess) return e;
    k<<<grid, kSweepThreads, sh.smem + tiles, st>>>(cf, N, in, out, M, (int64_t)N, L);
  } else {
    k_sweep_st<BW, ADJ, false, C, Sin, Sout, PER, UNI><<<grid, kSweepThreads, tiles, st>>>(cf, N, in, out, M, (int64_t)N, L);
  }
  return cudaGetLastError();
}

// Dispatch over band width, direction, layout and vector width for one
// storage/compute type combination.
template <typename C, typename Sin, typename Sout, int VEC>
cudaError_t dispatch_sweep(const SweepPlan& p, bool adjoint, int N, const Sin* in, Sout* out,
                           bs_layout layout, int64_t M, cudaStream_t st, int L = 0, int P = 1) {
  if (L <= 0) L = N;
  const C* base;
  if constexpr (sizeof(C) == 8)
    base = reinterpret_cast<const C*>(p.c64);
  else
    base = reinterpret_cast<const C*>(p.c32);
  Coefs<C> cf = coefs_of<C>(base, N);
  cf.per_lo = p.per_lo;
  cf.per_hi = p.per_hi;
  cf.eps = (C)p.eps;
  bool vec = (M % VEC == 0) && (reinterpret_cast<uintptr_t>(in) % (VEC * sizeof(Sin)) == 0) &&
                   (reinterpret_cast<uintptr_t>(out) % (VEC * sizeof(Sout)) == 0);
  // FP32 with few systems per SM: half-width vectors (8-byte lane rows) give
  // twice the warps to hide the latency of the recurrences
  constexpr bool kHalf = std::is_same<Sin, float>::value && VEC == 4;
  const bool few = M / VEC * P < (int64_t)device_info().sms * 32 * 8;
  const bool half = kHalf && (M % 2 == 0) && (reinterpret_cast<uintptr_t>(in) % 8 == 0) &&
                    (reinterpret_cast<uintptr_t>(out) % 8 == 0) && few;
  // FP64 with few systems per SM: one system per thread (twice the warps)
  if (std::is_same<Sin, double>::value && few) vec = false;
#define BS_DISPATCH(BWV, ADJV, PERV, UNIV)                                                                    \
  if (layout == BS_STRIDED) return launch_st<BWV, ADJV, PERV, UNIV, C, Sin, Sout>(cf, N, in, out, M, L, P, st); \
  if constexpr (kHalf) {                                                                                      \
    if (half)                                                                                                 \
      return launch_il<BWV, ADJV, PERV, UNIV, C, Sin, Sout, (kHalf ? 2 : VEC)>(cf, N, in, out, M, L, P, st);  \
  }                                                                                                           \
  if (vec) return launch_il<BWV, ADJV, PERV, UNIV, C, Sin, Sout, VEC>(cf, N, in, out, M, L, P, st);            \
  return launch_il<BWV, ADJV, PERV, UNIV, C, Sin, Sout, 1>(cf, N, in, out, M, L, P, st);
  if (p.bw == 1 && p.periodic) {
    if (!adjoint) { BS_DISPATCH(1, false, true, false) } else { BS_DISPATCH(1, true, true, false) }
  } else if (p.bw == 1) {
    if (!adjoint) { BS_DISPATCH(1, false, false, false) } else { BS_DISPATCH(1, true, false, false) }
  } else if (sizeof(C) == 4 && p.uniform && option(BS_OPT_UNIFORM) == 2) {
    // on request only, FP32 arithmetic only: with the per-row coefficient
    // records the scalar saves no load and its w_{i-2} link takes three
    // dependent operations per two rows instead of two (measured equal or
    // slower except BF16 storage at N >= 8192, 3 % faster); in FP64, bound
    // by the FP64 pipe, 3 % slower
    if constexpr (sizeof(C) == 4) {
      if (!adjoint) { BS_DISPATCH(2, false, false, true) } else { BS_DISPATCH(2, true, false, true) }
    }
  } else {
    if (!adjoint) { BS_DISPATCH(2, false, false, false) } else { BS_DISPATCH(2, true, false, false) }
  }
#undef BS_DISPATCH
  return cudaErrorNotSupported;  // not reached: every branch above returns
}

}  // namespace bs
