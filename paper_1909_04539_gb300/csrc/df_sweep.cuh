// Per-group arithmetic of the FP64 solves carried in FP32 pairs, shared by
// the two-sweep kernel (sweep_df.cu) and the grouped serving kernel
// (grouped.cu), so that a system gets bitwise the same result from both.
//
// A group is U consecutive rows of the V systems one lane owns.  Every value
// a lane computes depends only on its own systems: the conversions take a
// fast path and fall back, value by value, to the careful ones (df_math.cuh);
// a lane whose input leaves the pairs' range switches itself to native FP64
// from the first row of that group on (rsw), its two recurrence values
// converted exactly.  Warp votes only skip the rare code when no lane needs
// it.
#pragma once

#include "df_math.cuh"
#include "sweep_kernels.cuh"

namespace bs {

// Packed per-row coefficient pairs of one plan (SweepPlan::dfrec layout):
// per sweep a float4 of the first two pairs and a float2 of the third; the
// pairs present, in order, are (s), l1, (l2) forward and (t), u1, (u2)
// backward.
struct DfRecs {
  const float4* f4;
  const float4* b4;
  const float2* f2;
  const float2* b2;
  const float4* pq = nullptr;  // periodic plans: scaled (pw', pc') pairs per row (SweepPlan::dfper)
  double per_unscale = 1.0;    // sigma = per_unscale sigma'
};

__host__ __device__ inline DfRecs df_recs_of(const float* dfrec, int64_t N) {
  const float4* f4 = reinterpret_cast<const float4*>(dfrec);
  return DfRecs{f4, f4 + N, reinterpret_cast<const float2*>(f4 + 2 * N), reinterpret_cast<const float2*>(f4 + 2 * N) + N};
}

template <bool ADJ, int BW>
struct DfCount {
  static constexpr int F = (ADJ ? 0 : 1) + BW;  // forward pairs
  static constexpr int B = (ADJ ? 1 : 0) + BW;  // backward pairs
};

__device__ __forceinline__ df::Pair dpair(float h, float l) { return df::Pair{h, l}; }

// One step of either sweep from its packed record: HAS_A = the scale pair is
// present (primal forward, adjoint backward).
template <bool HAS_A, int BW>
__device__ __forceinline__ df::Pair df_row(float4 q, float2 q2, df::Pair F, df::Pair Y1, df::Pair Y2) {
  df::Pair A{1.f, 0.f}, B1, B2{0.f, 0.f};
  if (HAS_A) {
    A = dpair(q.x, q.y);
    B1 = dpair(q.z, q.w);
    if (BW == 2) B2 = dpair(q2.x, q2.y);
  } else {
    B1 = dpair(q.x, q.y);
    if (BW == 2) B2 = dpair(q.z, q.w);
  }
  return df::rec_step<HAS_A, BW>(A, F, B1, Y1, B2, Y2);
}

__device__ __forceinline__ double pair_to_f64(df::Pair p) { return (double)p.h + (double)p.l; }
// a forward value as 8 bytes: a pair (h, l) or an FP64 value
__device__ __forceinline__ uint2 pair_bits(df::Pair p) { return make_uint2(__float_as_uint(p.h), __float_as_uint(p.l)); }
__device__ __forceinline__ df::Pair bits_pair(uint2 b) { return dpair(__uint_as_float(b.x), __uint_as_float(b.y)); }
__device__ __forceinline__ uint2 f64_bits(double d) {
  return make_uint2((uint32_t)__double2loint(d), (uint32_t)__double2hiint(d));
}
__device__ __forceinline__ double bits_f64(uint2 b) { return __hiloint2double((int)b.y, (int)b.x); }

// Per-lane state of the V systems of a lane.
template <int V>
struct DfState {
  df::Pair p1[V], p2[V];  // last two recurrence values in pairs
  double d1[V], d2[V];    // ... in FP64 (after a switch)
  bool f64;               // this lane runs native FP64 from row rsw on
  int rsw;
  __device__ __forceinline__ void reset_values() {
#pragma unroll
    for (int v = 0; v < V; v++) {
      p1[v] = p2[v] = dpair(0.f, 0.f);
      d1[v] = d2[v] = 0.0;
    }
  }
  // periodic plans: sigma' = sum pw'_i f_i of the forward sweep in pairs
  // (the FP64 sigma = 2^-k sigma' after a switch), read by the backward sweep
  df::Pair sig[V];
  double dsig[V];
  __device__ __forceinline__ void reset_sigma() {
#pragma unroll
    for (int v = 0; v < V; v++) {
      sig[v] = dpair(0.f, 0.f);
      dsig[v] = 0.0;
    }
  }
};

// s + (ch + cl) y in pairs, unnormalised: the product a TwoProduct of the high
// parts plus both cross terms, the sum a TwoSum of the high parts
__device__ __forceinline__ df::Pair df_muladd(df::Pair s, float ch, float cl, df::Pair y) {
  const float p = df::mul(ch, y.h);
  float e = df::fma_(ch, y.h, -p);
  e = df::fma_(ch, y.l, e);
  e = df::fma_(cl, y.h, e);
  float h, t;
  df::two_sum(s.h, p, h, t);
  return dpair(h, df::add(s.l, df::add(t, e)));
}

// Periodic plans keep inputs below 2^80 in pairs (their correction term
// sigma pc_i then stays inside FP32); larger ones go to FP64.
__device__ __forceinline__ bool df_per_small(double f) {
  return ((uint32_t)__double2hiint(f) & 0x7fffffffu) < ((1023u + 80u) << 20);
}

// Forward group: rows i0 .. i0+n-1 (FULL: n == U), FP64 inputs f; out: the
// forward values as 8-byte patterns (pairs, or FP64 from rsw on).
template <int BW, bool ADJ, int V, int U, bool FULL, bool PER = false>
__device__ __forceinline__ void df_fwd_group(const DfRecs& rc, const Coefs<double>& c64, int i0, int n,
                                             double (&f)[U][V], uint2 (&out)[U][V], DfState<V>& st) {
  constexpr bool F2 = DfCount<ADJ, BW>::F > 2;
  // the rows' coefficient records first: their shared-memory latency
  // overlaps the splits below
  float4 q[U];
  float2 q2[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    const int i = (FULL || u < n) ? i0 + u : i0;
    q[u] = rc.f4[i];
    q2[u] = F2 ? rc.f2[i] : make_float2(0.f, 0.f);
  }
  df::Pair y[U][V];
  bool need = false;
  if (!st.f64) {
#pragma unroll
    for (int u = 0; u < U; u++)
#pragma unroll
      for (int v = 0; v < V; v++) {
        y[u][v] = dpair(0.f, 0.f);
        if (FULL || u < n) need |= !df::split_fast(f[u][v], y[u][v]) || (PER && !df_per_small(f[u][v]));
      }
  }
  if (__any_sync(__activemask(), need)) {
    if (need) {  // zeros or range edges: the careful split, or the switch to FP64
      bool bad = false;
#pragma unroll
      for (int u = 0; u < U; u++)
#pragma unroll
        for (int v = 0; v < V; v++) {
          bool ok = true;
          if (FULL || u < n) {
            y[u][v] = df::split(f[u][v], ok);
            if (PER) ok = ok && df_per_small(f[u][v]);
          }
          bad |= !ok;
        }
      if (bad) {
        st.f64 = true;
        st.rsw = i0;
#pragma unroll
        for (int v = 0; v < V; v++) {
          st.d1[v] = pair_to_f64(st.p1[v]);
          st.d2[v] = pair_to_f64(st.p2[v]);
          if (PER) st.dsig[v] = pair_to_f64(st.sig[v]) * rc.per_unscale;
        }
      }
    }
  }
  if constexpr (PER) {  // sigma += pw_i f_i outside the rows without correction terms (pw' in pairs)
    if (i0 < c64.per_lo || i0 + n > c64.per_hi) {
      if (!st.f64) {
#pragma unroll
        for (int u = 0; u < U; u++)
          if (FULL || u < n) {
            const float4 w = rc.pq[i0 + u];
#pragma unroll
            for (int v = 0; v < V; v++) st.sig[v] = df_muladd(st.sig[v], w.x, w.y, y[u][v]);
          }
      } else {
        per_dot<double, V, U>(c64, i0, n, f, st.dsig);
      }
    }
  }
  if (!st.f64) {
#pragma unroll
    for (int u = 0; u < U; u++)
      if (FULL || u < n)
#pragma unroll
        for (int v = 0; v < V; v++) {
          const df::Pair w = df_row<!ADJ, BW>(q[u], q2[u], y[u][v], st.p1[v], st.p2[v]);
          st.p2[v] = st.p1[v];
          st.p1[v] = w;
          out[u][v] = pair_bits(w);
        }
  } else {
    fwd_block<BW, ADJ, double, V, U, false>(c64, i0, n, f, st.d1, st.d2);
#pragma unroll
    for (int u = 0; u < U; u++)
#pragma unroll
      for (int v = 0; v < V; v++) out[u][v] = f64_bits(f[u][v]);
  }
}

// Backward group: rows top, top-1, .., top-n+1; in: their forward values as
// stored by df_fwd_group (8-byte patterns); x: the solution in FP64.
template <int BW, bool ADJ, int V, int U, bool FULL, bool PER = false>
__device__ __forceinline__ void df_bwd_group(const DfRecs& rc, const Coefs<double>& c64, int top, int n,
                                             const uint2 (&in)[U][V], double (&x)[U][V], DfState<V>& st) {
  constexpr bool B2 = DfCount<ADJ, BW>::B > 2;
  // periodic plans: x_i = y_i - sigma pc_i outside the rows without
  // correction terms (the recurrence keeps the uncorrected y)
  const bool corr = PER && (top + 1 - n < c64.per_lo || top + 1 > c64.per_hi);
  if (!st.f64) {
    float4 q[U];
    float2 q2[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int i = (FULL || u < n) ? top - u : top;
      q[u] = rc.b4[i];
      q2[u] = B2 ? rc.b2[i] : make_float2(0.f, 0.f);
    }
    df::Pair y[U][V];
    bool need = false;
#pragma unroll
    for (int u = 0; u < U; u++)
#pragma unroll
      for (int v = 0; v < V; v++) {
        y[u][v] = dpair(0.f, 0.f);
        if (FULL || u < n) {
          y[u][v] = df_row<ADJ, BW>(q[u], q2[u], bits_pair(in[u][v]), st.p1[v], st.p2[v]);
          st.p2[v] = st.p1[v];
          st.p1[v] = y[u][v];
          if (PER && corr) {
            const float4 w = rc.pq[top - u];
            const df::Pair z = df_muladd(y[u][v], -w.z, -w.w, st.sig[v]);
            df::fast_two_sum(z.h, z.l, y[u][v].h, y[u][v].l);
          }
          need |= !df::combine_ok(y[u][v].h);
        }
        x[u][v] = df::combine_fast(y[u][v].h, y[u][v].l);
      }
    // one FP64 addition per value; the integer conversion for values below
    // 2^-70 (zeros)
    if (__any_sync(__activemask(), need)) {
#pragma unroll
      for (int u = 0; u < U; u++)
#pragma unroll
        for (int v = 0; v < V; v++)
          if (!df::combine_ok(y[u][v].h)) x[u][v] = df::combine(y[u][v].h, y[u][v].l);
    }
  } else {
    if (top - (U - 1) >= st.rsw) {  // the whole group was stored in FP64
#pragma unroll
      for (int u = 0; u < U; u++)
#pragma unroll
        for (int v = 0; v < V; v++) x[u][v] = bits_f64(in[u][v]);
    } else {
#pragma unroll
      for (int u = 0; u < U; u++)
#pragma unroll
        for (int v = 0; v < V; v++)
          x[u][v] = (top - u >= st.rsw) ? bits_f64(in[u][v]) : pair_to_f64(bits_pair(in[u][v]));
    }
    bwd_block<BW, ADJ, double, V, U, false>(c64, top, n, x, st.d1, st.d2);
    if (PER && corr) per_fix<double, V, U>(c64, top, n, x, st.dsig);
  }
}

// V lane-rows of 8-byte values (pairs or FP64) in a ring slot or in memory
template <int V>
__device__ __forceinline__ void ld8(const void* p, uint2 (&o)[V]) {
  if constexpr (V == 2) {
    const uint4 t = *reinterpret_cast<const uint4*>(p);
    o[0] = make_uint2(t.x, t.y);
    o[1] = make_uint2(t.z, t.w);
  } else {
    o[0] = *reinterpret_cast<const uint2*>(p);
  }
}
template <int V>
__device__ __forceinline__ void st8(void* p, const uint2 (&x)[V]) {
  if constexpr (V == 2)
    *reinterpret_cast<uint4*>(p) = make_uint4(x[0].x, x[0].y, x[1].x, x[1].y);
  else
    *reinterpret_cast<uint2*>(p) = x[0];
}
template <int V>
__device__ __forceinline__ void ld_f64v(const void* p, double (&o)[V]) {
  if constexpr (V == 2) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    o[0] = t.x;
    o[1] = t.y;
  } else {
    o[0] = *reinterpret_cast<const double*>(p);
  }
}
template <int V>
__device__ __forceinline__ void st_f64v(void* p, const double (&x)[V]) {
  if constexpr (V == 2)
    *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
  else
    *reinterpret_cast<double*>(p) = x[0];
}

// The backward sweep of df_sweep_systems, after a forward sweep that left the
// forward values of rows 0 .. N-D-1 at pout (as 8-byte patterns) and those of
// rows N-D .. N-1 in the ring slots (row i in slot i % D), with st as the
// forward sweep left it (its switch row kept).
template <int BW, bool ADJ, int V, int D, bool PER = false>
__device__ __forceinline__ void df_sweep_backward(const DfRecs& rc, const Coefs<double>& c64, int N, double* pout,
                                                  int64_t M, unsigned char* ring, uint32_t ring_s, uint32_t pitch,
                                                  DfState<V>& st) {
  constexpr int U = 4;
  // backward sweep: rows N-1 .. N-D are in the ring; row i - D is requested
  // into the slot row i frees (blocks aligned to N - 1, one group each)
  const int tail = N - D;
  double* prow = pout + (int64_t)(N - 1) * M;
  const double* pback = pout + (int64_t)(N - 1 - D) * M;
  st.reset_values();
  auto bwd = [&](auto full_tag, int top) {
    constexpr bool FULL = decltype(full_tag)::value;
    const int n = FULL ? U : ((top + 1) < U ? (top + 1) : U);
    if (FULL || top - (n - 1) < tail) cp_wait<D / U - 1>();
    uint2 w[U][V];
    double x[U][V];
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (FULL || u < n)
        ld8<V>(ring + (size_t)((top - u) % D) * pitch, w[u]);
      else
#pragma unroll
        for (int v = 0; v < V; v++) w[u][v] = make_uint2(0u, 0u);
    }
    df_bwd_group<BW, ADJ, V, U, FULL, PER>(rc, c64, top, n, w, x, st);
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int i = top - u;
      if (FULL || u < n) {
        st_f64v<V>(prow, x[u]);
        if (FULL || i - D >= 0) copy_row<double, V>(ring_s + (i % D) * pitch, pback);
      }
      prow -= M;
      pback -= M;
    }
    cp_commit();
  };
  int top = N - 1;
#pragma unroll 1
  for (; top >= D + U - 1; top -= U) bwd(std::true_type{}, top);
#pragma unroll 1
  for (; top >= 0; top -= U) bwd(std::false_type{}, top);
  cp_wait<0>();
}

// The two sweeps of the V systems at pout (row stride M) through the
// lane's ring of D slots of 8 V bytes (ring: its first slot, generic and
// shared-window addresses; pitch: bytes between slots): rows 0..D-1 are
// requested up front, one copy group per block of U = 4 rows; the forward
// values go to pout in place as pairs, the last D stay in the ring; the
// backward sweep streams them back and writes X in FP64.
template <int BW, bool ADJ, int V, int D, bool PER = false>
__device__ __forceinline__ void df_sweep_systems(const DfRecs& rc, const Coefs<double>& c64, int N,
                                                 double* pout, int64_t M, unsigned char* ring,
                                                 uint32_t ring_s, uint32_t pitch) {
  constexpr int U = 4;  // rows per block; D is a multiple of U
  static_assert(D % U == 0, "ring depth must be a multiple of the block");
  DfState<V> st;
  st.reset_values();
  if (PER) st.reset_sigma();
  st.f64 = false;
  st.rsw = N;
  // forward sweep: rows 0..D-1 requested up front (one copy group per
  // block of U rows); each block then waits for its group, computes and
  // refills its slots with the rows D further down
  const double* pnext = pout;
#pragma unroll 1
  for (int r = 0; r < D; r++) {
    if (r < N) copy_row<double, V>(ring_s + r * pitch, pnext);
    pnext += M;
    if ((r + 1) % U == 0) cp_commit();
  }
  double* prow = pout;
  auto fwd = [&](auto full_tag, int i0) {
    constexpr bool FULL = decltype(full_tag)::value;
    cp_wait<D / U - 1>();
    const int n = FULL ? U : ((N - i0) < U ? (N - i0) : U);
    const int s0 = i0 % D;
    double f[U][V];
    uint2 w[U][V];
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (FULL || u < n)
        ld_f64v<V>(ring + (size_t)(s0 + u) * pitch, f[u]);
      else
#pragma unroll
        for (int v = 0; v < V; v++) f[u][v] = 0.0;
    }
    df_fwd_group<BW, ADJ, V, U, FULL, PER>(rc, c64, i0, n, f, w, st);
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int i = i0 + u;
      if (FULL || u < n) {
        const bool keep = !FULL && i + D >= N;  // tail row: stays in the ring
        st8<V>(keep ? static_cast<void*>(ring + (size_t)(s0 + u) * pitch) : static_cast<void*>(prow), w[u]);
        if (!keep) copy_row<double, V>(ring_s + (s0 + u) * pitch, pnext);
      }
      prow += M;
      pnext += M;
    }
    cp_commit();
  };
  int i0 = 0;
#pragma unroll 1
  for (; i0 + U + D <= N; i0 += U) fwd(std::true_type{}, i0);
#pragma unroll 1
  for (; i0 < N; i0 += U) fwd(std::false_type{}, i0);
  df_sweep_backward<BW, ADJ, V, D, PER>(rc, c64, N, pout, M, ring, ring_s, pitch, st);
}


}  // namespace bs
