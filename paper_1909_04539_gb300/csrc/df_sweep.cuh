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
};

// Forward group: rows i0 .. i0+n-1 (FULL: n == U), FP64 inputs f; out: the
// forward values as 8-byte patterns (pairs, or FP64 from rsw on).
template <int BW, bool ADJ, int V, int U, bool FULL>
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
        if (FULL || u < n) need |= !df::split_fast(f[u][v], y[u][v]);
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
          if (FULL || u < n) y[u][v] = df::split(f[u][v], ok);
          bad |= !ok;
        }
      if (bad) {
        st.f64 = true;
        st.rsw = i0;
#pragma unroll
        for (int v = 0; v < V; v++) {
          st.d1[v] = pair_to_f64(st.p1[v]);
          st.d2[v] = pair_to_f64(st.p2[v]);
        }
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
template <int BW, bool ADJ, int V, int U, bool FULL>
__device__ __forceinline__ void df_bwd_group(const DfRecs& rc, const Coefs<double>& c64, int top, int n,
                                             const uint2 (&in)[U][V], double (&x)[U][V], DfState<V>& st) {
  constexpr bool B2 = DfCount<ADJ, BW>::B > 2;
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
  }
}

}  // namespace bs
