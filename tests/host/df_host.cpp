// Host build of the pair-arithmetic header the FP64-accurate FP32-pair
// sweeps use (paper_1909_04539_gb300/csrc/df_math.cuh), for CPU tests of its
// conversions and of the two sweeps as the kernel runs them (same operations
// in the same order, IEEE single precision, no contraction).
#include "../../paper_1909_04539_gb300/csrc/df_math.cuh"

using namespace bs::df;

static void sweep_impl(const double* s, const double* l1, const double* l2, const double* t, const double* u1,
                       const double* u2, int has_s, int has_t, int bw, long N, const double* f, double* x) {
  auto P = [](double c) {
    const float h = (float)c;
    return Pair{h, (float)(c - (double)h)};
  };
  Pair* w = new Pair[N];
  const Pair z{0.f, 0.f};
  for (long i = 0; i < N; i++) {
    bool ok = true;
    const Pair F = split(f[i], ok);
    const Pair Y1 = i >= 1 ? w[i - 1] : z, Y2 = i >= 2 ? w[i - 2] : z;
    const Pair B2 = bw == 2 ? P(l2[i]) : z;
    w[i] = has_s ? (bw == 2 ? rec_step<true, 2>(P(s[i]), F, P(l1[i]), Y1, B2, Y2)
                            : rec_step<true, 1>(P(s[i]), F, P(l1[i]), Y1, B2, Y2))
                 : (bw == 2 ? rec_step<false, 2>(Pair{1.f, 0.f}, F, P(l1[i]), Y1, B2, Y2)
                            : rec_step<false, 1>(Pair{1.f, 0.f}, F, P(l1[i]), Y1, B2, Y2));
  }
  Pair x1 = z, x2 = z;
  for (long i = N - 1; i >= 0; i--) {
    const Pair B2 = bw == 2 ? P(u2[i]) : z;
    const Pair y = has_t ? (bw == 2 ? rec_step<true, 2>(P(t[i]), w[i], P(u1[i]), x1, B2, x2)
                                    : rec_step<true, 1>(P(t[i]), w[i], P(u1[i]), x1, B2, x2))
                         : (bw == 2 ? rec_step<false, 2>(Pair{1.f, 0.f}, w[i], P(u1[i]), x1, B2, x2)
                                    : rec_step<false, 1>(Pair{1.f, 0.f}, w[i], P(u1[i]), x1, B2, x2));
    x2 = x1;
    x1 = y;
    x[i] = combine(y.h, y.l);
  }
  delete[] w;
}

// s + (ch + cl) y in pairs, unnormalised, in the operation order of the
// periodic pair sweeps (TwoProduct of the high parts plus both cross terms,
// TwoSum of the high parts)
static Pair muladd(Pair s, float ch, float cl, Pair y) {
  const float p = mul(ch, y.h);
  float e = fma_(ch, y.h, -p);
  e = fma_(ch, y.l, e);
  e = fma_(cl, y.h, e);
  float h, t;
  two_sum(s.h, p, h, t);
  return Pair{h, add(s.l, add(t, e))};
}

extern "C" {

// x[n] -> h[n], l[n], ok[n]
void df_split(const double* x, float* h, float* l, int* ok, long n) {
  for (long i = 0; i < n; i++) {
    bool o = false;
    const Pair p = split(x[i], o);
    h[i] = p.h;
    l[i] = p.l;
    ok[i] = o ? 1 : 0;
  }
}

void df_combine(const float* h, const float* l, double* out, long n) {
  for (long i = 0; i < n; i++) out[i] = combine(h[i], l[i]);
}

// split_fast: ok[i] = 1 where the fast path applies (then h, l as split())
void df_split_fast(const double* x, float* h, float* l, int* ok, long n) {
  for (long i = 0; i < n; i++) {
    Pair p{0.f, 0.f};
    ok[i] = split_fast(x[i], p) ? 1 : 0;
    h[i] = p.h;
    l[i] = p.l;
  }
}

// combine_fast where combine_ok, else -1 in ok
void df_combine_fast(const float* h, const float* l, double* out, int* ok, long n) {
  for (long i = 0; i < n; i++) {
    ok[i] = combine_ok(h[i]) ? 1 : 0;
    out[i] = ok[i] ? combine_fast(h[i], l[i]) : 0.0;
  }
}

void df_two_sum(const float* a, const float* b, float* s, float* t, long n) {
  for (long i = 0; i < n; i++) two_sum(a[i], b[i], s[i], t[i]);
}

// One system of the recurrence pair in pair arithmetic (coefficient arrays of
// N doubles, split into pairs as the handle does; has_s / has_t: the scale
// coefficient is present; bw = 1 or 2), input f (N doubles, all in range),
// output x (N doubles).
void df_sweep(const double* s, const double* l1, const double* l2, const double* t, const double* u1,
              const double* u2, int has_s, int has_t, int bw, long N, const double* f, double* x) {
  sweep_impl(s, l1, l2, t, u1, u2, has_s, has_t, bw, N, f, x);
}

// One system of a periodic tridiagonal solve in pair arithmetic, as the
// periodic pair sweeps run it (Sherman-Morrison, Sec. 3.3): the tridiagonal
// recurrences of the corner-free matrix (coefficients as for df_sweep, bw 1),
// sigma' = sum pw'_i f_i accumulated in pairs during the forward sweep over
// the rows outside [per_lo, per_hi), and x_i = y_i - sigma' pc'_i formed in
// pairs after each backward row there, the recurrence keeping y.  pw, pc:
// the scaled weights as (hi, lo) float pairs (4 N floats: pw hi, pw lo, pc
// hi, pc lo per row).
void df_sweep_periodic(const double* s, const double* l1, const double* t, const double* u1, int has_s, int has_t,
                       const float* pq, long per_lo, long per_hi, long N, const double* f, double* x) {
  auto P = [](double c) {
    const float h = (float)c;
    return Pair{h, (float)(c - (double)h)};
  };
  Pair* w = new Pair[N];
  const Pair z{0.f, 0.f};
  Pair sig{0.f, 0.f};
  for (long i = 0; i < N; i++) {
    bool ok = true;
    const Pair F = split(f[i], ok);
    if (i < per_lo || i >= per_hi) sig = muladd(sig, pq[4 * i], pq[4 * i + 1], F);
    const Pair Y1 = i >= 1 ? w[i - 1] : z;
    w[i] = has_s ? rec_step<true, 1>(P(s[i]), F, P(l1[i]), Y1, z, z)
                 : rec_step<false, 1>(Pair{1.f, 0.f}, F, P(l1[i]), Y1, z, z);
  }
  Pair x1 = z;
  for (long i = N - 1; i >= 0; i--) {
    Pair y = has_t ? rec_step<true, 1>(P(t[i]), w[i], P(u1[i]), x1, z, z)
                   : rec_step<false, 1>(Pair{1.f, 0.f}, w[i], P(u1[i]), x1, z, z);
    x1 = y;
    if (i < per_lo || i >= per_hi) {
      const Pair c = muladd(y, -pq[4 * i + 2], -pq[4 * i + 3], sig);
      fast_two_sum(c.h, c.l, y.h, y.l);
    }
    x[i] = combine(y.h, y.l);
  }
  delete[] w;
}

// One Crank-Nicolson step C <- A^{-1} (2I - A) C of one system as the fused
// pair kernel runs it: the explicit side f_i = 2 C_i - sum_k A(i, i+k-h)
// C_{i+k-h} in pairs (each band entry as a (hi, lo) pair, each product a
// TwoProduct of the high parts plus the cross terms, the sum TwoSums of the
// high parts with the rest in the low part, renormalised), then the pair
// solve of A (plan coefficients as for df_sweep).  bands: width x N doubles
// (row k = entries A(i, i+k-h), zero outside the matrix unless periodic);
// periodic (width 3): the window wraps around and pq, per_lo, per_hi carry
// the Sherman-Morrison weights as for df_sweep_periodic.
void df_cn_step(const double* bands, int width, int periodic, const double* s, const double* l1, const double* l2,
                const double* u1, const double* u2, const float* pq, long per_lo, long per_hi, long N,
                const double* c, double* x) {
  auto P = [](double v) {
    const float h = (float)v;
    return Pair{h, (float)(v - (double)h)};
  };
  const int h = width / 2;
  const int bw = h;
  Pair* y = new Pair[N];
  Pair* w = new Pair[N];
  for (long i = 0; i < N; i++) {
    bool ok = true;
    y[i] = split(c[i], ok);
  }
  const Pair z{0.f, 0.f};
  Pair sig{0.f, 0.f};
  for (long i = 0; i < N; i++) {
    float sh = mul(2.f, y[i].h), lo = mul(2.f, y[i].l);
    for (int k = 0; k < width; k++) {
      long j = i + k - h;
      Pair zz = z;
      if (j >= 0 && j < N)
        zz = y[j];
      else if (periodic)
        zz = y[(j + N) % N];
      const Pair cp = P(bands[(long)k * N + i]);
      const float p = mul(cp.h, zz.h);
      float e = fma_(cp.h, zz.h, -p);
      e = fma_(cp.h, zz.l, e);
      e = fma_(cp.l, zz.h, e);
      float t;
      two_sum(sh, -p, sh, t);
      lo = add(lo, sub(t, e));
    }
    Pair f;
    fast_two_sum(sh, lo, f.h, f.l);
    if (periodic && (i < per_lo || i >= per_hi)) sig = muladd(sig, pq[4 * i], pq[4 * i + 1], f);
    const Pair Y1 = i >= 1 ? w[i - 1] : z, Y2 = i >= 2 ? w[i - 2] : z;
    const Pair B2 = bw == 2 ? P(l2[i]) : z;
    w[i] = bw == 2 ? rec_step<true, 2>(P(s[i]), f, P(l1[i]), Y1, B2, Y2)
                   : rec_step<true, 1>(P(s[i]), f, P(l1[i]), Y1, B2, Y2);
  }
  Pair x1 = z, x2 = z;
  for (long i = N - 1; i >= 0; i--) {
    const Pair B2 = bw == 2 ? P(u2[i]) : z;
    Pair v = bw == 2 ? rec_step<false, 2>(Pair{1.f, 0.f}, w[i], P(u1[i]), x1, B2, x2)
                     : rec_step<false, 1>(Pair{1.f, 0.f}, w[i], P(u1[i]), x1, B2, x2);
    x2 = x1;
    x1 = v;
    if (periodic && (i < per_lo || i >= per_hi)) {
      const Pair cc = muladd(v, -pq[4 * i + 2], -pq[4 * i + 3], sig);
      fast_two_sum(cc.h, cc.l, v.h, v.l);
    }
    x[i] = combine(v.h, v.l);
  }
  delete[] y;
  delete[] w;
}

}  // extern "C"
