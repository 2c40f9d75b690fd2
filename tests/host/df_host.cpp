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

}  // extern "C"
