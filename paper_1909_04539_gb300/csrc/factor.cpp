// Host side of the library: one-off FP64 factorisation of the shared LHS,
// handle lifetime, error reporting.
//
// The factorisation is done once on the host in FP64, as in the paper
// ("pre-factorisation step for the single LHS performed on the CPU", Sec. 2),
// and turned into the per-row sweep coefficients the kernels read.  Divisions
// by pivots are replaced by stored reciprocals so the sweeps contain no
// divides; every coefficient is a plain FP64 expression of the paper's
// factors, rounded once more to FP32 for the reduced-precision sweeps.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "internal.h"

namespace bs {

static thread_local std::string g_last_error = "no error";
static std::mutex g_handles_mu;
static std::set<bs_handle> g_handles;

bs_status set_error(bs_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

bs_status cuda_error(cudaError_t e, const char* what) {
  return set_error(BS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool valid_handle(bs_handle h) {
  std::lock_guard<std::mutex> lk(g_handles_mu);
  return h != nullptr && g_handles.count(h) != 0;
}

bool handle_ref(bs_handle h) {
  std::lock_guard<std::mutex> lk(g_handles_mu);
  if (h == nullptr || g_handles.count(h) == 0) return false;
  h->server_refs++;
  return true;
}

void handle_unref(bs_handle h) {
  std::lock_guard<std::mutex> lk(g_handles_mu);
  if (h != nullptr && g_handles.count(h) != 0 && h->server_refs > 0) h->server_refs--;
}

const DeviceInfo& device_info() {
  static DeviceInfo info[64];
  static bool have[64] = {false};
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  std::lock_guard<std::mutex> lk(mu);
  if (!have[dev]) {
    DeviceInfo d{};
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&d.l2_bytes, cudaDevAttrL2CacheSize, dev);
    cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (d.sms <= 0) d.sms = 1;
    info[dev] = d;
    have[dev] = true;
  }
  return info[dev];
}

}  // namespace bs

using namespace bs;

namespace {

// Host copies of one plan before upload: C_COUNT arrays of N.
struct HostPlan {
  int bw = 1;
  bool fwd_scale = false, bwd_scale = false, periodic = false;
  int per_lo = 0, per_hi = 0;
  bool uniform = false;  // see SweepPlan
  double eps = 0.0;
  std::vector<double> c;
};

bool bad(double v) { return v == 0.0 || !std::isfinite(v); }

// Thomas pre-factorisation (Sec. 3.1): pivots p_i = b_i - a_i chat_{i-1}
// (p_1 = b_1), chat_i = c_i / p_i, with c_N taken as 0.  Returns the row of
// the first bad pivot (1-based) or 0.
int64_t tri_factor(const double* a, const double* b, const double* c, int64_t N,
                   std::vector<double>& r, std::vector<double>& chat) {
  r.assign(N, 0.0);
  chat.assign(N, 0.0);
  for (int64_t i = 0; i < N; i++) {
    const double p = (i == 0) ? b[0] : b[i] - a[i] * chat[i - 1];
    if (bad(p)) return i + 1;
    r[i] = 1.0 / p;
    chat[i] = (i + 1 < N) ? c[i] * r[i] : 0.0;
  }
  return 0;
}

// Pentadiagonal A = L R (Sec. 4.1), written as one loop over rows with the
// entries that fall outside the matrix read as zero; this reproduces the
// paper's special-cased first, second, (N-1)-th and N-th rows.
int64_t penta_factor(const double* const* bd, int64_t N, std::vector<double>& al,
                     std::vector<double>& be, std::vector<double>& ga, std::vector<double>& de,
                     std::vector<double>& ep) {
  al.assign(N, 0.0);
  be.assign(N, 0.0);
  ga.assign(N, 0.0);
  de.assign(N, 0.0);
  ep.assign(N, 0.0);
  auto at = [&](int k, int64_t i) { return bd[k][i]; };
  for (int64_t i = 0; i < N; i++) {
    const double a = (i >= 2) ? at(0, i) : 0.0;
    const double b = (i >= 1) ? at(1, i) : 0.0;
    const double c = at(2, i);
    const double d = (i + 1 < N) ? at(3, i) : 0.0;
    const double e = (i + 2 < N) ? at(4, i) : 0.0;
    const double ga2 = (i >= 2) ? ga[i - 2] : 0.0, de2 = (i >= 2) ? de[i - 2] : 0.0;
    const double ga1 = (i >= 1) ? ga[i - 1] : 0.0, de1 = (i >= 1) ? de[i - 1] : 0.0;
    ep[i] = a;
    be[i] = b - a * ga2;
    al[i] = c - a * de2 - be[i] * ga1;
    if (bad(al[i])) return i + 1;
    ga[i] = (d - be[i] * de1) / al[i];
    de[i] = e / al[i];
  }
  return 0;
}

// Sweep coefficients of the primal (A^{-1}) and adjoint (A^{-T}) solves.
// Returns the 1-based row of a bad pivot, or 0.
int64_t make_plans(const double* const* bd, int width, int64_t N, HostPlan& P, HostPlan& Q,
                   std::vector<double>* entries = nullptr) {
  auto C = [&](HostPlan& p, int k, int64_t i) -> double& { return p.c[(size_t)k * N + i]; };
  if (width == 3) {
    std::vector<double> r, chat;
    const int64_t bad_row = tri_factor(bd[0], bd[1], bd[2], N, r, chat);
    if (bad_row) return bad_row;
    // primal: dhat_i = r_i d_i - (a_i r_i) dhat_{i-1};  x_i = dhat_i - chat_i x_{i+1}
    P.bw = 1;
    P.fwd_scale = true;
    P.bwd_scale = false;
    for (int64_t i = 0; i < N; i++) {
      C(P, C_S, i) = r[i];
      C(P, C_L1, i) = (i > 0) ? bd[0][i] * r[i] : 0.0;
      C(P, C_T, i) = 1.0;
      C(P, C_U1, i) = chat[i];
    }
    // adjoint, A^T = U^T L^T with L = (p_i diag, a_i sub), U = (1, chat_i super):
    // z_i = g_i - chat_{i-1} z_{i-1};  y_i = r_i z_i - (a_{i+1} r_i) y_{i+1}
    Q.bw = 1;
    Q.fwd_scale = false;
    Q.bwd_scale = true;
    for (int64_t i = 0; i < N; i++) {
      C(Q, C_S, i) = 1.0;
      C(Q, C_L1, i) = (i > 0) ? chat[i - 1] : 0.0;
      C(Q, C_T, i) = r[i];
      C(Q, C_U1, i) = (i + 1 < N) ? bd[0][i + 1] * r[i] : 0.0;
    }
    if (entries) {  // the primal sweep coefficients s, l1, l2, u1, u2
      entries->assign((size_t)5 * N, 0.0);
      for (int64_t i = 0; i < N; i++) {
        (*entries)[0 * N + i] = C(P, C_S, i);
        (*entries)[1 * N + i] = C(P, C_L1, i);
        (*entries)[3 * N + i] = C(P, C_U1, i);
      }
    }
    return 0;
  }
  std::vector<double> al, be, ga, de, ep;
  const int64_t bad_row = penta_factor(bd, N, al, be, ga, de, ep);
  if (bad_row) return bad_row;
  // primal: g_i = f_i/al_i - (ep_i/al_i) g_{i-2} - (be_i/al_i) g_{i-1};
  //         x_i = g_i - ga_i x_{i+1} - de_i x_{i+2}
  P.bw = 2;
  P.fwd_scale = true;
  P.bwd_scale = false;
  for (int64_t i = 0; i < N; i++) {
    const double ia = 1.0 / al[i];
    C(P, C_S, i) = ia;
    C(P, C_L1, i) = (i >= 1) ? be[i] * ia : 0.0;
    C(P, C_L2, i) = (i >= 2) ? ep[i] * ia : 0.0;
    C(P, C_T, i) = 1.0;
    C(P, C_U1, i) = (i + 1 < N) ? ga[i] : 0.0;
    C(P, C_U2, i) = (i + 2 < N) ? de[i] : 0.0;
  }
  // adjoint, A^T = R^T L^T:
  // z_i = g_i - ga_{i-1} z_{i-1} - de_{i-2} z_{i-2};
  // y_i = z_i/al_i - (be_{i+1}/al_i) y_{i+1} - (ep_{i+2}/al_i) y_{i+2}
  Q.bw = 2;
  Q.fwd_scale = false;
  Q.bwd_scale = true;
  for (int64_t i = 0; i < N; i++) {
    const double ia = 1.0 / al[i];
    C(Q, C_S, i) = 1.0;
    C(Q, C_L1, i) = (i >= 1) ? ga[i - 1] : 0.0;
    C(Q, C_L2, i) = (i >= 2) ? de[i - 2] : 0.0;
    C(Q, C_T, i) = ia;
    C(Q, C_U1, i) = (i + 1 < N) ? be[i + 1] * ia : 0.0;
    C(Q, C_U2, i) = (i + 2 < N) ? ep[i + 2] * ia : 0.0;
  }
  if (entries) {  // the primal sweep coefficients s, l1, l2, u1, u2
    entries->assign((size_t)5 * N, 0.0);
    const int idx[5] = {C_S, C_L1, C_L2, C_U1, C_U2};
    for (int k = 0; k < 5; k++)
      for (int64_t i = 0; i < N; i++) (*entries)[(size_t)k * N + i] = C(P, idx[k], i);
  }
  return 0;
}

void free_handle(bs_handle h) {
  if (!h) return;
  for (auto& p : h->plan) {
    if (p.c64) cudaFree(p.c64);
    if (p.c32) cudaFree(p.c32);
    if (p.dfrec) cudaFree(p.dfrec);
    if (p.dfper) cudaFree(p.dfper);
    if (p.rec32) cudaFree(p.rec32);
  }
  if (h->bands64) cudaFree(h->bands64);
  if (h->bands_hi) cudaFree(h->bands_hi);
  if (h->bands_lo) cudaFree(h->bands_lo);
  if (h->lu_hi) cudaFree(h->lu_hi);
  if (h->lu_lo) cudaFree(h->lu_lo);
  for (auto& p : h->tplan) {
    if (p.c64) cudaFree(p.c64);
    if (p.c32) cudaFree(p.c32);
  }
  for (auto& pp : h->part) {
    if (pp.blk.c64) cudaFree(pp.blk.c64);
    if (pp.blk.c32) cudaFree(pp.blk.c32);
    for (void* ptr : {(void*)pp.spk64, (void*)pp.spk32, (void*)pp.red64, (void*)pp.red32})
      if (ptr) cudaFree(ptr);
  }
  delete h;
}

// Applies one host plan to a single right-hand side in FP64 (the same
// recurrence pair the kernels run), in place.
void apply_plan(const HostPlan& p, int64_t N, std::vector<double>& x) {
  auto C = [&](int k, int64_t i) { return p.c[(size_t)k * N + i]; };
  for (int64_t i = 0; i < N; i++) {
    double w = p.fwd_scale ? C(C_S, i) * x[i] : x[i];
    if (i >= 1) w -= C(C_L1, i) * x[i - 1];
    if (p.bw == 2 && i >= 2) w -= C(C_L2, i) * x[i - 2];
    x[i] = w;
  }
  for (int64_t i = N - 1; i >= 0; i--) {
    double v = p.bwd_scale ? C(C_T, i) * x[i] : x[i];
    if (i + 1 < N) v -= C(C_U1, i) * x[i + 1];
    if (p.bw == 2 && i + 2 < N) v -= C(C_U2, i) * x[i + 2];
    x[i] = v;
  }
}

// Host side of a row partition (see PartPlan) of the banded matrix with
// half-width h = width / 2 given by its bands (outside entries ignored).
struct HostPart {
  int P = 0, L = 0, R = 0, kv = 0, kw = 0, h = 0, p = 0, q = 0;
  HostPlan blk;
  std::vector<double> spk;  // 2h x N: V_1 .. V_h, then W_1 .. W_h
  std::vector<double> red;  // (p + q + 1) x R: reduced-system LU (see PartPlan)
};

// Rows per block at least this many; blocks at most kPartMax.
constexpr int kPartMinRows = 192;
constexpr int kPartMax = 32;

bool make_partition(const double* const* bd, int width, int64_t N, HostPart& hp) {
  const int h = width / 2;
  int P = 1;
  while (P * 2 <= kPartMax && (int64_t)P * 2 * kPartMinRows <= N) P *= 2;
  if (P < 2) return false;
  const int64_t L = (N + P - 1) / P;
  P = (int)((N + L - 1) / L);
  if (P < 2) return false;
  auto top = [&](int k) { return (int64_t)k * L; };
  auto bot = [&](int k) { return std::min<int64_t>(N, (int64_t)(k + 1) * L) - 1; };
  auto blk_of = [&](int64_t i) { return (int)(i / L); };
  // band k of row i as a matrix entry at column i + k - h (0 outside)
  auto band = [&](int k, int64_t i) -> double {
    const int64_t col = i + k - h;
    return (col >= 0 && col < N) ? bd[k][i] : 0.0;
  };
  // block-diagonal matrix: every entry whose row and column lie in
  // different blocks removed
  std::vector<double> mod((size_t)width * N);
  for (int k = 0; k < width; k++)
    for (int64_t i = 0; i < N; i++) {
      const int64_t col = i + k - h;
      const bool inside = col >= 0 && col < N && blk_of(col) == blk_of(i);
      mod[(size_t)k * N + i] = inside ? bd[k][i] : 0.0;
    }
  const double* mbd[5];
  for (int k = 0; k < width; k++) mbd[k] = mod.data() + (size_t)k * N;
  HostPlan bq;
  hp.blk.c.assign((size_t)C_COUNT * N, 0.0);
  bq.c.assign((size_t)C_COUNT * N, 0.0);
  if (make_plans(mbd, width, N, hp.blk, bq)) return false;
  // spikes: V_m = A_blk^{-1} (the removed entries of column top - m, every
  // block), W_m likewise for column bot + m
  std::vector<std::vector<double>> V(h, std::vector<double>(N, 0.0)), W(h, std::vector<double>(N, 0.0));
  for (int m = 1; m <= h; m++) {
    for (int b = 0; b < P; b++) {
      for (int64_t i = top(b); i < std::min<int64_t>(N, top(b) + h); i++) {
        const int k = (int)(top(b) - m - i + h);
        if (b > 0 && k >= 0 && k < width) V[m - 1][i] += band(k, i);
      }
      for (int64_t i = std::max<int64_t>(0, bot(b) - h + 1); i <= bot(b); i++) {
        const int k = (int)(bot(b) + m - i + h);
        if (b < P - 1 && k >= 0 && k < width) W[m - 1][i] += band(k, i);
      }
    }
    apply_plan(hp.blk, N, V[m - 1]);
    apply_plan(hp.blk, N, W[m - 1]);
  }
  // entries below 2^-60 of a spike's maximum are dropped (each x_i gets at
  // most 2h such terms, so nothing changes above rounding)
  int64_t kv = 0, kw = 0;
  for (auto* set : {&V, &W})
    for (auto& vec : *set) {
      double mx = 0.0;
      for (double v : vec) mx = std::fmax(mx, std::fabs(v));
      for (double& v : vec)
        if (std::fabs(v) <= mx * 0x1p-60) v = 0.0;
    }
  for (int b = 0; b < P; b++)
    for (int64_t i = top(b); i <= bot(b); i++)
      for (int m = 0; m < h; m++) {
        if (V[m][i] != 0.0) kv = std::max<int64_t>(kv, i - top(b) + 1);
        if (W[m][i] != 0.0) kw = std::max<int64_t>(kw, bot(b) - i + 1);
      }
  // the correction is meant to touch a small part of each block
  if (kv + kw > L / 2) return false;
  // Reduced system: per block edge b the unknowns x at rows bot(b)-h+1 ..
  // bot(b) and top(b+1) .. top(b+1)+h-1 (in row order), z index 2h b + t.
  // Row r of block k: x_r + sum_m V_m(r) x_{top(k)-m} + sum_m W_m(r) x_{bot(k)+m} = y_r.
  const int R = 2 * h * (P - 1);
  auto zrow = [&](int zi) -> int64_t {
    const int b = zi / (2 * h), t = zi % (2 * h);
    return t < h ? bot(b) - h + 1 + t : top(b + 1) + (t - h);
  };
  std::vector<double> A((size_t)R * R, 0.0);
  for (int zi = 0; zi < R; zi++) {
    const int64_t r = zrow(zi);
    const int k = blk_of(r);
    A[(size_t)zi * R + zi] = 1.0;
    for (int m = 1; m <= h; m++) {
      if (k >= 1) A[(size_t)zi * R + (2 * h * (k - 1) + h - m)] += V[m - 1][r];
      if (k <= P - 2) A[(size_t)zi * R + (2 * h * k + h + m - 1)] += W[m - 1][r];
    }
  }
  int pl = 0, qu = 0;  // lower and upper bandwidth
  for (int i = 0; i < R; i++)
    for (int j = 0; j < R; j++)
      if (A[(size_t)i * R + j] != 0.0) {
        pl = std::max(pl, i - j);
        qu = std::max(qu, j - i);
      }
  if (pl > 3 * h - 1 || qu > 3 * h - 1) return false;  // the kernels' fixed band limit
  // LU without pivoting (the fill stays inside the band)
  for (int c = 0; c < R; c++) {
    const double piv = A[(size_t)c * R + c];
    if (bad(piv)) return false;
    for (int i = c + 1; i <= std::min(R - 1, c + pl); i++) {
      const double l = A[(size_t)i * R + c] / piv;
      A[(size_t)i * R + c] = l;
      for (int j = c + 1; j <= std::min(R - 1, c + qu); j++) A[(size_t)i * R + j] -= l * A[(size_t)c * R + j];
    }
  }
  // layout: [0, p): L multipliers of columns i-1 .. i-p; [p]: 1 / U_ii;
  // [p+1, p+q+1): U entries of columns i+1 .. i+q
  hp.red.assign((size_t)(pl + qu + 1) * R, 0.0);
  for (int i = 0; i < R; i++) {
    for (int k = 1; k <= pl; k++)
      if (i - k >= 0) hp.red[(size_t)(k - 1) * R + i] = A[(size_t)i * R + (i - k)];
    hp.red[(size_t)pl * R + i] = 1.0 / A[(size_t)i * R + i];
    for (int k = 1; k <= qu; k++)
      if (i + k < R) hp.red[(size_t)(pl + k) * R + i] = A[(size_t)i * R + (i + k)];
  }
  hp.P = P;
  hp.L = (int)L;
  hp.R = R;
  hp.kv = (int)kv;
  hp.kw = (int)kw;
  hp.h = h;
  hp.p = pl;
  hp.q = qu;
  hp.spk.assign((size_t)2 * h * N, 0.0);
  for (int m = 0; m < h; m++) {
    std::copy(V[m].begin(), V[m].end(), hp.spk.begin() + (size_t)m * N);
    std::copy(W[m].begin(), W[m].end(), hp.spk.begin() + (size_t)(h + m) * N);
  }
  return true;
}

// Records of the FP32-pair sweeps (sweep_df.cu) of a primal (fwd_scale) or
// adjoint (bwd_scale) plan: each coefficient c as the pair (fl32(c),
// fl32(c - fl32(c))), per row and sweep the pairs present -- (s), l1, (l2)
// forward, (t), u1, (u2) backward -- the first two in a float4, the third in a
// float2 (layout of SweepPlan::dfrec).  Returns whether pair arithmetic is
// safe for the plan: every coefficient is zero or of magnitude in
// [2^-100, 2^100), and the sweep gains bound every intermediate by 2^24 times
// the largest input, so that inputs below 2^101 keep every value below 2^125.
// The gains follow the recurrences on magnitudes: with |f_i| <= 1,
// |w_i| <= W_i = |s_i| + |l1_i| W_{i-1} + |l2_i| W_{i-2} and
// |x_i| <= X_i = |t_i| W_i + |u1_i| X_{i+1} + |u2_i| X_{i+2}.
bool make_df_records(const HostPlan& hp, int64_t N, std::vector<float>& rec) {
  auto C = [&](int k, int64_t i) { return hp.c[(size_t)k * N + i]; };
  bool ok = true;
  auto pair = [&](double c, float& h, float& l) {
    const double a = std::fabs(c);
    if (!std::isfinite(c) || (c != 0.0 && (a < std::ldexp(1.0, -100) || a >= std::ldexp(1.0, 100)))) ok = false;
    h = (float)c;
    l = (float)(c - (double)h);
  };
  rec.assign((size_t)12 * N, 0.f);
  float* f4 = rec.data();
  float* b4 = f4 + 4 * N;
  float* f2 = b4 + 4 * N;
  float* b2 = f2 + 2 * N;
  const bool adj = hp.bwd_scale;
  for (int64_t i = 0; i < N; i++) {
    float v[6] = {0, 0, 0, 0, 0, 0};
    int n = 0;
    if (!adj) pair(C(C_S, i), v[0], v[1]), n = 2;
    pair(C(C_L1, i), v[n], v[n + 1]);
    n += 2;
    if (hp.bw == 2) pair(C(C_L2, i), v[n], v[n + 1]);
    for (int q = 0; q < 4; q++) f4[4 * i + q] = v[q];
    f2[2 * i] = v[4], f2[2 * i + 1] = v[5];
    for (float& x : v) x = 0.f;
    n = 0;
    if (adj) pair(C(C_T, i), v[0], v[1]), n = 2;
    pair(C(C_U1, i), v[n], v[n + 1]);
    n += 2;
    if (hp.bw == 2) pair(C(C_U2, i), v[n], v[n + 1]);
    for (int q = 0; q < 4; q++) b4[4 * i + q] = v[q];
    b2[2 * i] = v[4], b2[2 * i + 1] = v[5];
  }
  std::vector<double> W(N), X(N);
  double g = 0.0;
  for (int64_t i = 0; i < N; i++) {
    double w = adj ? 1.0 : std::fabs(C(C_S, i));
    if (i >= 1) w += std::fabs(C(C_L1, i)) * W[i - 1];
    if (i >= 2) w += std::fabs(C(C_L2, i)) * W[i - 2];
    W[i] = w;
    g = std::max(g, w);
  }
  for (int64_t i = N - 1; i >= 0; i--) {
    double x = (adj ? std::fabs(C(C_T, i)) : 1.0) * W[i];
    if (i + 1 < N) x += std::fabs(C(C_U1, i)) * X[i + 1];
    if (i + 2 < N) x += std::fabs(C(C_U2, i)) * X[i + 2];
    X[i] = x;
    g = std::max(g, x);
  }
  return ok && std::isfinite(g) && g <= std::ldexp(1.0, 24);
}

// The Sherman-Morrison weights of a periodic plan as FP32 pairs, per row
// (pw hi, pw lo, pc hi, pc lo) (layout of SweepPlan::dfper), scaled by an
// exact power of two: pw' = 2^k pw with max |pw'| in [1, 2), pc' = 2^-k pc,
// so that sigma' pc' = sigma pc (unscale = 2^-k).  Weights decay
// geometrically away from the first and last rows; the small ones may fall
// below the FP32 range and drop out, each changing x by less than 2^-120
// of max |f|.  Returns whether the pair sweeps may carry the correction:
// all weights finite, sum |pw'| <= 2^20 and max |pc'| in [2^-40, 2^20] (or
// zero), so that with inputs below 2^80 (the pair sweeps of a periodic plan
// take larger ones to FP64) sigma' stays below 2^100 and sigma' pc' below
// 2^120.
bool make_df_periodic(const HostPlan& hp, int64_t N, std::vector<float>& rec, double& unscale) {
  bool ok = true;
  double wmax = 0.0, cmax = 0.0;
  for (int64_t i = 0; i < N; i++) {
    const double w = hp.c[(size_t)C_PW * N + i], c = hp.c[(size_t)C_PC * N + i];
    if (!std::isfinite(w) || !std::isfinite(c)) ok = false;
    wmax = std::fmax(wmax, std::fabs(w));
    cmax = std::fmax(cmax, std::fabs(c));
  }
  const int k = (ok && wmax > 0.0) ? -std::ilogb(wmax) : 0;
  unscale = std::ldexp(1.0, -k);
  double sum = 0.0;
  rec.assign((size_t)4 * N, 0.f);
  for (int64_t i = 0; i < N && ok; i++) {
    const double w = std::ldexp(hp.c[(size_t)C_PW * N + i], k), c = std::ldexp(hp.c[(size_t)C_PC * N + i], -k);
    sum += std::fabs(w);
    const float wh = (float)w, ch = (float)c;
    rec[4 * i] = wh;
    rec[4 * i + 1] = (float)(w - (double)wh);
    rec[4 * i + 2] = ch;
    rec[4 * i + 3] = (float)(c - (double)ch);
  }
  const double cm = std::ldexp(cmax, -k);
  return ok && k > -1000 && k < 1000 && sum <= 0x1p20 && (cmax == 0.0 || (cm >= 0x1p-40 && cm <= 0x1p20));
}

// Window lengths of the windowed sweeps (sweep_win.cu) of one plan.  A
// backward sweep started from zero at row e instead of from the true x_e,
// x_{e+1} is off at row j < e by psi1_j x_e + psi2_j x_{e+1}, where psi1,
// psi2 follow the homogeneous recurrence psi_j = -u1_j psi_{j+1} - u2_j
// psi_{j+2} from (1, 0) and (0, 1).  The window for a threshold is the
// largest, over every e, distance e - j at which |psi1_j| + |psi2_j| is still
// above it, for rows up to `cap` above e; 0 if the responses are above it
// anywhere between cap and 2 cap rows above some e (no decay within reach).
// The window is measured for every e, so it holds for any block size.
void make_windows(const HostPlan& hp, int64_t N, int cap32, int capdf, int& w32, int& wdf) {
  w32 = wdf = 0;
  if (N > ((int64_t)1 << 20) || hp.periodic) return;
  auto C = [&](int k, int64_t i) { return hp.c[(size_t)k * N + i]; };
  const double t32 = std::ldexp(1.0, -28), tdf = std::ldexp(1.0, -50);
  const int cap = std::max(cap32, capdf);
  int m32 = 0, mdf = 0;
  bool ok32 = true, okdf = true;
  std::vector<double> a(2 * cap + 3), b(2 * cap + 3);
  for (int64_t e = 1; e < N && (ok32 || okdf); e++) {
    // a[d], b[d]: responses at row e - d (d = 0: row e, d = -1: row e + 1)
    double a1 = 1.0, a2 = 0.0, b1 = 0.0, b2 = 1.0;  // values at rows j + 1, j + 2
    for (int d = 1; d <= 2 * cap && e - d >= 0; d++) {
      const int64_t j = e - d;
      const double u1 = C(C_U1, j), u2 = hp.bw == 2 ? C(C_U2, j) : 0.0;
      const double an = -u1 * a1 - u2 * a2, bn = -u1 * b1 - u2 * b2;
      a2 = a1, a1 = an, b2 = b1, b1 = bn;
      const double r = std::fabs(an) + (hp.bw == 2 ? std::fabs(bn) : 0.0);
      if (r > t32) {
        if (d > cap32) ok32 = false;
        m32 = std::max(m32, d);
      }
      if (r > tdf) {
        if (d > capdf) okdf = false;
        mdf = std::max(mdf, d);
      }
    }
  }
  w32 = ok32 ? std::max(m32, 1) : 0;
  wdf = okdf ? std::max(mdf, 1) : 0;
}

// FP32 records of the windowed FP32 sweeps (layout of SweepPlan::rec32).
void make_rec32(const HostPlan& hp, int64_t N, std::vector<float>& rec) {
  auto C = [&](int k, int64_t i) { return (float)hp.c[(size_t)k * N + i]; };
  rec.assign((size_t)8 * N, 0.f);
  for (int64_t i = 0; i < N; i++) {
    float* f = rec.data() + 4 * i;
    float* b = rec.data() + 4 * N + 4 * i;
    f[0] = hp.fwd_scale ? C(C_S, i) : 1.f;
    f[1] = C(C_L1, i);
    f[2] = hp.bw == 2 ? C(C_L2, i) : 0.f;
    b[0] = hp.bwd_scale ? C(C_T, i) : 1.f;
    b[1] = C(C_U1, i);
    b[2] = hp.bw == 2 ? C(C_U2, i) : 0.f;
  }
}

cudaError_t upload_plan(const HostPlan& hp, SweepPlan& sp, size_t& bytes) {
  sp.bw = hp.bw;
  sp.fwd_scale = hp.fwd_scale;
  sp.bwd_scale = hp.bwd_scale;
  sp.periodic = hp.periodic;
  sp.per_lo = hp.per_lo;
  sp.per_hi = hp.per_hi;
  sp.uniform = hp.uniform;
  sp.eps = hp.eps;
  std::vector<float> c32(hp.c.size());
  for (size_t q = 0; q < c32.size(); q++) c32[q] = (float)hp.c[q];
  cudaError_t e = cudaMalloc(&sp.c64, sizeof(double) * hp.c.size());
  if (e == cudaSuccess) e = cudaMalloc(&sp.c32, sizeof(float) * c32.size());
  if (e == cudaSuccess) e = cudaMemcpy(sp.c64, hp.c.data(), sizeof(double) * hp.c.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(sp.c32, c32.data(), sizeof(float) * c32.size(), cudaMemcpyHostToDevice);
  bytes += (sizeof(double) + sizeof(float)) * hp.c.size();
  return e;
}

cudaError_t upload_part(const HostPart& hp, int64_t N, PartPlan& pp, size_t& bytes) {
  pp.P = hp.P;
  pp.L = hp.L;
  pp.R = hp.R;
  pp.kv = hp.kv;
  pp.kw = hp.kw;
  pp.h = hp.h;
  pp.p = hp.p;
  pp.q = hp.q;
  cudaError_t e = upload_plan(hp.blk, pp.blk, bytes);
  {  // whether the block sweeps may run in FP32 pairs (the ADI half-steps)
    std::vector<float> rec;
    pp.blk.df_ok = make_df_records(hp.blk, N, rec);
  }
  auto up = [&](const std::vector<double>& v, double** d64, float** d32) {
    std::vector<float> v32(v.size());
    for (size_t i = 0; i < v.size(); i++) v32[i] = (float)v[i];
    if (e == cudaSuccess) e = cudaMalloc(d64, sizeof(double) * v.size());
    if (e == cudaSuccess) e = cudaMalloc(d32, sizeof(float) * v.size());
    if (e == cudaSuccess) e = cudaMemcpy(*d64, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(*d32, v32.data(), sizeof(float) * v.size(), cudaMemcpyHostToDevice);
    bytes += (sizeof(double) + sizeof(float)) * v.size();
  };
  up(hp.spk, &pp.spk64, &pp.spk32);
  up(hp.red, &pp.red64, &pp.red32);
  return e;
}

// The explicit side e = 2I - A of a Crank-Nicolson step in FP32 pairs (cn.cu)
// keeps the pairs' range and accuracy when every band entry is zero or of
// magnitude in [2^-20, 2^20] (products with inputs in the pairs' range stay
// inside FP32's) and every row's sum of |e| entries is at most 16 (its
// rounding, ~2^-48 of that sum times |C|, then stays near FP64's).
bool cn_pairs_ok(int width, int64_t N, const std::vector<double>& b64) {
  const int h = width / 2;
  for (int64_t i = 0; i < N; i++) {
    double sum = 0.0;
    for (int k = 0; k < width; k++) {
      const double b = b64[(size_t)k * N + i];
      const double a = std::fabs(b);
      if (!(a == 0.0 || (a >= 0x1p-20 && a <= 0x1p20))) return false;
      sum += std::fabs((k == h ? 2.0 : 0.0) - b);
    }
    if (!(sum <= 16.0)) return false;
  }
  return true;
}

// Copies the host plans, factor entries and bands (b64, width * N) of one
// LHS to the current device and registers the handle.
bs_status upload_handle(int width, int64_t N, HostPlan* hp, bool has_ul, bool periodic,
                        const std::vector<double>& entries, const std::vector<double>& b64, bs_handle* out,
                        const HostPart* parts = nullptr) {
  std::vector<float> bhi(b64.size()), blo(b64.size());
  for (size_t q = 0; q < b64.size(); q++) {
    const float hi = (float)b64[q];
    bhi[q] = hi;
    blo[q] = (float)(b64[q] - (double)hi);
  }
  bs_handle hd = new (std::nothrow) bs_factor_s();
  if (!hd) return set_error(BS_ENOMEM, "factor: host allocation failed");
  std::memset(hd, 0, sizeof(*hd));
  hd->width = width;
  hd->N = N;
  cudaGetDevice(&hd->device);
  size_t bytes = 0;
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < 3 && e == cudaSuccess; p++) e = upload_plan(hp[p], hd->plan[p], bytes);
  // FP32-pair sweep records of the primal and adjoint plans (periodic plans:
  // and their correction weights); FP32 records and windows (not periodic)
  for (int p = 0; p < 2 && e == cudaSuccess; p++) {
    std::vector<float> rec;
    hd->plan[p].df_ok = make_df_records(hp[p], N, rec);
    e = cudaMalloc(&hd->plan[p].dfrec, sizeof(float) * rec.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(hd->plan[p].dfrec, rec.data(), sizeof(float) * rec.size(), cudaMemcpyHostToDevice);
    bytes += sizeof(float) * rec.size();
    if (periodic) {
      hd->plan[p].df_ok = make_df_periodic(hp[p], N, rec, hd->plan[p].dfper_unscale) && hd->plan[p].df_ok;
      if (e == cudaSuccess) e = cudaMalloc(&hd->plan[p].dfper, sizeof(float) * rec.size());
      if (e == cudaSuccess)
        e = cudaMemcpy(hd->plan[p].dfper, rec.data(), sizeof(float) * rec.size(), cudaMemcpyHostToDevice);
      bytes += sizeof(float) * rec.size();
      continue;
    }
    make_rec32(hp[p], N, rec);
    if (e == cudaSuccess) e = cudaMalloc(&hd->plan[p].rec32, sizeof(float) * rec.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(hd->plan[p].rec32, rec.data(), sizeof(float) * rec.size(), cudaMemcpyHostToDevice);
    bytes += sizeof(float) * rec.size();
    make_windows(hp[p], N, win_rows(false), win_rows(true), hd->plan[p].win32, hd->plan[p].win_df);
  }
  if (parts) {
    for (int p = 0; p < 2 && e == cudaSuccess; p++) e = upload_part(parts[p], N, hd->part[p], bytes);
    hd->has_part = true;
  }
  {
    std::vector<float> ehi(entries.size()), elo(entries.size());
    for (size_t q = 0; q < entries.size(); q++) {
      ehi[q] = (float)entries[q];
      elo[q] = (float)(entries[q] - (double)ehi[q]);
    }
    if (e == cudaSuccess) e = cudaMalloc(&hd->lu_hi, sizeof(float) * ehi.size());
    if (e == cudaSuccess) e = cudaMalloc(&hd->lu_lo, sizeof(float) * elo.size());
    if (e == cudaSuccess) e = cudaMemcpy(hd->lu_hi, ehi.data(), sizeof(float) * ehi.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(hd->lu_lo, elo.data(), sizeof(float) * elo.size(), cudaMemcpyHostToDevice);
    bytes += 2 * sizeof(float) * ehi.size();
  }
  if (e == cudaSuccess) e = cudaMalloc(&hd->bands64, sizeof(double) * b64.size());
  if (e == cudaSuccess) e = cudaMalloc(&hd->bands_hi, sizeof(float) * bhi.size());
  if (e == cudaSuccess) e = cudaMalloc(&hd->bands_lo, sizeof(float) * blo.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(hd->bands64, b64.data(), sizeof(double) * b64.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(hd->bands_hi, bhi.data(), sizeof(float) * bhi.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(hd->bands_lo, blo.data(), sizeof(float) * blo.size(), cudaMemcpyHostToDevice);
  bytes += (sizeof(double) + 2 * sizeof(float)) * b64.size();
  if (e != cudaSuccess) {
    free_handle(hd);
    if (e == cudaErrorMemoryAllocation) return set_error(BS_ENOMEM, "factor: cudaMalloc failed");
    return cuda_error(e, "factor upload");
  }
  hd->device_bytes = bytes;
  hd->has_ul = has_ul;
  hd->periodic = periodic;
  hd->cn_pairs = cn_pairs_ok(width, N, b64);
  {
    std::lock_guard<std::mutex> lk(g_handles_mu);
    g_handles.insert(hd);
  }
  *out = hd;
  return BS_OK;
}

// Primal plan, in original row order, of the row-reversed matrix J A J:
// A = U' L' with its first sweep over decreasing rows.  Returns false on a
// bad pivot.
bool reversed_plan(const double* const* bd, int width, int64_t N, HostPlan& out) {
  std::vector<double> rev((size_t)width * N);
  const double* rbd[5];
  for (int k = 0; k < width; k++) {
    for (int64_t i = 0; i < N; i++) rev[(size_t)k * N + i] = bd[width - 1 - k][N - 1 - i];
    rbd[k] = rev.data() + (size_t)k * N;
  }
  HostPlan rp, ra;
  rp.c.assign((size_t)C_COUNT * N, 0.0);
  ra.c.assign((size_t)C_COUNT * N, 0.0);
  const bool ok = make_plans(rbd, width, N, rp, ra) == 0;
  out.bw = rp.bw;
  out.fwd_scale = rp.fwd_scale;
  out.bwd_scale = rp.bwd_scale;
  out.c.assign((size_t)C_COUNT * N, 0.0);
  for (int k = 0; k < C_COUNT; k++)
    for (int64_t i = 0; i < N; i++) out.c[(size_t)k * N + i] = rp.c[(size_t)k * N + (N - 1 - i)];
  return ok;
}

// Meeting rows of the two-ended sweeps (see bs::TwistPlan) of a matrix with
// zeroed out-of-range bands bz (width x N), given its plans top (A = L U /
// L R) and bot (A = U' L').  False if the meeting system is singular or not
// finite.
bool twist_rows(const std::vector<double>& bz, int width, const HostPlan& top, const HostPlan& bot, int64_t N,
                bs::TwistPlan& t) {
  auto band = [&](int q, int64_t i) { return (i >= 0 && i < N) ? bz[(size_t)q * N + i] : 0.0; };
  auto cf = [&](const HostPlan& p, int q, int64_t i) { return (i >= 0 && i < N) ? p.c[(size_t)q * N + i] : 0.0; };
  std::memset(t.m, 0, sizeof(t.m));
  if (width == 3) {
    // g_k = b_k - a_k chat_{k-1} - c_k chat'_{k+1}
    const int64_t k = N / 2;
    const double a = band(0, k), c = band(2, k);
    const double g = band(1, k) - a * cf(top, C_U1, k - 1) - c * cf(bot, C_U1, k + 1);
    if (bad(g)) return false;
    t.k = (int)k;
    t.m[0] = -a;
    t.m[1] = -c;
    t.m[2] = 1.0 / g;
  } else {
    // rows k, k+1 with x_{k-1}, x_{k-2} (top back-substitution) and x_{k+2},
    // x_{k+3} (bottom) as affine functions of x_k, x_{k+1}
    const int64_t k = (N - 2) / 2;
    const double g1 = cf(top, C_U1, k - 1), g2 = cf(top, C_U1, k - 2);
    const double d1 = cf(top, C_U2, k - 1), d2 = cf(top, C_U2, k - 2);
    const double v1 = cf(bot, C_U1, k + 2), v3 = cf(bot, C_U1, k + 3);
    const double y1 = cf(bot, C_U2, k + 2), y3 = cf(bot, C_U2, k + 3);
    const double p2k = g2 * g1 - d2, p2m = g2 * d1;  // x_{k-2}
    const double p1k = -g1, p1m = -d1;               // x_{k-1}
    const double q2k = -y1, q2m = -v1;               // x_{k+2}
    const double q3k = -v3 * q2k, q3m = -v3 * q2m - y3;  // x_{k+3}
    const double ak = band(0, k), bk = band(1, k), ck = band(2, k), dk = band(3, k), ek = band(4, k);
    const double a1 = band(0, k + 1), b1 = band(1, k + 1), c1 = band(2, k + 1), d1b = band(3, k + 1),
                 e1 = band(4, k + 1);
    const double m00 = ck + ak * p2k + bk * p1k + ek * q2k, m01 = dk + ak * p2m + bk * p1m + ek * q2m;
    const double m10 = b1 + a1 * p1k + d1b * q2k + e1 * q3k, m11 = c1 + a1 * p1m + d1b * q2m + e1 * q3m;
    const double det = m00 * m11 - m01 * m10;
    if (bad(det)) return false;
    t.k = (int)k;
    t.m[0] = -ak;
    t.m[1] = ak * g2 - bk;
    t.m[2] = -ek;
    t.m[3] = -a1;
    t.m[4] = e1 * v3 - d1b;
    t.m[5] = -e1;
    t.m[6] = m11 / det;
    t.m[7] = -m01 / det;
    t.m[8] = -m10 / det;
    t.m[9] = m00 / det;
    for (double v : t.m)
      if (!std::isfinite(v)) return false;
  }
  t.ok = true;
  return true;
}

}  // namespace

extern "C" {

const char* bs_last_error(void) { return g_last_error.c_str(); }

const char* bs_strerror(bs_status s) {
  switch (s) {
    case BS_OK: return "ok";
    case BS_EINVAL: return "invalid argument";
    case BS_ESINGULAR: return "zero or non-finite pivot (matrix needs pivoting or is singular)";
    case BS_ENOMEM: return "device allocation failed";
    case BS_ECUDA: return "CUDA runtime error";
    case BS_ETIMEOUT: return "bounded device wait timed out";
    case BS_EUNSUPPORTED: return "unsupported combination";
  }
  return "unknown status";
}

int64_t bs_lhs_bytes(int width, int64_t N, int elem_bytes) {
  if ((width != 3 && width != 5) || N < 0 || elem_bytes <= 0) return -1;
  return (int64_t)width * N * elem_bytes;
}

bs_status bs_factor(const double* bands, int width, int64_t N, bs_handle* out) {
  if (!out) return set_error(BS_EINVAL, "bs_factor: out is NULL");
  *out = nullptr;
  if (!bands) return set_error(BS_EINVAL, "bs_factor: bands is NULL");
  if (width != 3 && width != 5) return set_error(BS_EINVAL, "bs_factor: width must be 3 or 5");
  if ((width == 3 && N < 2) || (width == 5 && N < 4))
    return set_error(BS_EINVAL, "bs_factor: N must be >= 2 (tri) or >= 4 (penta)");
  if (N > (int64_t)1 << 28) return set_error(BS_EINVAL, "bs_factor: N too large");

  const double* bd[5];
  for (int k = 0; k < width; k++) bd[k] = bands + (size_t)k * N;

  HostPlan hp[3];
  bool has_ul = false;
  for (auto& p : hp) p.c.assign((size_t)C_COUNT * N, 0.0);
  std::vector<double> entries;
  int64_t bad_row = make_plans(bd, width, N, hp[0], hp[1], &entries);
  if (bad_row) return set_error(BS_ESINGULAR, "bs_factor: bad pivot at row " + std::to_string(bad_row));
  if (width == 5) {
    // uniform outermost sub-diagonal (Sec. 4.1, cuPentUniformBatch): a_i for
    // the in-range rows i >= 2 (0-based) all equal; then eps_i = a_i is one
    // scalar in the primal forward and the adjoint backward sweep
    bool uni = true;
    for (int64_t i = 3; i < N && uni; i++) uni = bd[0][i] == bd[0][2];
    if (uni && std::isfinite(bd[0][2])) {
      for (int p = 0; p < 2; p++) {
        hp[p].uniform = true;
        hp[p].eps = bd[0][2];
      }
    }
  }
  // Reversed matrix J A J (J the row reversal): band k of row i is band
  // (width-1-k) of row N-1-i.  A matrix whose reversed elimination meets a
  // bad pivot still gets a handle; only the refined solve (which needs
  // U' L') and the two-ended sweeps are then refused.
  has_ul = reversed_plan(bd, width, N, hp[2]);

  // Bands with the outside entries zeroed.
  std::vector<double> b64((size_t)width * N, 0.0);
  const int h = width / 2;
  for (int k = 0; k < width; k++)
    for (int64_t i = 0; i < N; i++) {
      const int64_t col = i + k - h;
      b64[(size_t)k * N + i] = (col >= 0 && col < N) ? bd[k][i] : 0.0;
    }
  // row partitions of A and of A^T for small batches
  HostPart parts[2];
  std::vector<double> tb((size_t)width * N, 0.0);  // bands of A^T: band k of row i = band w-1-k of row i+k-h
  for (int k = 0; k < width; k++)
    for (int64_t i = 0; i < N; i++) {
      const int64_t r = i + k - h;
      if (r >= 0 && r < N) tb[(size_t)k * N + i] = bd[width - 1 - k][r];
    }
  const double* tbd[5];
  for (int k = 0; k < width; k++) tbd[k] = tb.data() + (size_t)k * N;
  const bool has_part = make_partition(bd, width, N, parts[0]) && make_partition(tbd, width, N, parts[1]);
  const bs_status st = upload_handle(width, N, hp, has_ul, false, entries, b64, out, has_part ? parts : nullptr);
  if (st != BS_OK) return st;
  // two-ended sweeps (small batches): for A with plans 0 and 2; for A^T with
  // its own two plans, uploaded here
  bs_handle hd = *out;
  if (has_ul && twist_rows(b64, width, hp[0], hp[2], N, hd->twist[0])) {
    hd->twist[0].top = &hd->plan[0];
    hd->twist[0].bot = &hd->plan[2];
  }
  HostPlan tt[2], tq;
  tt[0].c.assign((size_t)C_COUNT * N, 0.0);
  tq.c.assign((size_t)C_COUNT * N, 0.0);
  bs::TwistPlan ta{};
  if (make_plans(tbd, width, N, tt[0], tq) == 0 && reversed_plan(tbd, width, N, tt[1]) &&
      twist_rows(tb, width, tt[0], tt[1], N, ta)) {
    size_t bytes = 0;
    cudaError_t e = upload_plan(tt[0], hd->tplan[0], bytes);
    if (e == cudaSuccess) e = upload_plan(tt[1], hd->tplan[1], bytes);
    hd->device_bytes += bytes;
    if (e != cudaSuccess) {
      bs_destroy(hd);
      *out = nullptr;
      return cuda_error(e, "bs_factor: upload");
    }
    hd->twist[1] = ta;
    hd->twist[1].top = &hd->tplan[0];
    hd->twist[1].bot = &hd->tplan[1];
  }
  return st;
}

bs_status bs_factor_periodic(const double* bands, int64_t N, bs_handle* out) {
  if (!out) return set_error(BS_EINVAL, "bs_factor_periodic: out is NULL");
  *out = nullptr;
  if (!bands) return set_error(BS_EINVAL, "bs_factor_periodic: bands is NULL");
  if (N < 3) return set_error(BS_EINVAL, "bs_factor_periodic: N must be >= 3");
  if (N > (int64_t)1 << 28) return set_error(BS_EINVAL, "bs_factor_periodic: N too large");
  const double* a = bands;
  const double* b = bands + N;
  const double* c = bands + 2 * N;
  // Sherman-Morrison split (Sec. 3.3): A = A' + u v^T, gamma = -b_1,
  // u = (gamma, 0, .., 0, c_N), v = (1, 0, .., 0, a_1 / gamma).
  const double gam = -b[0];
  if (bad(gam)) return set_error(BS_ESINGULAR, "bs_factor_periodic: b_1 must be non-zero");
  const double v_last = a[0] / gam;
  std::vector<double> mod((size_t)3 * N);
  for (int64_t i = 0; i < N; i++) {
    mod[i] = (i > 0) ? a[i] : 0.0;
    mod[N + i] = b[i];
    mod[2 * N + i] = (i + 1 < N) ? c[i] : 0.0;
  }
  mod[N] = b[0] - gam;
  mod[N + N - 1] = b[N - 1] - c[N - 1] * v_last;
  const double* bd[3] = {mod.data(), mod.data() + N, mod.data() + 2 * N};

  HostPlan hp[3];
  for (auto& p : hp) p.c.assign((size_t)C_COUNT * N, 0.0);
  std::vector<double> entries;
  const int64_t bad_row = make_plans(bd, 3, N, hp[0], hp[1], &entries);
  if (bad_row)
    return set_error(BS_ESINGULAR, "bs_factor_periodic: bad pivot of the corner-free matrix at row " +
                                       std::to_string(bad_row));
  // z = A'^{-1} u and q = A'^{-T} v, in FP64 with the plans themselves.
  std::vector<double> z(N, 0.0), q(N, 0.0);
  z[0] = gam;
  z[N - 1] = c[N - 1];
  q[0] = 1.0;
  q[N - 1] = v_last;
  apply_plan(hp[0], N, z);
  apply_plan(hp[1], N, q);
  const double vz = z[0] + v_last * z[N - 1];
  const double den = 1.0 + vz;
  // 1 + v.z is zero exactly when A is singular; within a few rounding errors
  // of zero no digit of the correction can be trusted either.
  if (bad(den) || std::fabs(den) <= 4.0 * (double)N * 2.220446049250313e-16 * (1.0 + std::fabs(vz)))
    return set_error(BS_ESINGULAR, "bs_factor_periodic: 1 + v.z is zero to rounding (the periodic matrix is singular)");
  // For a diagonally dominant A', q and z decay geometrically away from the
  // first and last rows.  Entries below 2^-60 max / N change sigma, or any
  // x_i, by less than 2^-60 of max|q| max|d| (resp. max|z|), far below FP64
  // rounding; they are set to zero, and the middle range of rows where both
  // are zero is recorded so that the kernels skip its correction terms.
  double qmax = 0.0, zmax = 0.0;
  for (int64_t i = 0; i < N; i++) {
    qmax = std::fmax(qmax, std::fabs(q[i]));
    zmax = std::fmax(zmax, std::fabs(z[i]));
  }
  const double tq = qmax * 0x1p-60 / (double)N, tz = zmax * 0x1p-60 / (double)N;
  int64_t lo = 0, hi = N;
  for (int64_t i = 0; i < N; i++) {
    const bool active = std::fabs(q[i]) > tq || std::fabs(z[i]) > tz;
    if (!active) {
      q[i] = 0.0;
      z[i] = 0.0;
    }
  }
  for (int64_t i = 0; i < N / 2; i++)
    if (q[i] != 0.0 || z[i] != 0.0) lo = i + 1;
  for (int64_t i = N - 1; i >= N / 2; i--)
    if (q[i] != 0.0 || z[i] != 0.0) hi = i;
  if (lo > hi) lo = hi;
  // primal: sigma = q.d (= v.y), x = y - sigma z / den;
  // adjoint of A = A' + u v^T: sigma = z.g (= u.(A'^{-T} g)), x = y - sigma q / den
  for (int64_t i = 0; i < N; i++) {
    hp[0].c[(size_t)C_PW * N + i] = q[i];
    hp[0].c[(size_t)C_PC * N + i] = z[i] / den;
    hp[1].c[(size_t)C_PW * N + i] = z[i];
    hp[1].c[(size_t)C_PC * N + i] = q[i] / den;
  }
  hp[0].periodic = hp[1].periodic = true;
  hp[0].per_lo = hp[1].per_lo = (int)lo;
  hp[0].per_hi = hp[1].per_hi = (int)hi;
  hp[2] = hp[0];  // no reversed elimination for the periodic case (never read)
  hp[2].periodic = true;

  // The periodic bands themselves, corners included.
  std::vector<double> b64(bands, bands + 3 * N);
  return upload_handle(3, N, hp, false, true, entries, b64, out);
}

bs_status bs_destroy(bs_handle h) {
  if (!h) return BS_OK;
  {
    std::lock_guard<std::mutex> lk(g_handles_mu);
    if (!g_handles.count(h)) return set_error(BS_EINVAL, "bs_destroy: unknown handle");
    if (h->server_refs > 0)
      return set_error(BS_EINVAL, "bs_destroy: " + std::to_string(h->server_refs) +
                                      " server request(s) using this handle have not finished");
    g_handles.erase(h);
  }
  free_handle(h);
  return BS_OK;
}

bs_status bs_handle_info(bs_handle h, int* width, int64_t* N, size_t* device_bytes) {
  if (!valid_handle(h)) return set_error(BS_EINVAL, "bs_handle_info: unknown handle");
  if (width) *width = h->width;
  if (N) *N = h->N;
  if (device_bytes) *device_bytes = h->device_bytes;
  return BS_OK;
}

}  // extern "C"
