/*
 * Plain CPU FP64 oracle for the shared-LHS batched banded solvers of
 * "Efficient Interleaved Batch Matrix Solvers for CUDA" (Gloster, Carroll,
 * Bustamante, O Naraigh, arXiv:1909.04539).
 *
 * THIS IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT. Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it. It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Everything here is deliberately plain: one system at a time, true
 * divisions where the paper divides, no blocking or fusion, in the order the
 * paper states the steps.  Rows are 0-based in code (the paper's row i is
 * index i-1 here).
 *
 * Storage of a batch: element (row i, system j) of a batch of M systems of N
 * rows lives at X[i*rs + j*ss].  The paper's interleaved layout is rs = M,
 * ss = 1 (Sec. 2, "interleaved data format"); the system-contiguous layout
 * used on the second ADI axis is rs = 1, ss = N.
 *
 * Band storage: bands[k*N + i] is band k of row i.  Tridiagonal (Sec. 3.1):
 * k = 0,1,2 -> a_i (column i-1), b_i (diagonal), c_i (column i+1).
 * Pentadiagonal (Sec. 4.1, note the diagonal is c there): k = 0..4 ->
 * a_i, b_i, c_i, d_i, e_i at columns i-2 .. i+2.  Entries that fall outside
 * the matrix (tri a_1, c_N; penta a_1, a_2, b_1, d_N, e_{N-1}, e_N) are never
 * read by the algorithms below.
 *
 * Compiled with -ffp-contract=off so the x86 and aarch64 builds round alike.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EL(X, i, j) (X)[(int64_t)(i) * rs + (int64_t)(j) * ss]

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* Tridiagonal: Thomas algorithm, Sec. 3.1                             */
/* ------------------------------------------------------------------ */

/* Pre-factorisation (Sec. 3.1, the equations for c-hat):
 *   chat_1 = c_1 / b_1,  chat_i = c_i / (b_i - a_i chat_{i-1}),  i = 2..N.
 * c_N lies outside the matrix; it is taken as 0, so chat_N = 0 (unused).
 * piv[i] receives the denominator (b_1 for the first row), which the tests
 * use to rebuild A = L U.  Returns 0, or 1 + the row of the first zero or
 * non-finite pivot. */
int oracle_tri_factor(int64_t N, const double* bands, double* chat, double* piv) {
  const double* a = bands;
  const double* b = bands + N;
  const double* c = bands + 2 * N;
  for (int64_t i = 0; i < N; i++) {
    double den = (i == 0) ? b[0] : b[i] - a[i] * chat[i - 1];
    double ci = (i == N - 1) ? 0.0 : c[i];
    piv[i] = den;
    if (den == 0.0 || !isfinite(den)) return (int)(i + 1);
    chat[i] = ci / den;
  }
  return 0;
}

/* Forward and backward sweep for one system, overwriting d with x
 * (Sec. 3.1):
 *   dhat_1 = d_1 / b_1,  dhat_i = (d_i - a_i dhat_{i-1}) / (b_i - a_i chat_{i-1});
 *   x_N = dhat_N,        x_i = dhat_i - chat_i x_{i+1},  i = N-1..1.
 * The backward equation is printed garbled in the paper (a_i chat_i); the
 * form used here is the only one for which A x = d. */
static void tri_sweep_one(int64_t N, const double* bands, const double* chat,
                          double* X, int64_t j, int64_t rs, int64_t ss) {
  const double* a = bands;
  const double* b = bands + N;
  EL(X, 0, j) = EL(X, 0, j) / b[0];
  for (int64_t i = 1; i < N; i++)
    EL(X, i, j) = (EL(X, i, j) - a[i] * EL(X, i - 1, j)) / (b[i] - a[i] * chat[i - 1]);
  for (int64_t i = N - 2; i >= 0; i--)
    EL(X, i, j) = EL(X, i, j) - chat[i] * EL(X, i + 1, j);
}

/* Solve A X = B in place for M systems with one shared tridiagonal A. */
int oracle_tri_solve(int64_t N, const double* bands, double* X, int64_t M,
                     int64_t rs, int64_t ss) {
  double* chat = (double*)malloc(sizeof(double) * N);
  double* piv = (double*)malloc(sizeof(double) * N);
  int st = oracle_tri_factor(N, bands, chat, piv);
  if (st == 0) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; j++) tri_sweep_one(N, bands, chat, X, j, rs, ss);
  }
  free(chat);
  free(piv);
  return st;
}

/* ------------------------------------------------------------------ */
/* Pentadiagonal: A = L R, then L g = f, then R x = g (Sec. 4.1)        */
/* ------------------------------------------------------------------ */

/* Factorisation A = L R (Sec. 4.1, the fourteen factorisation steps).
 * L has alpha_i on the diagonal, beta_i one below, eps_i two below; R is unit
 * upper with gamma_i, delta_i on the first and second super-diagonals.
 * Output f[k*N + i] for k = 0..4 -> alpha, beta, gamma, delta, eps.  Values
 * the paper does not define (beta_1, gamma_N, delta_{N-1}, delta_N) are 0.
 * Requires N >= 4 (the special first and last rows would overlap below).
 * Returns 0, or 1 + the row of the first zero or non-finite alpha. */
int oracle_penta_factor(int64_t N, const double* bands, double* f) {
  const double* a = bands;
  const double* b = bands + N;
  const double* c = bands + 2 * N;
  const double* d = bands + 3 * N;
  const double* e = bands + 4 * N;
  double* al = f;
  double* be = f + N;
  double* ga = f + 2 * N;
  double* de = f + 3 * N;
  double* ep = f + 4 * N;
  if (N < 4) return -1;
  memset(f, 0, sizeof(double) * 5 * N);
#define CHECK_ALPHA(i) do { if (al[i] == 0.0 || !isfinite(al[i])) return (int)((i) + 1); } while (0)
  /* steps 1-3: first row */
  al[0] = c[0];
  CHECK_ALPHA(0);
  ga[0] = d[0] / al[0];
  de[0] = e[0] / al[0];
  /* steps 4-7: second row */
  be[1] = b[1];
  al[1] = c[1] - be[1] * ga[0];
  CHECK_ALPHA(1);
  ga[1] = (d[1] - be[1] * de[0]) / al[1];
  de[1] = e[1] / al[1];
  /* step 8: rows 3 .. N-2 */
  for (int64_t i = 2; i <= N - 3; i++) {
    be[i] = b[i] - a[i] * ga[i - 2];
    al[i] = c[i] - a[i] * de[i - 2] - be[i] * ga[i - 1];
    CHECK_ALPHA(i);
    ga[i] = (d[i] - be[i] * de[i - 1]) / al[i];
    de[i] = e[i] / al[i];
  }
  /* steps 9-11: row N-1 */
  {
    int64_t i = N - 2;
    be[i] = b[i] - a[i] * ga[i - 2];
    al[i] = c[i] - a[i] * de[i - 2] - be[i] * ga[i - 1];
    CHECK_ALPHA(i);
    ga[i] = (d[i] - be[i] * de[i - 1]) / al[i];
  }
  /* steps 12-13: row N */
  {
    int64_t i = N - 1;
    be[i] = b[i] - a[i] * ga[i - 2];
    al[i] = c[i] - a[i] * de[i - 2] - be[i] * ga[i - 1];
    CHECK_ALPHA(i);
  }
  /* step 14: eps_i = a_i (rows 3..N; rows 1, 2 have no such entry) */
  for (int64_t i = 2; i < N; i++) ep[i] = a[i];
#undef CHECK_ALPHA
  return 0;
}

/* L g = f then R x = g for one system, overwriting f with x (Sec. 4.1):
 *   g_1 = f_1/alpha_1, g_2 = (f_2 - beta_2 g_1)/alpha_2,
 *   g_i = (f_i - eps_i g_{i-2} - beta_i g_{i-1})/alpha_i,  i = 3..N;
 *   x_N = g_N, x_{N-1} = g_{N-1} - gamma_{N-1} x_N,
 *   x_i = g_i - gamma_i x_{i+1} - delta_i x_{i+2},  i = N-2..1. */
static void penta_sweep_one(int64_t N, const double* f, double* X, int64_t j,
                            int64_t rs, int64_t ss) {
  const double* al = f;
  const double* be = f + N;
  const double* ga = f + 2 * N;
  const double* de = f + 3 * N;
  const double* ep = f + 4 * N;
  EL(X, 0, j) = EL(X, 0, j) / al[0];
  EL(X, 1, j) = (EL(X, 1, j) - be[1] * EL(X, 0, j)) / al[1];
  for (int64_t i = 2; i < N; i++)
    EL(X, i, j) = (EL(X, i, j) - ep[i] * EL(X, i - 2, j) - be[i] * EL(X, i - 1, j)) / al[i];
  EL(X, N - 2, j) = EL(X, N - 2, j) - ga[N - 2] * EL(X, N - 1, j);
  for (int64_t i = N - 3; i >= 0; i--)
    EL(X, i, j) = EL(X, i, j) - ga[i] * EL(X, i + 1, j) - de[i] * EL(X, i + 2, j);
}

int oracle_penta_solve(int64_t N, const double* bands, double* X, int64_t M,
                       int64_t rs, int64_t ss) {
  double* f = (double*)malloc(sizeof(double) * 5 * N);
  int st = oracle_penta_factor(N, bands, f);
  if (st == 0) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; j++) penta_sweep_one(N, f, X, j, rs, ss);
  }
  free(f);
  return st;
}

/* Dispatch on band width (3 or 5). */
int oracle_solve(int width, int64_t N, const double* bands, double* X, int64_t M,
                 int64_t rs, int64_t ss) {
  if (width == 3) return oracle_tri_solve(N, bands, X, M, rs, ss);
  if (width == 5) return oracle_penta_solve(N, bands, X, M, rs, ss);
  return -1;
}

/* ------------------------------------------------------------------ */
/* Banded operator pieces used by the adjoint, refinement and ADI paths */
/* ------------------------------------------------------------------ */

/* Bands of A^T: entry (i, i+k-h) of A^T is entry (i+k-h, i) of A, i.e. band
 * (width-1-k) of row i+k-h.  Outside entries are set to 0. */
void oracle_transpose_bands(int width, int64_t N, const double* bands, double* bt) {
  int h = width / 2;
  for (int k = 0; k < width; k++)
    for (int64_t i = 0; i < N; i++) {
      int64_t r = i + k - h;
      bt[k * N + i] = (r >= 0 && r < N) ? bands[(int64_t)(width - 1 - k) * N + r] : 0.0;
    }
}

/* Y = A X for a batch (plain banded product). */
void oracle_band_matvec(int width, int64_t N, const double* bands, const double* X,
                        double* Y, int64_t M, int64_t rs, int64_t ss) {
  int h = width / 2;
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < M; j++)
    for (int64_t i = 0; i < N; i++) {
      double s = 0.0;
      for (int k = 0; k < width; k++) {
        int64_t col = i + k - h;
        if (col >= 0 && col < N) s += bands[(int64_t)k * N + i] * EL(X, col, j);
      }
      EL(Y, i, j) = s;
    }
}

/* Residual R = B - A X for a batch. */
void oracle_residual(int width, int64_t N, const double* bands, const double* B,
                     const double* X, double* R, int64_t M, int64_t rs, int64_t ss) {
  int h = width / 2;
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < M; j++)
    for (int64_t i = 0; i < N; i++) {
      double s = 0.0;
      for (int k = 0; k < width; k++) {
        int64_t col = i + k - h;
        if (col >= 0 && col < N) s += bands[(int64_t)k * N + i] * EL(X, col, j);
      }
      EL(R, i, j) = EL(B, i, j) - s;
    }
}

/* Gradient of a scalar loss with respect to the band entries, given
 * GB = dL/dB = A^{-T} dL/dX and X = A^{-1} B:
 *   dL/dA = -GB X^T, so dL/d(band k of row i) = -sum_j GB[i,j] X[i+k-h, j].
 * Entries outside the matrix get 0.  Summed over j in increasing order. */
void oracle_band_grad(int width, int64_t N, const double* GB, const double* X,
                      int64_t M, int64_t rs, int64_t ss, double* dbands) {
  int h = width / 2;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++)
    for (int k = 0; k < width; k++) {
      int64_t col = i + k - h;
      double s = 0.0;
      if (col >= 0 && col < N)
        for (int64_t j = 0; j < M; j++) s += EL(GB, i, j) * EL(X, col, j);
      dbands[(int64_t)k * N + i] = -s;
    }
}

/* The same for a periodic tridiagonal A (columns modulo N): every one of
 * the 3N band entries is a matrix entry, the corners being a_1 (k = 0, i = 0,
 * column N-1) and c_N (k = 2, i = N-1, column 0). */
void oracle_band_grad_periodic(int64_t N, const double* GB, const double* X,
                               int64_t M, int64_t rs, int64_t ss, double* dbands) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; i++)
    for (int k = 0; k < 3; k++) {
      int64_t col = (i + k - 1 + N) % N;
      double s = 0.0;
      for (int64_t j = 0; j < M; j++) s += EL(GB, i, j) * EL(X, col, j);
      dbands[(int64_t)k * N + i] = -s;
    }
}

/* ------------------------------------------------------------------ */
/* Periodic tridiagonal via Sherman-Morrison (Sec. 3.3)                */
/* ------------------------------------------------------------------ */

/* Periodic tridiagonal A: row i has a_i at column i-1, b_i on the diagonal
 * and c_i at column i+1, columns taken modulo N (so a_1 sits in the top-right
 * corner and c_N in the bottom-left one; Sec. 3.3 has constant a, b, c).
 * Written as A = A' + u v^T with g = -b_1, u = (g, 0, .., 0, c_N)^T and
 * v = (1, 0, .., 0, a_1 / g)^T, so that A' is tridiagonal with its corners
 * removed, A'_11 = b_1 - g = 2 b_1 and A'_NN = b_N - c_N a_1 / g.  Solve
 * A' y = d and A' z = u, then x = y - (v.y)/(1 + v.z) z.  For constant
 * coefficients this is the paper's u = (-b, 0, .., c), v = (1, 0, .., -a/b).
 * (The paper prints A' with the corners still present and the second solve
 * as A' x = u; the reading used here is the one for which A = A' + u v^T.) */
int oracle_periodic_tri_solve_bands(int64_t N, const double* pb, double* X, int64_t M, int64_t rs, int64_t ss) {
  const double* a = pb;
  const double* b = pb + N;
  const double* c = pb + 2 * N;
  double* bands = (double*)calloc(3 * N, sizeof(double));
  double* z = (double*)calloc(N, sizeof(double));
  int st;
  const double g = -b[0];
  for (int64_t i = 0; i < N; i++) {
    bands[i] = (i > 0) ? a[i] : 0.0;
    bands[N + i] = b[i];
    bands[2 * N + i] = (i < N - 1) ? c[i] : 0.0;
  }
  bands[N + 0] = b[0] - g;
  bands[N + N - 1] = b[N - 1] - c[N - 1] * a[0] / g;
  z[0] = g;
  z[N - 1] = c[N - 1];
  st = oracle_tri_solve(N, bands, z, 1, 1, 1);
  if (st == 0) st = oracle_tri_solve(N, bands, X, M, rs, ss);
  if (st == 0) {
    const double vz = z[0] + (a[0] / g) * z[N - 1];
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; j++) {
      double vy = EL(X, 0, j) + (a[0] / g) * EL(X, N - 1, j);
      double s = vy / (1.0 + vz);
      for (int64_t i = 0; i < N; i++) EL(X, i, j) = EL(X, i, j) - s * z[i];
    }
  }
  free(bands);
  free(z);
  return st;
}

/* The paper's constant-coefficient case (Sec. 3.3). */
int oracle_periodic_tri_solve(int64_t N, double a, double b, double c, double* X, int64_t M, int64_t rs,
                              int64_t ss) {
  double* pb = (double*)malloc(sizeof(double) * 3 * N);
  int st;
  for (int64_t i = 0; i < N; i++) {
    pb[i] = a;
    pb[N + i] = b;
    pb[2 * N + i] = c;
  }
  st = oracle_periodic_tri_solve_bands(N, pb, X, M, rs, ss);
  free(pb);
  return st;
}

/* ------------------------------------------------------------------ */
/* Crank-Nicolson time steps (the paper's benchmark problems, Sec. 3.2  */
/* and Sec. 4.2)                                                       */
/* ------------------------------------------------------------------ */

/* The CN scheme for C_t = L C writes A C^{n+1} = B C^n with
 * A = I - (dt/2) L and B = I + (dt/2) L, so that B = 2I - A: for the
 * diffusion benchmark A = (-s, 1 + 2s, -s) and B = (s, 1 - 2s, s); for the
 * hyperdiffusion benchmark A = (s, -4s, 1 + 6s, -4s, s) and
 * B = (-s, 4s, 1 - 6s, 4s, -s).  One step: F = 2 C - A C, then solve
 * A C = F (periodic != 0: A is the periodic tridiagonal matrix of Sec. 3.3,
 * columns modulo N; else A is banded).  Repeated `steps` times in place. */
int oracle_cn_steps(int width, int64_t N, const double* bands, int periodic, double* X, int64_t M, int64_t rs,
                    int64_t ss, int steps) {
  int h = width / 2;
  int st = 0;
  double* F = (double*)malloc(sizeof(double) * N * M);
  for (int n = 0; n < steps && st == 0; n++) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; j++)
      for (int64_t i = 0; i < N; i++) {
        double s = 0.0;
        for (int k = 0; k < width; k++) {
          int64_t col = i + k - h;
          if (periodic) col = (col + N) % N;
          if (col >= 0 && col < N) s += bands[(int64_t)k * N + i] * EL(X, col, j);
        }
        F[i * M + j] = 2.0 * EL(X, i, j) - s;
      }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; j++)
      for (int64_t i = 0; i < N; i++) EL(X, i, j) = F[i * M + j];
    if (periodic)
      st = oracle_periodic_tri_solve_bands(N, bands, X, M, rs, ss);
    else
      st = oracle_solve(width, N, bands, X, M, rs, ss);
  }
  free(F);
  return st;
}

/* ------------------------------------------------------------------ */
/* 2D ADI (Peaceman-Rachford) half-step for u_t = u_xx + u_yy           */
/* ------------------------------------------------------------------ */

/* Field u[y*nx + x], homogeneous Dirichlet (zero outside the grid).
 * implicit_axis = 0 (x): (I - r dxx) out = (I + r dyy) u, solved along x,
 *   i.e. system j = y with rows i = x at out[j*nx + i] (system-contiguous).
 * implicit_axis = 1 (y): (I - r dyy) out = (I + r dxx) u, solved along y,
 *   i.e. system j = x with rows i = y at out[i*nx + j] (interleaved, M = nx).
 * The shared LHS is the tridiagonal (-r, 1 + 2r, -r). */
int oracle_adi_halfstep(int64_t ny, int64_t nx, double r, const double* u,
                        double* out, int implicit_axis) {
  int64_t n_sys = implicit_axis == 0 ? ny : nx;
  int64_t n_row = implicit_axis == 0 ? nx : ny;
  double* bands = (double*)malloc(sizeof(double) * 3 * n_row);
  int st;
#pragma omp parallel for schedule(static)
  for (int64_t y = 0; y < ny; y++)
    for (int64_t x = 0; x < nx; x++) {
      double c0 = u[y * nx + x], lo, hi;
      if (implicit_axis == 0) { /* explicit along y */
        lo = (y > 0) ? u[(y - 1) * nx + x] : 0.0;
        hi = (y < ny - 1) ? u[(y + 1) * nx + x] : 0.0;
      } else { /* explicit along x */
        lo = (x > 0) ? u[y * nx + x - 1] : 0.0;
        hi = (x < nx - 1) ? u[y * nx + x + 1] : 0.0;
      }
      out[y * nx + x] = c0 + r * (lo - 2.0 * c0 + hi);
    }
  for (int64_t i = 0; i < n_row; i++) {
    bands[i] = -r;
    bands[n_row + i] = 1.0 + 2.0 * r;
    bands[2 * n_row + i] = -r;
  }
  if (implicit_axis == 0)
    st = oracle_tri_solve(n_row, bands, out, n_sys, 1, nx);
  else
    st = oracle_tri_solve(n_row, bands, out, n_sys, nx, 1);
  free(bands);
  return st;
}

/* ADI half-step with a general implicit operator and its transpose: the
 * explicit operator E = I + r d2 (second difference, zero outside the
 * grid) along the explicit axis, then a solve with the shared banded S
 * (width 3 or 5, n_row x width bands of S, Sec. 3.1 / Sec. 4.1 layout) or,
 * with transpose = 1, with S^T along the implicit axis.  transpose = 1 is
 * the transpose of the map u -> S^{-1} E u: (S^{-1} E)^T = E^T S^{-T} = E
 * S^{-T}, and E, acting on the other axis, commutes with S^{-T}.  Axes and
 * storage as oracle_adi_halfstep. */
int oracle_adi_halfstep_bands(int64_t ny, int64_t nx, double r, int width, const double* bands,
                              const double* u, double* out, int implicit_axis, int transpose) {
  int64_t n_sys = implicit_axis == 0 ? ny : nx;
  int64_t n_row = implicit_axis == 0 ? nx : ny;
  double* s = (double*)malloc(sizeof(double) * width * n_row);
  int st;
#pragma omp parallel for schedule(static)
  for (int64_t y = 0; y < ny; y++)
    for (int64_t x = 0; x < nx; x++) {
      double c0 = u[y * nx + x], lo, hi;
      if (implicit_axis == 0) {
        lo = (y > 0) ? u[(y - 1) * nx + x] : 0.0;
        hi = (y < ny - 1) ? u[(y + 1) * nx + x] : 0.0;
      } else {
        lo = (x > 0) ? u[y * nx + x - 1] : 0.0;
        hi = (x < nx - 1) ? u[y * nx + x + 1] : 0.0;
      }
      out[y * nx + x] = c0 + r * (lo - 2.0 * c0 + hi);
    }
  if (transpose)
    oracle_transpose_bands(width, n_row, bands, s);
  else
    for (int64_t q = 0; q < (int64_t)width * n_row; q++) s[q] = bands[q];
  if (implicit_axis == 0)
    st = oracle_solve(width, n_row, s, out, n_sys, 1, nx);
  else
    st = oracle_solve(width, n_row, s, out, n_sys, nx, 1);
  free(s);
  return st;
}
