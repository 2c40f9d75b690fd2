/*
 * bsolve: batched shared-LHS tridiagonal / pentadiagonal solves on GB300
 * (sm_103a).  C ABI.
 *
 * The method is that of "Efficient Interleaved Batch Matrix Solvers for CUDA"
 * (Gloster, Carroll, Bustamante, O Naraigh, arXiv:1909.04539): one banded
 * LHS A (N x N) is factorised once and kept as a single copy shared by every
 * system of the batch (Sec. 2); M right-hand sides are stored interleaved,
 * row i of system j at B[i*M + j] (Sec. 2, Sec. 3.1); each system is solved
 * by one forward and one backward sweep, one thread per system.
 *
 * Conventions for every entry point below:
 *  - Bands are passed row-aligned as width x N doubles: band k of row i at
 *    bands[k*N + i].  Tridiagonal (width 3, Sec. 3.1): a_i, b_i, c_i at
 *    columns i-1, i, i+1.  Pentadiagonal (width 5, Sec. 4.1, diagonal c):
 *    a_i .. e_i at columns i-2 .. i+2.  Entries outside the matrix are ignored.
 *  - B, G, X, U and dbands are caller-owned DEVICE memory on the current
 *    device.  The library never frees or keeps them.
 *  - Layouts: BS_INTERLEAVED puts row i of system j at [i*M + j] (the
 *    paper's layout); BS_STRIDED puts it at [j*N + i] (system-contiguous,
 *    the second axis of a 2D ADI step).
 *  - Every solve is enqueued on `stream` (NULL = legacy default stream) and
 *    returns without waiting.  Argument errors are reported synchronously
 *    and nothing is enqueued; a kernel never traps.  Sizes are row counts and
 *    system counts, not bytes.
 *  - A handle is immutable after bs_factor, so solves with one handle may run
 *    concurrently on different streams.  bs_destroy must not race with them.
 */
#ifndef BSOLVE_H
#define BSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* bs_stream; /* a cudaStream_t */

typedef struct bs_factor_s* bs_handle; /* opaque, owned by the library */

typedef enum {
  BS_OK = 0,
  BS_EINVAL = 1,      /* bad argument: null pointer, size, alignment, combination */
  BS_ESINGULAR = 2,   /* zero or non-finite pivot met while factorising */
  BS_ENOMEM = 3,      /* device allocation failed */
  BS_ECUDA = 4,       /* a CUDA runtime call failed (see bs_last_error) */
  BS_ETIMEOUT = 5,    /* a bounded device-side wait ran out */
  BS_EUNSUPPORTED = 6 /* valid request this build does not implement */
} bs_status;

typedef enum {
  BS_F64 = 0,  /* FP64 storage, FP64 arithmetic */
  BS_F32 = 1,  /* FP32 storage, FP32 arithmetic */
  BS_BF16 = 2  /* BF16 storage of the input, FP32 arithmetic and output */
} bs_dtype;

typedef enum { BS_INTERLEAVED = 0, BS_STRIDED = 1 } bs_layout;

/* Factorise the shared LHS once (Sec. 3.1 Thomas pre-factorisation for
 * width 3; Sec. 4.1 A = L R for width 5) on the host in FP64, then copy the
 * sweep coefficients (FP64 and FP32 copies) and the bands to the current
 * device.  bands: host pointer, width x N doubles (read only, not kept).
 * N >= 2 for width 3, N >= 4 for width 5.  No pivoting (the paper relies on
 * diagonal dominance or symmetric positive definiteness, Sec. 4.3): a zero
 * or non-finite pivot returns BS_ESINGULAR and *out stays NULL.
 * Blocking (synchronous device copies).  The handle owns its device memory
 * until bs_destroy.  A width-5 matrix whose outermost sub-diagonal entries
 * a_3 .. a_N (1-based) are all equal is marked uniform (see BS_OPT_UNIFORM). */
bs_status bs_factor(const double* bands, int width, int64_t N, bs_handle* out);

/* Factorise a periodic (cyclic) tridiagonal LHS, Sec. 3.3: row i has a_i at
 * column i-1, b_i on the diagonal and c_i at column i+1, columns taken
 * modulo N, so a_1 (band 0, row 0) sits in the top-right corner and c_N
 * (band 2, row N-1) in the bottom-left one; the paper's case is constant
 * a, b, c.  bands: host pointer, 3 x N doubles.  N >= 3.
 * The matrix is split as A = A' + u v^T with gamma = -b_1,
 * u = (gamma, 0, .., 0, c_N), v = (1, 0, .., 0, a_1 / gamma), A' tridiagonal
 * with A'_11 = 2 b_1 and A'_NN = b_N - c_N a_1 / gamma.  A' is factorised as
 * bs_factor does, and z = A'^{-1} u and q = A'^{-T} v are formed once on the
 * host in FP64, so that every later solve applies x = y - (q.d)/(1 + v.z) z
 * (y = A'^{-1} d) inside its own two sweeps with no extra pass; the adjoint
 * applies the transposed correction the same way.  Returns BS_ESINGULAR for
 * b_1 == 0, a bad pivot of A', or 1 + v.z == 0 or non-finite.
 * The handle works with bs_solve, bs_solve_bf16, bs_solve_adjoint and the
 * band gradients (whose output then includes the two corner entries);
 * bs_solve_refine, bs_adi_halfstep and the server return BS_EUNSUPPORTED for
 * it.  Blocking; the handle owns its device memory until bs_destroy. */
bs_status bs_factor_periodic(const double* bands, int64_t N, bs_handle* out);

/* Release a handle's device memory.  The caller must ensure no solve using it
 * is still running (synchronise its streams first).  A handle named by server
 * requests that have not finished (bs_server_submit) is not released:
 * BS_EINVAL, and the handle stays valid.  NULL is a no-op. */
bs_status bs_destroy(bs_handle h);

/* Width, N and device bytes held by a handle (any pointer may be NULL). */
bs_status bs_handle_info(bs_handle h, int* width, int64_t* N, size_t* device_bytes);

/* Bytes of shared LHS data one solve reads: width x N values of the sweep
 * coefficients (3N tridiagonal, 5N pentadiagonal; Sec. 3.1, Sec. 4.1), for an
 * element of elem_bytes.  Host-only arithmetic. */
int64_t bs_lhs_bytes(int width, int64_t N, int elem_bytes);

/* Solve A X = B for M systems, in place (the paper overwrites the RHS with
 * the solution, Sec. 3.1): forward sweep then backward sweep per system
 * (Sec. 3.1 tridiagonal, Sec. 4.1 pentadiagonal).
 *   dtype BS_F64: B is double[N*M], FP64 arithmetic.
 *   dtype BS_F32: B is float[N*M], FP32 arithmetic.
 *   dtype BS_BF16: not in place -- use bs_solve_bf16.
 * The intermediate forward-sweep values are kept in B itself between the two
 * sweeps.  M >= 1.  A small batch may be solved row-partitioned (see
 * BS_OPT_PARTITION): the result is the same to rounding, and the call then
 * also allocates 2h (P - 1) x M values of stream-ordered scratch for the
 * block-edge system.  A periodic handle
 * (bs_factor_periodic) solves the cyclic system. */
bs_status bs_solve(bs_handle h, void* B, bs_dtype dtype, bs_layout layout, int64_t M,
                   bs_stream stream);

/* BF16 storage, FP32 arithmetic: reads B (bf16[N*M]), writes X (float[N*M]).
 * X also holds the forward-sweep intermediates.  B and X must not overlap. */
bs_status bs_solve_bf16(bs_handle h, const void* B, float* X, bs_layout layout, int64_t M,
                        bs_stream stream);

/* Mixed-precision solve (FP32 storage, FP64 result): X = A^{-1} B with B
 * stored in FP32 (float[N*M], device, read only) or BF16 (b_dtype BS_BF16,
 * bf16[N*M], widened exactly to FP32) and X written in FP64 (double[N*M],
 * device).  The sweeps run in FP32; refinement corrects them with residuals
 * evaluated to FP64 accuracy and adds the corrections in FP64:
 *   mode BS_REFINE_FACTOR (default, two passes per system, one kernel): the
 *     first step refines each triangular factor of A = L U once, solved in
 *     FP32 with its own residual evaluated to FP64 accuracy in FP32
 *     arithmetic (FP64 coefficients split into FP32 pairs, error-free
 *     products and sums) -- B - L w on the way up, y - U x on the way down;
 *   mode BS_REFINE_SYSTEM (three passes, one kernel): the first step refines
 *     the whole system, r = B - A X0 of the FP32 solution X0 driving one
 *     correction solve through the reversed elimination A = U' L'
 *     (factorised once with the handle) so that its first sweep follows the
 *     backward sweep of X0;
 *   mode BS_REFINE_AUTO: BS_REFINE_FACTOR, except for batches with fewer
 *     than 256 systems per SM, whose FP32 passes are bound by their chains
 *     of dependent rows: those are solved as an FP64 solve of B widened
 *     exactly to FP64 in X (as bs_solve does it, row-partitioned or
 *     two-ended), which is faster there and exact to FP64 rounding (not in
 *     the paper).
 * refine_steps = 0 returns the FP32 solution widened to FP64 (mode ignored),
 * 1 the first step above (~1e-15 relative error on well-conditioned bands);
 * each further step (up to 8) refines the whole system once more: r = B - A X
 * in FP64 rounded to FP32, A d = r by the FP32 sweeps (as bs_solve does it),
 * X += d -- each step multiplies the error by about kappa(A) 2^-24, for bands
 * too ill-conditioned for one step (stiff Crank-Nicolson hyperdiffusion
 * I + s D4 with large s, Sec. 4.2).  Further steps and the BF16 input take
 * stream-ordered scratch: N*M floats.
 * Layout BS_INTERLEAVED or BS_STRIDED (B[j*N + i] in, X[j*N + i] out; the
 * kernels run interleaved: B is transposed into scratch and X out of
 * N*M doubles of scratch).  X doubles as the workspace of the passes.  B and
 * X must not overlap.  BS_REFINE_SYSTEM returns BS_ESINGULAR if the reversed
 * elimination of A met a bad pivot when the handle was built (the other
 * solves still work then).
 * Not in the paper: the paper's solvers work in a single precision. */
typedef enum { BS_REFINE_FACTOR = 0, BS_REFINE_SYSTEM = 1, BS_REFINE_AUTO = 2 } bs_refine_mode;
bs_status bs_solve_refine(bs_handle h, const void* B, bs_dtype b_dtype, double* X, bs_layout layout,
                          int64_t M, int refine_steps, bs_refine_mode mode, bs_stream stream);

/* Adjoint solve: G <- A^{-T} G, in place, reusing the same factorisation
 * (A^T = R^T L^T, a forward sweep with R^T then a backward sweep with L^T).
 * If X (the primal solution A^{-1} B, same dtype and layout as G) and dbands
 * are both non-NULL, also writes the gradient of a scalar loss with respect
 * to the band entries, given dL/dX = G on entry:
 *   dbands[k*N + i] = -sum_j (A^{-T} G)[i, j] * X[i + k - width/2, j]
 * (0 for entries outside the matrix), as double[width*N] in device memory,
 * reduced over the batch in a fixed order (deterministic, no atomics).
 * dtype BS_F64 or BS_F32.  Band gradients are accumulated in FP64.  The
 * reduction takes stream-ordered scratch (cudaMallocAsync/cudaFreeAsync on
 * `stream`) of (number of system chunks) x width x N doubles, about 160 KB for
 * N = 512. */
bs_status bs_solve_adjoint(bs_handle h, void* G, bs_dtype dtype, bs_layout layout, int64_t M,
                           const void* X, double* dbands, bs_stream stream);

/* bs_band_grad without any device allocation (the paper has no counterpart).
 * Some callers cannot allocate device memory at call time: a service that has
 * handed all device memory to its own pool allocator, or a latency-bound loop
 * where an allocation could block on the driver.  This entry point computes
 * exactly what bs_band_grad computes (same kernels, same fixed reduction
 * order, bitwise the same result) but keeps its partial sums in a fixed
 * device array inside the library (2 MiB, held on every GPU that loads the
 * library until the process exits) and allocates nothing.  The caller still
 * provides GB, X and dbands as for bs_band_grad.
 * Limit: the partial sums need about (N / 3 + 8 G) x 3 x width doubles
 * (row blocks of 3 rows taken four at a time; G = the reduction's CTA count,
 * SMs x resident CTAs per SM: 304 on GB300) and the array holds 262144 of
 * them: on GB300 N above about 47000 (width 5) or 80000 (width 3) is
 * rejected with BS_EINVAL and a message naming the size -- use bs_band_grad
 * there.
 * The first call on a device looks up the array's device address (with that
 * device current); a first call made while its stream is being captured
 * returns BS_EINVAL.  All calls
 * share the one array and it keeps the last call's contents (every partial is
 * written before it is read, so nothing needs clearing): calls that can
 * overlap on the GPU -- on different streams, or from different host threads
 * -- race and must be serialised by the caller. */
bs_status bs_band_grad_noalloc(bs_handle h, const void* GB, const void* X, bs_dtype dtype, bs_layout layout,
                               int64_t M, double* dbands, bs_stream stream);

/* `steps` Crank-Nicolson time steps of the batch C (device, interleaved,
 * N x M, dtype BS_F64 or BS_F32), in place: C <- A^{-1} (2I - A) C, where A
 * is the handle's matrix.  For C_t = L C the scheme's LHS is A = I - (dt/2) L
 * and its explicit side is I + (dt/2) L = 2I - A, so the handle alone defines
 * the step: the paper's benchmarks are the periodic diffusion equation
 * (A = (-s, 1 + 2s, -s) from bs_factor_periodic, Sec. 3.2-3.3) and the
 * hyperdiffusion equation (A = (s, -4s, 1 + 6s, -4s, s), Sec. 4.2).  The
 * explicit side is applied while the forward sweep reads the rows (no
 * separate stencil pass); for a periodic handle it wraps around and the
 * Sherman-Morrison correction is fused as in bs_solve.  One kernel launch
 * per step, stream-ordered.  FP64 steps of a handle whose band entries
 * (corners included) are zero or of magnitude in [2^-20, 2^20] and whose
 * explicit side has every row's sum of |entries| at most 16 run in FP32
 * pairs like bs_solve's FP64 path, the Sherman-Morrison terms of a periodic
 * handle included (errors of a few 1e-14 instead of 1e-15; the
 * BS_OPT_F64_PAIRS option set to 1 keeps FP64 arithmetic).  A system with
 * a value the pairs do not hold (|C| >= 2^97, 2^76 for a periodic handle;
 * nonzero |C| < 2^-72; inf, NaN) continues in FP64 from that row on.
 * BS_EUNSUPPORTED for the strided layout. */
bs_status bs_cn_steps(bs_handle h, void* C, bs_dtype dtype, bs_layout layout, int64_t M, int steps,
                      bs_stream stream);

/* One Peaceman-Rachford ADI half-step for u_t = u_xx + u_yy on an ny x nx
 * grid stored row-major (U[y*nx + x], device), homogeneous Dirichlet
 * boundaries (zero outside the grid):
 *   implicit_axis 0: S out = (I + r d2/dy2) U, S solved along x for every row
 *                    y (each row is a system of nx unknowns; h->N == nx);
 *   implicit_axis 1: S out = (I + r d2/dx2) U, S solved
 *                    along y for every column x (interleaved, M = nx;
 *                    h->N == ny),
 * where S is the handle's shared LHS (for the heat equation the tridiagonal
 * I - r d2, one copy for every grid line -- the ADI use the paper's Sec. 1
 * names) and d2 the second difference.  The explicit operator is applied
 * while the forward sweep loads its rows.  adjoint = 1 applies the transpose
 * of the map U -> out instead: out = S^{-T} (I + r d2) U (the explicit
 * operator is symmetric and commutes with S, which acts on the other axis).
 * dtype BS_F64 or BS_F32 for both U and out; U and out must not overlap
 * (out also holds the forward-sweep values).  Not in the paper beyond the
 * motivation: the paper benchmarks 1D problems only. */
bs_status bs_adi_halfstep(bs_handle h, const void* U, void* out, bs_dtype dtype, int64_t ny, int64_t nx,
                          double r, int implicit_axis, int adjoint, bs_stream stream);

/* Band-gradient reduction alone, for a caller that already holds
 * GB = A^{-T} (dL/dX) (e.g. from bs_solve_adjoint without X):
 *   dbands[k*N + i] = -sum_j GB[i, j] * X[i + k - width/2, j]
 * (0 for entries outside the matrix; for a bs_factor_periodic handle the
 * column index is taken modulo N and every entry is defined, the corners
 * being dbands[0] (a_1) and dbands[3N-1] (c_N)), reduced in a fixed order
 * (equal contiguous ranges of (row block, system) per CTA, then the CTAs'
 * partials in CTA order), bitwise reproducible on a given device.  GB and X:
 * device, same dtype (BS_F64 or BS_F32) and layout; dbands: device
 * double[width*N], overwritten.  Uses stream-ordered scratch as
 * bs_solve_adjoint does. */
bs_status bs_band_grad(bs_handle h, const void* GB, const void* X, bs_dtype dtype, bs_layout layout,
                       int64_t M, double* dbands, bs_stream stream);

/* ------------------------------------------------------------------------
 * Request server (not in the paper): continuous batching of solves with many
 * factorised LHS resident on one GPU.
 *
 * A server reserves `hbm_budget_bytes` of device memory as an arena and runs
 * a worker thread.  Each request names a resident handle, a host input B and
 * a host output X (both must stay valid until the request has finished; pinned
 * host memory gives the fastest copies):
 *   mode BS_SERVE_F64        : B double[N*M], X double[N*M] (X may equal B);
 *                              plain FP64 solve (as bs_solve); arena N*M*8 B.
 *   mode BS_SERVE_F32_REFINE : B float[N*M], X double[N*M]; mixed-precision
 *                              solve with one refinement step (as
 *                              bs_solve_refine, BS_REFINE_FACTOR); arena
 *                              N*M*12 B.
 * Layout is interleaved.  The worker admits queued requests in arrival order
 * while their arena bytes fit, puts every newly admitted request into one
 * batch and runs the batch on one of `n_streams` streams: host-to-device
 * copies, one replay of a captured CUDA graph (work-list copy + one grouped
 * persistent launch for all requests of the batch), device-to-host copies.
 * Batches overlap across streams; requests arriving meanwhile join the next
 * batch as soon as memory and a stream are free.  A request's result is
 * bitwise the same whatever else shares its batch (one lane per system, the
 * arithmetic of the standalone one-thread-per-system solves).
 * Request states: 0 queued, 1 running, 2 done, 3 cancelled, 4 failed.
 * Latency = host submission to host-observed completion.
 * ---------------------------------------------------------------------- */
typedef struct bs_server_s* bs_server;
enum { BS_SERVE_F64 = 0, BS_SERVE_F32_REFINE = 1 };

/* Creates a server on the current device (1 <= n_streams <= 16).  Fails with
 * BS_ENOMEM if the budget cannot be reserved. */
bs_status bs_server_create(size_t hbm_budget_bytes, int n_streams, bs_server* out);
/* Stops the worker (in-flight batches finish first) and frees everything.
 * Requests still queued are dropped. */
bs_status bs_server_destroy(bs_server s);
/* Queues one request; *request_id identifies it.  BS_ENOMEM if the request
 * alone exceeds the budget (it could never be admitted); 1 <= M <= 524288.
 * host_B and host_X must be page-locked host memory (cudaHostAlloc,
 * cudaHostRegister, torch's pin_memory): copies from pageable memory would
 * block the worker; other memory is rejected with BS_EINVAL.  The handle is
 * pinned until the request has finished: bs_destroy refuses it meanwhile. */
bs_status bs_server_submit(bs_server s, bs_handle h, const void* host_B, void* host_X, int mode, int64_t M,
                           int64_t* request_id);
/* Non-blocking state query; *latency_s is -1 until the request has finished. */
bs_status bs_server_poll(bs_server s, int64_t request_id, int* state, double* latency_s);
/* Blocks until the request has finished or `timeout_s` passed (BS_ETIMEOUT). */
bs_status bs_server_wait(bs_server s, int64_t request_id, double timeout_s, int* state);
/* Cancels a request that has not been admitted yet (BS_EINVAL otherwise). */
bs_status bs_server_cancel(bs_server s, int64_t request_id);
/* Forgets a finished request (its id becomes unknown). */
bs_status bs_server_release(bs_server s, int64_t request_id);
/* Stops (paused != 0) or resumes admitting new batches; running batches
 * continue.  For draining and for tests. */
bs_status bs_server_pause(bs_server s, int paused);
/* Host-side fault injection for tests: the queued request fails at admission
 * as a failed device copy would make it fail (its memory is released, the
 * other requests are unaffected). */
bs_status bs_server_fail_on_admit(bs_server s, int64_t request_id);
/* Counters, first n of: batches, completed, failed, queued, running, arena
 * bytes in use, peak arena bytes, arena size, most requests in one batch,
 * most batches in flight at once.  Returns BS_ECUDA if a batch ever failed. */
bs_status bs_server_stats(bs_server s, int64_t* out, int n);

/* Launch tuning knobs (process-wide; 0 restores the default).
 *  BS_OPT_INFLIGHT_BYTES: upper bound on the bytes of forward-sweep values
 *    that all systems in flight keep between their two sweeps, which sets how
 *    many systems run at once (default 0: no bound, every system that fits
 *    on the device runs at once).
 *  BS_OPT_BLOCKS_PER_SM: cap on resident CTAs per SM of the persistent grids
 *    (default 0: as many as shared memory and threads allow).
 *  BS_OPT_SWEEP_KERNEL: 0 (default) and 1 use the streaming kernels; 2 lets
 *    FP32-arithmetic interleaved solves use the on-chip kernel (forward values
 *    kept in shared memory, rows moved by TMA) where the shape qualifies.  The
 *    on-chip kernel moves only the compulsory bytes but fits ~100 systems per
 *    SM at N = 512, too few to hide latency; it is slower on the workloads
 *    measured so far and kept as an option.
 *  BS_OPT_TMA_AHEAD: row chunks (32 rows each) the on-chip kernel keeps in
 *    flight ahead of its forward sweep (default 0: 4).
 *  BS_OPT_PARTITION: row-partitioned solves (not in the paper; for batches
 *    too small to fill the GPU one thread per system).  bs_factor prepares,
 *    for N >= 384 when the matrix's spikes decay within a quarter of a block,
 *    a split of the rows into P blocks (2 <= P <= 32, blocks of >= 192 rows)
 *    for A and for A^T.  A solve then runs one thread per (system, block) on
 *    the matrix without its entries that couple different blocks, solves a
 *    banded system of the 2h (P - 1) block-edge values per system (h = 1
 *    tridiagonal, 2 pentadiagonal; its LU computed once with the handle), and
 *    corrects the rows near the block edges; the result is the same as the
 *    unpartitioned solve's to rounding.  0 (default): used by bs_solve, bs_solve_bf16,
 *    bs_solve_adjoint and bs_adi_halfstep when the batch has fewer than 256
 *    systems per SM (except that bs_solve, bs_solve_bf16 and bs_solve_adjoint
 *    take the two-ended sweep of BS_OPT_TWISTED instead of a two-block
 *    partition);
 *    1: never; 2: whenever the handle has one.
 *  BS_OPT_UNIFORM: uniform pentadiagonal solves (Sec. 4.1, cuPentUniformBatch).
 *    bs_factor marks a pentadiagonal handle uniform when every in-range entry
 *    of its outermost sub-diagonal (a_i, i = 3..N, 1-based) is the same value
 *    eps; the unpartitioned FP32-arithmetic sweeps of bs_solve (BS_F32),
 *    bs_solve_bf16 and bs_solve_adjoint (BS_F32) then read eps as a scalar
 *    instead of a coefficient array (one array fewer staged and read per
 *    row; the same number of operations, in a different order, so results
 *    differ from the general sweeps by rounding only).  On GB300 the general
 *    FP32 sweeps read each row's coefficients as one packed record, so the
 *    scalar saves no load and its longer dependency chain makes it equal or
 *    slower (FP64 solves, bound by the FP64 pipe, are 3 % slower with it);
 *    it is therefore used only on request.  0 (default) and 1: the general
 *    sweeps; 2: the scalar form for uniform handles (FP32 arithmetic).
 *  BS_OPT_TWISTED: two-ended solves for small batches (not in the paper).
 *    bs_factor also prepares, for a matrix (and for its transpose) whose
 *    row-reversed elimination (A = U' L') meets no bad pivot, the meeting
 *    rows of a solve in which two threads share a system: one eliminates
 *    the top rows with A = L U / L R, the other the bottom rows with
 *    A = U' L'; the meeting rows (one in the middle of a tridiagonal
 *    system, two of a pentadiagonal one) are solved from both, and each
 *    thread back-substitutes outward -- half the dependent steps per system.
 *    The result equals the one-thread solve to rounding.
 *    0 (default): used by bs_solve, bs_solve_bf16 and bs_solve_adjoint
 *    (interleaved layout) when a batch has at most 128 systems per SM and
 *    would not be row-partitioned into more than two blocks
 *    (BS_OPT_PARTITION 2 keeps the partition); 1: never; 2: whenever the
 *    handle allows (interleaved, not partitioned).
 *  BS_OPT_CTA_THREADS: threads per CTA of the streaming sweep and ADI
 *    kernels that size their CTAs by policy.  0 (default): the policy (128,
 *    halved while the batch would give fewer than two CTAs per SM, down to
 *    32; row-partitioned FP64 ADI half-steps then take whichever of 32, 64
 *    and 128 loads the busiest SM least); 32, 64 or 128: that size; a
 *    multiple of 64 up to 512: that size for the windowed sweeps
 *    (BS_OPT_WINDOW), 128 for the other kernels.  Other values are rejected
 *    (BS_EINVAL).  The result does not depend on it.
 *  BS_OPT_F64_PAIRS: arithmetic of the FP64 (BS_F64) solves of bs_solve and
 *    bs_solve_adjoint that run one thread per system (not row-partitioned,
 *    not two-ended), interleaved layout (not in the paper).  GB300 issues FP64 instructions at ~1/66 of the FP32 rate, so
 *    these sweeps carry every value as an unevaluated sum of two FP32 numbers
 *    (48 significant bits) formed with error-free products and sums, and
 *    convert the FP64 data with integer operations: FP64 in, FP64 out,
 *    relative error a few units of 2^-48 (about 1e-14) against the exact
 *    solution of the FP64 data instead of ~1e-16.  bs_factor admits a matrix
 *    for it when every sweep coefficient has magnitude in [2^-100, 2^100)
 *    (or is 0) and the sweeps' gains are at most 2^24 (intermediates at most
 *    2^24 times the largest input); other handles always take native FP64.
 *    A periodic handle also carries its Sherman-Morrison sum and correction
 *    in pairs (bs_factor_periodic scales the two weight vectors by a power
 *    of two and admits them when, so scaled, sum |pw| <= 2^20 and
 *    max |pc| lies in [2^-40, 2^20]).  A system that meets an input outside
 *    the pairs' range (nonzero |x| < 2^-72 or >= 2^101, for a periodic
 *    handle >= 2^80; inf, NaN) continues in native FP64 from that row on.  0 (default): pairs where admitted, two systems per thread when
 *    the batch has at least 2 x 256 systems per SM (else one); 1: native
 *    FP64 always; 2: pairs with one system per thread; 3: pairs with two
 *    systems per thread (even M and 16-byte aligned data).  The FP64 steps
 *    of bs_cn_steps follow it too (1: native FP64; otherwise pairs where
 *    admitted, one system per thread).
 *  BS_OPT_WINDOW: windowed sweeps that keep the forward-sweep values on chip
 *    (not in the paper).  For the matrices the method targets, a backward
 *    sweep started from zero at some row instead of from the true solution
 *    there agrees with the true one, a few tens of rows above it, to 2^-50
 *    of the system's largest value (2^-28 for FP32 arithmetic): bs_factor
 *    measures that distance Lw for A and A^T.  A windowed sweep then solves
 *    each system in blocks of rows held in shared memory: the backward sweep
 *    of a block starts from zero at the block's end and writes the rows more
 *    than Lw above it; the next block's backward sweep passes through the
 *    block's last Lw rows again and writes them.  B is read once and X
 *    written once, instead of the forward values also going to memory and
 *    back, at the price of Lw extra backward steps per block; the result
 *    differs from the two-sweep solve by at most 2^-50 (2^-28) of the
 *    system's largest value per row.  Used by the one-thread-per-system
 *    interleaved solves of bs_solve and bs_solve_adjoint (BS_F32) and by
 *    bs_solve_bf16 (even M) when the handle has a window (non-periodic,
 *    decay within 28 rows for FP32 arithmetic; 52 rows for pairs).  The FP64
 *    solves in pairs are bound by instruction issue, where the extra backward
 *    steps cost more than the round trip of the forward values through
 *    memory saves, so they use windows only on request.  0 (default): FP32
 *    arithmetic where available; 1: never; 2: FP32 and pair arithmetic. */
typedef enum {
  BS_OPT_INFLIGHT_BYTES = 0,
  BS_OPT_BLOCKS_PER_SM = 1,
  BS_OPT_SWEEP_KERNEL = 2,
  BS_OPT_TMA_AHEAD = 3,
  BS_OPT_PARTITION = 4,
  BS_OPT_UNIFORM = 5,
  BS_OPT_TWISTED = 6,
  BS_OPT_CTA_THREADS = 7,
  BS_OPT_F64_PAIRS = 8,
  BS_OPT_WINDOW = 9,
  BS_OPT_COUNT = 10
} bs_option;
bs_status bs_set_option(int opt, int64_t value);

/* Measurement aid (the paper has no counterpart): runs a short kernel of
 * independent FP64 fused multiply-adds on `stream`, waits for it, and stores
 * the device's FP64 FMA rate in FMA instructions per second.  This is the
 * ceiling of the sweeps that compute in native FP64 (on GB300 they are bound
 * by it before HBM).  Allocates and frees 8 bytes of device memory. */
bs_status bs_measure_fp64_rate(double* fma_per_s, bs_stream stream);

/* Sticky device-side status of the kernels with bounded waits (the on-chip
 * TMA sweeps): 0 = no problem, 1 = a wait for a TMA load ran out of its
 * iteration limit (the kernel then abandoned its tile; results of that launch
 * are invalid).  Synchronous (reads device memory); `reset` != 0 clears it. */
bs_status bs_device_status(int* code, int reset);

/* Last error message of the calling thread (static storage, never NULL). */
const char* bs_last_error(void);
const char* bs_strerror(bs_status s);

#ifdef __cplusplus
}
#endif

#endif /* BSOLVE_H */
