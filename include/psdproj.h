/*
 * psdproj.h -- C ABI of the GB300 (sm_103a) composite-polynomial projection
 * onto the cone of positive semidefinite matrices.
 *
 * The operation (paper: "Factorization-free Orthogonal Projection onto the
 * PSD Cone with Composite Polynomial Filtering"):
 *   Pi(X) = argmin_{Y PSD} ||Y - X||_F / 2                      (Sec. 1)
 * approximated by Algorithm 2:
 *   1. (sigma, q) = largest Ritz pair of a 20-step Lanczos run on X^2  (Sec. 3.4)
 *   2. lam~ = sqrt(sigma + ||X^2 q - sigma q||_2)    (Theorem 2, upper bound of ||X||_2)
 *   3. X_0 = X / lam~
 *   4. X_t = f_t(X_{t-1}) / s_t,  f_t(x) = a_t x + b_t x^3 + c_t x^5, t = 1..T
 *      (coefficients: Table 2, f~*_half, T = 7, or Table 1, f~*_single, T = 10;
 *       s_t: the 1/1.01 resp. 1/1.001 rescale of Sec. 3.4)
 *   5. return lam~ X_0 (I + X_T) / 2  =  (X + lam~ X_0 X_T) / 2
 * Each stage costs three symmetric matrix products (X^2, (X^2)^2,
 * X (a I + b X^2 + c X^4)), so a projection is 3T + 1 products: 22 (half),
 * 31 (single).
 *
 * Conventions shared by every entry point
 *  - Matrices are dense, FP32, column-major with leading dimension ld >= n,
 *    in device memory owned by the caller.  X must be symmetric; the library
 *    reads ONLY the upper triangle, i.e. the elements X[i + j*ld] with
 *    i <= j, and treats X[j + i*ld] as equal to X[i + j*ld].  The output is
 *    written in full (both triangles) and is exactly symmetric.
 *  - out may be the same buffer as X (same pointer and the same ld); any
 *    other overlap is rejected with PSD_ERR_INVALID_ARG.
 *  - Calls are asynchronous on `stream`.  Argument errors are returned
 *    synchronously; numerical and device-side conditions (non-finite input,
 *    a bound that turned out too small, a device wait that timed out) are
 *    written to a psd_info_t in device memory, whose `status` field holds a
 *    psd_status_t.
 *  - No entry point falls back to the CPU.  If the GPU is not an sm_103
 *    device the calls return PSD_ERR_UNSUPPORTED.
 *  - The Lanczos start vector is fixed: v_i = 2 u_i - 1 with
 *    u_i = (SplitMix64(seed + (i+1) * 0x9E3779B97F4A7C15) >> 11) * 2^-53,
 *    seed = 0x243F6A8885A308D3, normalised to unit length.
 */
#ifndef PSDPROJ_H
#define PSDPROJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *psd_stream_t;

typedef enum {
  PSD_OK = 0,
  PSD_ERR_INVALID_ARG = 1, /* bad size, pointer, ld, overlap or precision */
  PSD_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  PSD_ERR_NO_MEMORY = 3,   /* device allocation failed / workspace too small */
  PSD_ERR_NONFINITE = 4,   /* device: NaN or Inf in the input or an iterate */
  PSD_ERR_BOUND = 5,       /* device: max |X_T(i,j)| exceeded 1 + 1e-2: the norm
                              bound was below ||X||_2 and the filter diverged */
  PSD_ERR_TIMEOUT = 6,     /* device: a bounded wait inside a kernel gave up */
  PSD_ERR_UNSUPPORTED = 7, /* no sm_103 device, or precision not built */
  PSD_ERR_CANCELED = 8     /* server: the request was canceled before it ran */
} psd_status_t;

typedef enum {
  PSD_PREC_FP32 = 0,  /* f~*_single (Table 1), T = 10, 31 products; each product
                         is three TF32 tensor-core products of the hi/lo split
                         operands (Ootomo & Yokota 2022), FP32 accumulation */
  PSD_PREC_FP16 = 1,  /* f~*_half (Table 2), T = 7, 22 products, FP16 operands,
                         FP32 accumulation in tensor memory */
  PSD_PREC_BF16 = 2,  /* as FP16 with BF16 operands */
  PSD_PREC_MIXED = 3, /* f~*_half with FP16 iterates; in stages 1-4 the stage
                         polynomial P is an FP16 hi/lo pair (X P as two FP16
                         products), in stages 2-3 Y = X^2 too (Y^2 as three);
                         in stages 1 and 4 P is formed from a single Y with a
                         pair output; FP32 accumulation; 30 tensor products in
                         all */
  PSD_PREC_FP8_EARLY = 4, /* reserved, returns PSD_ERR_UNSUPPORTED: e4m3 iterates in
                             the first stages diverge (the stage-1 coefficients
                             amplify the rounding of X^2 beyond the filter's basin) */
  PSD_PREC_FP8_LATE = 5   /* f~*_half; stages 1-5 as FP16, stages 6-7 on e4m3
                             operands (kind::f8f6f4) with power-of-two per-matrix
                             scales, X_T and the final product in FP16; relative
                             error vs the FP64 filter output ~2-3e-2 */
} psd_precision_t;

/* Per-projection report, written by the device. */
typedef struct {
  int32_t status;        /* psd_status_t of the device-side work */
  int32_t lanczos_steps; /* m <= 20: Lanczos steps run (fewer on breakdown) */
  double lambda_bound;   /* lam~ used to scale X */
  double lanczos_sigma;  /* largest Ritz value of X^2 */
  double lanczos_resid;  /* ||X^2 q - sigma q||_2 */
  double fro_X;          /* ||X||_F (FP64) */
  double max_diag;       /* max_i |X_ii| */
  double overshoot_max;  /* max_ij |X_T(i,j)| of the last stage */
  double compl_resid;    /* <out, X - out> / ||X||_F^2: 0 for the exact projection Pi(X)
                            (Pi(X) and X - Pi(X) are orthogonal), so its size measures the
                            distance from a projection.  Summed in the final product's
                            epilogue (double-float per thread, FP64 per tile, fixed order).
                            NaN where not computed (psd_norm_bound*) */
} psd_info_t;

/* Project one matrix (Algorithm 2).  X: n x n upper triangle read, ld >= n.
 * out: n x n written, leading dimension ld.  Workspace comes from a library
 * cache keyed by (device, stream, n, precision) and is kept until
 * psd_release_workspaces(); the report goes to an internal device record
 * readable with psd_last_info().  n == 0 is a no-op. */
psd_status_t psd_project(int64_t n, const float *X, int64_t ld, float *out,
                         psd_precision_t precision, psd_stream_t stream);

/* As psd_project with a separate output leading dimension, a caller-owned
 * device report (d_info, may be NULL) and an optional caller-owned device
 * workspace of ws_bytes >= psd_workspace_size(n, precision) bytes (NULL: use
 * the library cache).  The workspace must stay untouched until the call has
 * finished on `stream`. */
psd_status_t psd_project_ex(int64_t n, const float *X, int64_t ld, float *out, int64_t ld_out,
                            psd_precision_t precision, psd_info_t *d_info, void *workspace,
                            size_t ws_bytes, psd_stream_t stream);

/* Bytes of device workspace psd_project_ex needs for (n, precision); 0 on bad args. */
size_t psd_workspace_size(int64_t n, psd_precision_t precision);

/* Waits for `stream` and copies the report of the last psd_project call on
 * that stream to *host_info.  PSD_ERR_INVALID_ARG if no call was made. */
psd_status_t psd_last_info(psd_stream_t stream, psd_info_t *host_info);

/* Frees every cached workspace and captured graph (synchronises the device). */
psd_status_t psd_release_workspaces(void);

/* Norm bound alone (Algorithm 2 steps 1-2): writes lam~ and the Lanczos
 * fields of *d_info (device memory).  Same X conventions as psd_project. */
psd_status_t psd_norm_bound(int64_t n, const float *X, int64_t ld, psd_info_t *d_info,
                            psd_stream_t stream);

/* Norm bound that allocates nothing (no counterpart in the paper: an addition
 * of this library).  For callers that must not allocate device memory while
 * they run, e.g. a loop whose device memory is reserved up front by a pool,
 * or a latency-critical loop that cannot take the implicit synchronisation of
 * cudaMalloc.  Same computation and report as psd_norm_bound, for
 * 1 <= n <= 4096 (larger n: PSD_ERR_INVALID_ARG); the scratch lives in a
 * static device array of about 3 MB that every GPU loading the library holds
 * until exit.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress) with that device current; make it before any stream
 * capture.  The address is kept with the CUDA context it was found in and
 * looked up again when the device's current context is another one (after
 * cudaDeviceReset).  All calls share the array: calls whose work overlaps on the GPU
 * (different streams) race and must not be issued; calls on one stream are
 * ordered.  X, d_info: caller-owned device memory as in psd_norm_bound. */
psd_status_t psd_norm_bound_noalloc(int64_t n, const float *X, int64_t ld, psd_info_t *d_info,
                                    psd_stream_t stream);

/* ---- Batched projection of a block-diagonal cone ------------------------ */
/* One block: X, out column-major device matrices of order n (1 <= n <= 1024),
 * upper triangle of X read; info may be NULL. */
typedef struct {
  int64_t n;
  const float *X;
  int64_t ld;
  float *out;
  int64_t ld_out;
  psd_info_t *info;
} psd_block_desc_t;

/* Projects `count` independent blocks with one sequence of grouped launches
 * (each phase of the norm bound -- a mat-vec over every block's upper tiles,
 * the blocks' Lanczos steps --, the cast and each of the 3T + 1 products is
 * one launch over all blocks), captured in a CUDA graph per (device, stream,
 * precision, block orders).  d_descs is an array of `count` descriptors in DEVICE memory; the
 * library reads it back once per call (a synchronous copy of count * 48
 * bytes) to find the plan for the block orders.  Every block's result depends
 * only on that block: it is bit-identical to a batched call with that block
 * alone.  Orders 1..1024; precisions FP16, BF16, MIXED, FP32. */
psd_status_t psd_project_batched(int32_t count, const psd_block_desc_t *d_descs,
                                 psd_precision_t precision, psd_stream_t stream);

/* ---- Building block exposed for tests and users ------------------------- */
/* Flags or-ed into psd_symm_product's `epi` (FP16 / BF16 operands, epi 0-2):
 *   PSD_EPI_GROUPED: run the kernel instance the grouped launches over many
 *     small matrices use (block-diagonal cones; 8 epilogue warps and a shallower
 *     operand ring) -- the same arithmetic per element, so the same bits;
 *   PSD_EPI_F16_PAIR_OUT (FP16, epi 0-1): write C as an FP16 hi/lo pair (hi
 *     at C, lo at C + n*ld elements), the Y and P outputs of the mixed
 *     precision;
 *   PSD_EPI_CTA_PAIR (FP16/BF16 epi 0-3, MIXED epi 0-2, not with
 *     PSD_EPI_GROUPED): run the form the projection uses for its 16-bit and
 *     FP16-pair products, on pairs of SMs (one
 *     tensor-core product of M = 256 per 256 x 256 tile, each SM staging its
 *     128 rows of A and half of B) -- the same bits as the one-SM form. */
#define PSD_EPI_GROUPED 0x100
#define PSD_EPI_F16_PAIR_OUT 0x200
#define PSD_EPI_CTA_PAIR 0x400

/* Symmetric product C = epi(A * B) of two n x n symmetric matrices in the
 * chain's storage (A, B, C share the leading dimension ld, a multiple of 8;
 * pointers 16-byte aligned).  Only the upper tiles of A * B are formed on the
 * tensor cores and mirrored, so C is exactly symmetric.
 *   precision FP16 / BF16: single 16-bit matrices;
 *   precision MIXED: FP16 pairs (epi 0-2), precision FP32: TF32 pairs (FP32
 *     containers): every operand (A, B, C, Y) is two matrices stored back to
 *     back, hi at M and lo at M + n*ld elements, value = hi + lo; the product
 *     is A_hi B_hi + A_hi B_lo + A_lo B_hi in one FP32 accumulator (TF32:
 *     folded every 128 K into a round-to-nearest running sum).
 *   epi 0: C = A B
 *   epi 1: C = a I + b Y + c A B          (Y = aux, same storage and ld)
 *   epi 2: C = (A B) * s
 *   epi 3: C = (Xf + lam * A B) / 2       (FP32 out with leading dim ld_out,
 *                                          Xf = aux FP32 upper triangle, ld_aux)
 *   precision FP8_LATE: single e4m3 matrices (1 byte per element, ld a
 *     multiple of 16); epi 0-2 only, output e4m3.  Every e4m3 matrix holds its
 *     values times a power of two: after the epilogue's own params come
 *     {in_scale, y_scale, out_scale}: the accumulator is multiplied by
 *     in_scale, Y by y_scale, and C is rounded (saturating) from
 *     value * out_scale.
 * params: {a, b, c} for epi 1, {s} for epi 2, {lam} for epi 3 (then the FP8 scales).
 * epi may carry the PSD_EPI_* flags above.
 * d_absmax (may be NULL): device float receiving max |C(i,j)| (atomic max). */
psd_status_t psd_symm_product(int64_t n, const void *A, const void *B, int64_t ld, void *C,
                              int64_t ld_out, psd_precision_t precision, int32_t epi,
                              const double *params, const void *aux, int64_t ld_aux,
                              float *d_absmax, psd_stream_t stream);

/* ---- Request server: continuous batching of projections ------------------
 * Not in the paper: a serving layer that runs Algorithm 2 for many requests
 * at once.  A server owns one device allocation of hbm_budget_bytes, carved at
 * creation into
 *   - an arena of 16-bit rows (row length ldm = max_order rounded up to 64):
 *     a request of order n holds 4 n contiguous rows for X_0, two rotating
 *     iterates and the stage polynomial, the four matrices of one stage, and
 *     ceil(32 T / (2 ldm)) more for the shares of <out, X - out> of its T
 *     final-product tiles (T = nb (nb + 1), nb = ceil(n / 256), an upper bound);
 *   - per-request records (argument block, device state, report), max_batch
 *     of them;
 *   - the Lanczos scratch of two preparation streams (norm bound of order up
 *     to max_order each).
 * A host thread admits queued requests in arrival order while their rows and
 * a record fit, runs their norm bound and X_0 = X / lam~ on a preparation
 * stream, and lets each join the running set at the next step.  A scheduler
 * step is one grouped launch per product (X^2, the polynomial, X P / s_t, the
 * final product) and operand type over the running requests, each at its own
 * stage with its own coefficients.  A step has a work budget (about 0.5 ms of
 * the GPU): requests are served smallest first, each with the next tiles of
 * its current product, and one that completes a product goes on to the next
 * in the same step, so a small request runs a whole stage per step while a
 * large one's products are spread over several steps (it always receives a
 * minimum share).  Requests that finish get their report in the same step.
 *
 * Results: each request's arithmetic (norm bound kernels, tile partition,
 * summation order, coefficients and roundings) is that of psd_project with the
 * same precision, so its output and report are bit-identical to a
 * psd_project call on the same input, however many other requests share its
 * launches.  Precisions: PSD_PREC_FP16 and PSD_PREC_BF16 (others return
 * PSD_ERR_UNSUPPORTED at submit).
 *
 * Threads: every function may be called from any host thread; the server's
 * own thread is the only one that issues GPU work for it. */
typedef struct psd_server psd_server_t;
/* Same type as cudaEvent_t. */
typedef struct CUevent_st *psd_event_t;

/* Creates a server on `device`.  max_order (1..131072)
 * bounds n of every request; max_batch (1..1024) bounds the requests admitted
 * at one time (prepared or running).  Returns PSD_ERR_NO_MEMORY if the budget
 * cannot hold one request of order max_order or the allocation fails,
 * PSD_ERR_UNSUPPORTED if the device is not sm_103. */
psd_status_t psd_server_create(size_t hbm_budget_bytes, int32_t device, int64_t max_order, int32_t max_batch,
                               psd_server_t **server);

/* Queues one projection and returns at once with *ticket.  X (upper triangle,
 * ld >= n) and out (ld_out >= n) are caller-owned device memory that must stay
 * valid and untouched until the ticket completes; out == X with ld_out == ld is
 * allowed.  If `ready` is not NULL the server's streams wait for that event
 * before reading X (record it on the stream that produced X).  n == 0 gives a
 * ticket that is complete at once.  Errors: PSD_ERR_INVALID_ARG (n > max_order,
 * bad pointer, ld or overlap), PSD_ERR_UNSUPPORTED (precision). */
psd_status_t psd_server_submit(psd_server_t *server, int64_t n, const float *X, int64_t ld, float *out,
                               int64_t ld_out, psd_precision_t precision, psd_event_t ready,
                               uint64_t *ticket);

/* *done = 1 once the result is in `out` (the server's GPU work for it has
 * finished).  A completed ticket is retired by the poll or wait that reports
 * it: host_info (may be NULL) receives the report (status: the psd_status_t of
 * the device-side work, or PSD_ERR_CANCELED) and latency_ms (may be NULL) the
 * time from submit to completion.  Unknown or retired tickets:
 * PSD_ERR_INVALID_ARG. */
psd_status_t psd_server_poll(psd_server_t *server, uint64_t ticket, int32_t *done, psd_info_t *host_info,
                             double *latency_ms);

/* Blocks until the ticket completes, then behaves as psd_server_poll with
 * done = 1.  timeout_ms > 0 bounds the wait (PSD_ERR_TIMEOUT, ticket kept). */
psd_status_t psd_server_wait(psd_server_t *server, uint64_t ticket, int64_t timeout_ms, psd_info_t *host_info,
                             double *latency_ms);

/* Cancels a request that is still queued (not admitted): it completes with
 * status PSD_ERR_CANCELED and `out` untouched.  An admitted request runs to
 * the end: PSD_ERR_UNSUPPORTED. */
psd_status_t psd_server_cancel(psd_server_t *server, uint64_t ticket);

typedef struct {
  uint64_t submitted, completed, canceled;
  uint64_t steps;            /* scheduler steps (one stage of every running request) */
  uint64_t kernel_launches;  /* kernels and graphs the server launched */
  int32_t queued, admitted;  /* now */
  int32_t max_running;       /* most requests advanced by one step */
  int32_t pad;
  double p50_ms, p99_ms, max_ms; /* submit -> completion, completed requests */
  int64_t arena_rows, peak_rows; /* arena size and most rows held at once */
} psd_server_stats_t;
psd_status_t psd_server_stats(psd_server_t *server, psd_server_stats_t *stats);

/* Cancels queued requests, lets admitted ones finish, stops the thread and
 * frees the server's memory.  Tickets not yet retired are lost. */
psd_status_t psd_server_destroy(psd_server_t *server);

/* ---- Schedule autotuning of psd_project_batched ------------------------- */
/* No counterpart in the paper: an addition of this library.  The tiles of each
 * grouped product can be dealt to the persistent CTAs in several orders (6
 * candidates: blocks largest first or all tiles by estimated cost in
 * boustrophedon rounds, times a raster group of 4, 8 or 16 for a block's
 * tiles), and for FP16 / BF16 plans the products can run with another tile
 * shape (candidate 6: 256 x 256 tiles on pairs of SMs, one M = 256
 * tensor-core product per K step, each SM staging 128 rows of A and half of
 * B).  No candidate changes any element's arithmetic: results are
 * bit-identical under every schedule and shape.  When a plan is built (first call per
 * device, stream, precision and block orders) the library times one product
 * of the chain's first stage under each candidate (median of 3 after a
 * warm-up, on a private stream, synchronising the device) and keeps the
 * fastest; the choice is cached for the life of the process per precision and
 * size profile (the number of blocks per order bucket n in (2^(k-1), 2^k]), so
 * later plans with the same profile are not re-timed. */

/* Forces schedule `index` (0..5, or 6: the pair shape, FP16 / BF16 only) for
 * plans built after the call; -1 restores autotuning (the default).  Returns
 * the previous setting.  Host-only. */
int32_t psd_batched_force_schedule(int32_t index);

/* Form of the products of plans built after the call: 1 = the chain form
 * (FP16 and BF16, 128-row tiles: all 3T + 1 products of every block in ONE
 * persistent cooperative launch; a block's next product starts as soon as all
 * tiles of its previous product are written, counted per block and product
 * and waited for with a bounded spin), 0 or -1 (the default) = one grouped
 * launch per product.  The chain form measured slower on 512 blocks of orders
 * 16-1024 (5.01 against 4.82 ms): its tiles are bound by the operand feed of
 * their main loops, not by launch boundaries.  Both forms give bit-identical
 * outputs; the complementarity residual of the report is summed from 8 shares
 * per tile in the chain form and 4 otherwise (equal to within rounding).
 * Returns the previous setting.  Host-only. */
int32_t psd_batched_force_form(int32_t form);

/* Form of the batched norm bound of plans built after the call: 1 = ONE
 * launch of resident CTAs that claim work items (a block's start vector,
 * mat-vec tiles, reductions, Lanczos steps, Ritz vector, bound) from a fixed
 * list in order and wait, bounded, only for the block's own earlier items,
 * counted per block, so that the Lanczos steps of large blocks overlap the
 * mat-vec tiles of the others; 0 or -1 (the default) = one grouped launch per
 * phase (about 125 launches, every block of a phase before any block of the
 * next).  The one-launch form measured slower on 512 blocks of orders 16-1024
 * (5.1-5.3 against 4.8-5.0 ms per call): its Lanczos steps, sharing SMs with
 * streaming mat-vec tiles, wait longer on their vector loads than the overlap
 * saves.  Both forms run the same arithmetic per block in the same order:
 * outputs and reports are bit-identical.  Returns the previous setting.
 * Host-only. */
int32_t psd_batched_force_bound(int32_t form);

/* Schedule of the most recently built batched plan: *chosen (0..6),
 * *candidates (7 for FP16 / BF16, else 6) and, if ms is not NULL, the
 * measured ms per candidate (ms[*candidates]; zeros when the schedule was
 * forced or taken from the cache).
 * PSD_ERR_INVALID_ARG before any plan was built.  Host-only. */
psd_status_t psd_batched_last_tuning(int32_t *chosen, int32_t *candidates, float *ms);

/* ---- Deflation of dominant eigenpairs ------------------------------------ */
/* Projection with the dominant eigenpairs taken out first: the remedy Sec. 6
 * (Limitations) names for spectra where a few eigenvalues of large modulus
 * push the rest into the band around 0 that the composite filter resolves
 * poorly (power-law and low-rank-plus-noise spectra).  Not part of
 * Algorithm 2.  Steps, on `stream`:
 *   1. the norm bound of X (Algorithm 2 steps 1-2, Theorem 2), keeping its
 *      Lanczos basis Q_m of K_m(X^2, q_0) and the products X Q_m;
 *   2. Rayleigh-Ritz with X on span(Q_m): eigenpairs (mu_j, w_j) of
 *      Q_m^T X Q_m, Ritz vectors v_j = Q_m w_j;
 *   3. of the kmax pairs of largest |mu_j|, those with
 *      ||X v_j - mu_j v_j||_2 <= 1e-6 lam~ are deflated:
 *      out = X - V diag(mu) V^T;
 *   4. out <- psd_project_ex(out) in place with `precision` (its own norm
 *      bound of the deflated matrix; *d_info is that call's report);
 *   5. out += V diag(max(mu, 0)) V^T.
 * For an invariant span(V) the result is Pi(X) up to the filter's error on
 * the deflated matrix; the residual bound keeps the dropped coupling near
 * 2 sqrt(k) 1e-6 lam~ in the Frobenius norm.  Eigenvalues +-lam of (nearly)
 * equal modulus share one eigenvalue of X^2, so K_m(X^2, q_0) may not
 * separate them; such pairs are deflated only if their residuals pass.
 * X: n x n column-major device matrix, upper triangle read, ld >= n.
 * out: n x n written (both triangles), ld_out >= n; out == X (same ld) is
 * allowed, other overlaps are PSD_ERR_INVALID_ARG.  0 <= kmax <= 16
 * (kmax == 0: plain psd_project_ex).  d_info (may be NULL): device report of
 * step 4.  d_kused (may be NULL): device int32, the number of pairs deflated.
 * Workspace: a library cache keyed by (device, stream, n), kept until
 * psd_release_workspaces(), plus the psd_project_ex cache.
 * Errors: PSD_ERR_INVALID_ARG for bad sizes/pointers, PSD_ERR_UNSUPPORTED off
 * sm_103, PSD_ERR_NO_MEMORY, PSD_ERR_CUDA; device-side statuses as for
 * psd_project_ex (a non-finite X deflates nothing and is reported by step 4). */
psd_status_t psd_project_deflate(int64_t n, const float *X, int64_t ld, float *out, int64_t ld_out,
                                 psd_precision_t precision, int32_t kmax, psd_info_t *d_info,
                                 int32_t *d_kused, psd_stream_t stream);

/* ---- Host-side fault injection (tests) ----------------------------------- */
/* No counterpart in the paper.  Sets a knob of the norm bound's kernels on the
 * current device for calls made after this one (captured graphs included):
 *   PSD_DEBUG_BOUND_SCALE (value > 0, default 1): lam~ is multiplied by value;
 *     below 1 the filter sees a spectrum beyond its basin and the report must
 *     show the overshoot (PSD_ERR_BOUND, or PSD_ERR_NONFINITE when the chain
 *     diverges);
 *   PSD_DEBUG_BARRIER_LIMIT_NS (value >= 0, default 4e9): how long a grid
 *     barrier of the persistent norm bound, or a dependency wait of the
 *     batched one-launch bound (psd_batched_force_bound), waits before it
 *     gives up; 0 makes every wait that is not already satisfied give up at
 *     once, so the bound and a projection built on it report PSD_ERR_TIMEOUT
 *     (every block of a batch; the kernel's CTAs leave at their next wait;
 *     nothing hangs or faults).
 * PSD_ERR_INVALID_ARG for an unknown knob or a value out of range,
 * PSD_ERR_CUDA if the copy to the device failed.  Synchronous. */
#define PSD_DEBUG_BOUND_SCALE 1
#define PSD_DEBUG_BARRIER_LIMIT_NS 2
psd_status_t psd_debug_set(int32_t knob, double value);

/* ---- Host-only queries (no GPU needed) ----------------------------------- */
const char *psd_status_string(psd_status_t status);
/* Copies the library's schedule for `precision`: *T stages, coef[3*t + {0,1,2}]
 * = (a_t, b_t, c_t), post_scale[t] = s_t.  Arrays must hold >= 10 entries
 * (coef >= 30).  Returns PSD_ERR_INVALID_ARG for an unknown precision. */
psd_status_t psd_schedule(psd_precision_t precision, int32_t *T, double *coef, double *post_scale);
/* Kernel launches one psd_project call on `stream` makes for (n, precision),
 * counted from its captured graph (0 before the first such call). */
int32_t psd_kernel_launches(int64_t n, psd_precision_t precision, psd_stream_t stream);
/* Number of tensor-core product launches one projection makes (3T + 1). */
int32_t psd_gemm_count(psd_precision_t precision);
/* Library version string. */
const char *psd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PSDPROJ_H */
