/*
 * bdu.h -- C ABI of the GB300 bidiagonal-update library (libbdu.so).
 *
 * The library keeps a bidiagonal factorization A = Q * Bd * P^T resident on
 * one GPU and updates it under low-rank changes A+ = A + B * C^T with the
 * Givens bidiagonal update (BGU) of Brust & Saunders, "Fast and Accurate
 * SVD-Type Updating in Streaming Data":
 *   - the factorization and its notation: Sec. 1, Eq. bidiag (Q m x m and
 *     P n x n orthogonal, Bd upper bidiagonal with diagonal alpha_i = d[i]
 *     and superdiagonal beta_i = e[i]);
 *   - the update model: Eq. main (B m x r, C n x r) and Sec. 3.2, Eqs. rk1,
 *     bidiagsubproblem, bidiagplus (b+ = Q^T b, c+ = P^T c, Q+ = Q Q1,
 *     P+ = P P1);
 *   - the reduction of Bd + b+ c+^T with Givens rotations and bulge chasing:
 *     Sec. 3.4, Algorithm 2 (Eqs. giv, giv1, gfill), including the m > n
 *     "spike" and the zero-entry handling.
 * Rank r is processed as r rank-1 steps (Sec. 3.2).  The rotation schedule is
 * fixed (the first right vector P(:,1) is never rotated), which makes Bd+
 * unique up to signs; in the FP64 form every result is bit-identical to the
 * library's CPU reference of the same schedule.
 *
 * Conventions for every entry point:
 *   - matrices are column-major, double precision on the host side;
 *   - m, n >= 1.  For m < n the factorization is A = Q L P^T with L lower
 *     bidiagonal (diagonal d[i] = L(i,i), subdiagonal e[i] = L(i+1,i)), the
 *     form whose transpose A^T = P L^T Q^T is the upper form above: the
 *     library holds that transpose and updates it with A^T + C B^T.  Every
 *     entry point still speaks of the caller's A, Q, P, B and C (left
 *     rotations act on Q, right ones on P); in this form Q(:,1), not P(:,1),
 *     is the vector that no rotation touches.  d has min(m, n) entries and e
 *     min(m, n) - 1;
 *   - host pointers are copied in or out and stay owned by the caller; all
 *     device memory is owned by the handle (see bdu_set_allocator);
 *   - functions return a bdu_status and never abort; the message of the most
 *     recent failure of a handle is available from bdu_last_error;
 *   - after BDU_ECUDA or BDU_ETIMEOUT a handle is poisoned: only bdu_read,
 *     bdu_last_error and bdu_destroy are accepted afterwards;
 *   - a handle is used by one host thread at a time (BDU_EBUSY otherwise).
 */
#ifndef BDU_H
#define BDU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bdu_ctx *bdu_handle;

typedef enum {
  BDU_OK = 0,
  BDU_EINVAL = 1,    /* bad argument (null pointer, m or n < 1, r < 0, NaN/Inf input, ...) */
  BDU_ENOMEM = 2,    /* device allocation failed; the handle stays usable */
  BDU_ECUDA = 3,     /* CUDA runtime error; handle poisoned */
  BDU_ETIMEOUT = 4,  /* a bounded device-side wait expired; handle poisoned */
  BDU_ENOTORTH = 5,  /* orthogonality check failed beyond repair */
  BDU_EBUSY = 6,     /* handle in use by another thread */
  BDU_EPOISONED = 7, /* handle poisoned by an earlier failure */
  BDU_EINTERNAL = 8  /* a device-side invariant check failed (band or schedule) */
} bdu_status;

/* Storage/arithmetic form of Q and P. */
enum {
  BDU_FP64 = 0, /* Q, P in FP64; every step in FP64 (bit-identical to the CPU reference) */
  BDU_MIXED = 1 /* Q, P stored and rotated in FP32; projection accumulated, rotations
                   generated and Bd kept in FP64 */
};

typedef struct {
  int precision;      /* BDU_FP64 (default) or BDU_MIXED */
  int nb;             /* tile shape of the rotation apply (all give identical results):
                         0 = picked by the autotuner (default): after the first update
                         of a shape not seen before, each candidate is timed on a
                         scratch copy of Q and P with that update's rotations, which
                         makes that first call wait for the device; choices are kept
                         per (GPU, form, order, SMs) for the process and, if the
                         environment variable BDU_TUNE_FILE names a file, in it (JSON).
                         FP64 form: an even number <= 64 = rows of Q/P per thread
                         block of the shared-memory apply.  Mixed form: 1..4 = a
                         register-resident layout of (columns x rows) per thread
                         12x8, 24x4, 6x16, 18x4; 5 = the shared-memory apply;
                         64, 96, 128 = the blocked tensor-core apply, whose
                         rotations are accumulated into nb x nb orthogonal blocks
                         (nb/2 consecutive chases over a window of nb/2 columns)
                         applied as 3xTF32 products (Sec. 3.2, Eq. bidiagplus);
                         its results agree with the other variants to FP32
                         rounding, not bit for bit.  With 0, a factor wider than
                         every register layout covers (about 8448 columns) uses
                         the blocked apply with nb = 128. */
  double reorth_tol;  /* BDU_MIXED: re-orthogonalize Q (P) when the estimated
                         ||Q^T Q - I||_2 exceeds this; 0 = never (default 5e-6) */
  int check_every;    /* BDU_MIXED: updates between orthogonality estimates (default 10) */
  void *cuda_stream;  /* cudaStream_t used for all work; NULL = library-owned stream */
  int device;         /* CUDA device ordinal (default 0) */
  int engine;         /* bulge-chase engine: 0 = by size (default), 1 = one thread block,
                         2 = a 16-block cluster; all give identical results */
  int overlap;        /* BDU_MIXED, rank-1 updates: 1 = apply each update to Q and P on a
                         second stream while the next update's rotations are generated.
                         The next projection is then formed from Q, P as they were
                         before that application and rotated by its rotations (the same
                         quantity, rounded differently; Sec. 3.2).  Doubles the memory
                         of the rotation records.  0 = off (default); ignored in the
                         FP64 form and when max(m, n) exceeds about 39000. */
  int graphs;         /* 1 = capture the launch sequence of an update (projection, the
                         chase and the applications of each rank-1 column) in a CUDA
                         graph the first time a rank and pair of input buffers are seen,
                         and replay it for later updates with the same ones (default);
                         0 = launch every kernel separately.  Results are identical.
                         Not used for overlapped rank-1 updates or while timing is on.
                         The capture runs on the handle's stream: work that other threads
                         enqueue on that stream during an update would be captured too. */
  int64_t step_budget; /* watchdog of the chase: synchronous steps allowed per rank-1
                         column before the kernel stops and the update fails with
                         BDU_ETIMEOUT (poisoning the handle); 0 = 64 (n + 16) + 4096
                         (default; a column needs about 11 n) */
  int reorth_every;   /* BDU_MIXED: one Newton-Schulz re-orthogonalization step of Q (P)
                         behind the application of a factor's first rank-1 column and
                         then of every reorth_every-th (in the overlapped and rank-r
                         paths on the apply stream, beside the next chase); 0 = only
                         when the check below finds the estimate above reorth_tol;
                         -1 (default) = every max(1, 100 / sqrt(k)) columns for a factor
                         of order k: FP32 rounding in the application moves
                         ||X^T X - I||_2 by about 3e-8 sqrt(k) per column (more in the
                         first), a step leaves ~1e-6, so the 1e-5 tolerance holds after
                         every update; every column for a factor that the blocked
                         tensor-core apply (nb = 64, 96, 128) updates, whose drift
                         is about ten times larger.  Graph replay is used only when the cadence is
                         in the state the graph was captured in. */
} bdu_options;

typedef struct {
  int64_t updates;          /* rank-1 columns processed */
  int64_t rot_left[4];      /* left rotations (on Q) by phase: spike, 1, 2, 3 */
  int64_t rot_right[4];     /* right rotations (on P) by phase */
  int64_t chase_steps;      /* synchronous steps of the bulge-chase engine */
  int64_t reorth_q, reorth_p; /* re-orthogonalizations performed */
  double ortho_q, ortho_p;  /* last estimate of ||Q^T Q - I||_2, ||P^T P - I||_2 (-1 = none) */
  int64_t launches;         /* CUDA kernels launched by the library so far */
  int64_t timed_updates;    /* updates covered by the timings below (see bdu_set_timing) */
  double ms_project;        /* device time of the projection kernels (K1) */
  double ms_chase;          /* device time of rotation generation / bulge chasing (K2) */
  double ms_apply_q;        /* device time of the rotation apply to Q (K3) */
  double ms_apply_p;        /* device time of the rotation apply to P (K3) */
  int64_t apply_launches;   /* apply-kernel launches covered by ms_apply_q + ms_apply_p */
  int64_t device_bytes;     /* device memory currently held by the handle */
  int64_t graph_replays;    /* updates issued by replaying a captured CUDA graph */
  int64_t apply_variant[2]; /* apply tile shape in use for Q, P (the nb values; 0 = default) */
  int64_t tunings;          /* apply variants this handle picked by timing */
} bdu_stats_t;

/* Fills *opt with the defaults listed above. */
void bdu_default_options(bdu_options *opt);

/* Creates a handle holding A = Q diag-band(d, e) P^T on the GPU (upper
 * bidiagonal for m >= n, lower for m < n).
 *   Q: m*m host doubles (column-major), P: n*n, d: k = min(m, n), e: k-1
 *   (may be NULL when k == 1).  Q and P are assumed orthogonal (not checked:
 *   O(m^3)).  opt may be NULL (defaults).
 * Errors: BDU_EINVAL (null pointers, m < 1, n < 1, non-finite input),
 *         BDU_ENOMEM, BDU_ECUDA.  On error *h is set to NULL. */
bdu_status bdu_create(bdu_handle *h, int64_t m, int64_t n, const double *Q, const double *d,
                      const double *e, const double *P, const bdu_options *opt);

/* A+ = A + B C^T with host matrices B (m*r) and C (n*r), column-major
 * (Eq. main).  The call returns once the work is queued on the handle's
 * stream; host buffers are consumed before return.  r == 0 is a no-op.
 * Errors: BDU_EINVAL (null pointer with r > 0, non-finite input), BDU_ENOMEM,
 *         BDU_ECUDA, BDU_EBUSY, BDU_EPOISONED. */
bdu_status bdu_update(bdu_handle h, const double *B, const double *C, int64_t r);

/* As bdu_update with B and C already in device memory (FP64, column-major,
 * leading dimensions m and n).  The buffers must stay valid until the work on
 * the handle's stream has completed. */
bdu_status bdu_update_dev(bdu_handle h, const double *dB, const double *dC, int64_t r);

/* Batched update of many resident factorizations (any mix of m, n and rank):
 * for every i, A_i + B_i C_i^T with device pointers dB[i] (m_i x r[i]) and
 * dC[i] (n_i x r[i]), FP64 column-major.  Rank 1 steps are taken in rounds
 * (round k serves the items with r[i] > k); each round is one launch of each
 * kernel kind -- projection (first round), staging, bulge chasing (one thread
 * block per factorization) and a fused apply whose blocks cover the row slabs
 * of every Q and P in the round.  The results are identical to bdu_update_dev
 * on each handle.  All handles must share a device and precision and appear
 * once.  stream: cudaStream_t for the batch (NULL = the first handle's); the
 * batch is ordered after each handle's queued work and each handle's later
 * work after the batch.  Errors: BDU_EINVAL, BDU_EBUSY, BDU_EPOISONED,
 * BDU_ENOMEM, BDU_ECUDA. */
bdu_status bdu_update_batch(bdu_handle *hs, int count, const double *const *dB, const double *const *dC,
                            const int64_t *r, void *stream);

/* ---- BHU: the bidiagonal Householder update (Sec. 3.3, Algorithm 1, Theorem 1)
 *
 * Algorithm 1 bidiagonalizes B + u v^T (B upper bidiagonal m x n, m >= n;
 * u = Q^T b, v = P^T c, Eq. rk1) with Householder reflectors applied
 * alternately from the left and the right (Sec. 2.1, Eq. house), keeping the
 * transformed matrix in the factored form of Theorem 1 (Eq. comp): nothing
 * dense of size m x n is formed.  Left reflector k zeroes column k below the
 * diagonal (k = 1..n-1, and k = n when m > n); right reflector k+1 zeroes row
 * k right of the superdiagonal (k = 1..n-2), so P's first column is kept.  The
 * products of the reflectors are Q_k = I - Y SL Y^T and P_k = I - W SR W^T
 * (Eq. QP with SL = 2 T^{-1}, SR = 2 R^{-1} of Eq. TR). */

/* Sizes after `steps` iterations of Algorithm 1 (0 <= steps <= n): *kl left
 * and *kr right reflectors, kl = min(steps, n if m > n else n-1),
 * kr = min(steps, n-2), and the bytes of device workspace bdu_bhu_factor
 * needs.  Any output pointer may be NULL.  Errors: BDU_EINVAL (m < n, n < 1,
 * steps out of range). */
bdu_status bdu_bhu_sizes(int64_t m, int64_t n, int64_t steps, int64_t *kl, int64_t *kr,
                         int64_t *workspace_bytes);

/* Columns of U, V one BHU sweep absorbs (bdu_bhu_factor's r). */
#define BDU_BHU_MAX_RANK 8

/* Algorithm 1 on B + U V^T, FP64, every pointer in device memory,
 * column-major:
 *   in:  d (n), e (n-1; may be NULL when n == 1), U (m x r, leading
 *        dimension m), V (n x r, leading dimension n), 1 <= r <=
 *        BDU_BHU_MAX_RANK: the projected columns U = Q^T B, V = P^T C (Eq. rk1);
 *        r > 1 absorbs a rank-r update in one sweep instead of r;
 *   out: alpha (steps), beta (min(steps, n-1); may be NULL when n == 1): the
 *        first `steps` diagonal and superdiagonal entries of the new
 *        bidiagonal (a partial factorization when steps < n, Sec. 3.3);
 *        Y (m x kl, leading dimension m): the normalized vectors y_1..y_kl
 *        (Eq. YW; zeros above row k); W (n x kr, leading dimension n):
 *        w_2..w_{kr+1} (zeros in rows 1..k); SL (kl x kl, leading dimension
 *        kl) and SR (kr x kr, leading dimension kr), upper triangular;
 *   workspace: bdu_bhu_sizes' bytes of device memory, 16-byte aligned, owned
 *        by the caller (not kept past the call's work);
 *   stream: cudaStream_t (NULL = the legacy default stream).
 * The call returns when the work is done (it synchronizes the stream); the
 * outputs are the caller's.  Results are deterministic (fixed summation
 * orders); they equal the dense Householder process up to rounding, not bit
 * for bit.  One cooperative launch runs the loop; its grid barriers are
 * bounded waits.
 * Errors: BDU_EINVAL (sizes, NULL pointers, unaligned workspace), BDU_ECUDA,
 * BDU_ETIMEOUT (a grid barrier ran out). */
bdu_status bdu_bhu_factor(int64_t m, int64_t n, int64_t r, int64_t steps, const double *d, const double *e,
                          const double *U, const double *V, double *alpha, double *beta, double *Y,
                          double *W, double *SL, double *SR, void *workspace, void *stream);

/* A+ = A + B C^T by BHU instead of the Givens update: the r columns in sweeps
 * of up to BDU_BHU_MAX_RANK (direct rank-r absorption): U = Q^T B(:, cols),
 * V = P^T C(:, cols) with the current factors, Algorithm 1 on B + U V^T to
 * completion, Q <- Q - (Q Y) SL Y^T, P <- P - (P W) SR W^T (cuBLAS FP64
 * products) and (d, e) <- (alpha, beta).  FP64 handles only; m < n through the
 * transposed form as bdu_update.  Host (bdu_update_bhu) or device
 * (bdu_update_bhu_dev) B, C as in bdu_update / bdu_update_dev.  The new
 * bidiagonal equals the Givens update's up to the signs of its entries (both
 * keep P's first column; Eq. bidiagplus), not bit for bit.
 * Errors: as bdu_update; BDU_EINVAL for a mixed-form handle. */
bdu_status bdu_update_bhu(bdu_handle h, const double *B, const double *C, int64_t r);
bdu_status bdu_update_bhu_dev(bdu_handle h, const double *dB, const double *dC, int64_t r);

/* ---- The symmetric variant (Sec. 6: the updating algorithms adapted to
 * generate a tridiagonal)
 *
 * A = Q T Q^T, n x n, T symmetric tridiagonal (diagonal a, off-diagonal b).
 * A + rho c c^T = Q (T + rho u u^T) Q^T with u = Q^T c is brought back to
 * tridiagonal form by the Householder process of BHU with one reflector per
 * step applied on both sides: reflector k (k = 1..n-2) is built from column k's
 * entries k+1..n and acts on rows and columns k+1..n, so Q's first column is
 * kept.  Its product is Q_k = I - Y S Y^T (S = 2 T^{-1} of Eq. TR). */

/* Sizes: *k = min(steps, n-2) reflectors, the device workspace bdu_tri_factor
 * needs for `steps` steps, and the workspace bdu_tri_update_dev needs.  Any
 * output may be NULL.  Errors: BDU_EINVAL (n < 1, steps out of range). */
bdu_status bdu_tri_sizes(int64_t n, int64_t steps, int64_t *k, int64_t *workspace_bytes, int64_t *update_bytes);

/* The tridiagonalization of T + rho u u^T, FP64, device pointers:
 *   in:  a (n), b (n-1; may be NULL when n == 1), u (n), rho (finite);
 *   out: alpha (steps), beta (min(steps, n-1); may be NULL when n == 1): the
 *        first `steps` diagonal and off-diagonal entries of the new
 *        tridiagonal; Y (n x k, leading dimension n): normalized reflector
 *        vectors, y_k with zeros in rows 1..k; S (k x k, leading dimension k),
 *        upper triangular, Q_k = I - Y S Y^T;
 *   workspace: bdu_tri_sizes' workspace bytes, 16-byte aligned, the caller's;
 *   stream: cudaStream_t (NULL = the legacy default stream).
 * Returns when the work is done.  Deterministic; equal to the dense Householder
 * process up to rounding.  Errors: BDU_EINVAL, BDU_ECUDA, BDU_ETIMEOUT (a grid
 * barrier ran out). */
bdu_status bdu_tri_factor(int64_t n, int64_t steps, const double *a, const double *b, double rho, const double *u,
                          double *alpha, double *beta, double *Y, double *S, void *workspace, void *stream);

/* A+ = A + rho c c^T in place: Q (n x n, column-major), a (n) and b (n-1) in
 * device memory are replaced by Q+ and the new tridiagonal; c (n) device
 * memory.  u = Q^T c, bdu_tri_factor, then Q <- Q - (Q Y)(S Y^T) (cuBLAS FP64).
 * workspace: bdu_tri_sizes' update bytes, 16-byte aligned.  Returns when the
 * work is done.  Errors: as bdu_tri_factor; BDU_ENOMEM if no cuBLAS handle. */
bdu_status bdu_tri_update_dev(int64_t n, double *Q, double *a, double *b, double rho, const double *c,
                              void *workspace, void *stream);

/* Waits for all queued work and reports device-side failures
 * (BDU_ETIMEOUT, BDU_EINTERNAL, BDU_ECUDA). */
bdu_status bdu_sync(bdu_handle h);

/* Copies the current factorization to host buffers (any may be NULL):
 * Q m*m, d min(m, n), e min(m, n)-1, P n*n.  Synchronizes the handle's
 * stream. */
bdu_status bdu_read(bdu_handle h, double *Q, double *d, double *e, double *P);

/* Copies the rotations of the most recent rank-1 column to host buffers, in
 * the order in which they are applied: side 0 = left rotations (on Q),
 * side 1 = right rotations (on P).  Each rotation is (c[k], s[k], a[k]) with
 * a 1-based pair (a, a+1) and pair update x_a <- c x_a + s x_b,
 * x_b <- -s x_a + c x_b (Eqs. giv, giv1).  The FP64 form returns the FP64
 * coefficients; the mixed form, which keeps only the FP32 coefficients its
 * FP32 factors are rotated with, returns those (exactly, as doubles).
 * *count receives the number of rotations; at most cap are written.
 * Synchronizes. */
bdu_status bdu_read_rotations(bdu_handle h, int side, double *c, double *s, int32_t *a,
                              int64_t cap, int64_t *count);

/* Truncated bidiagonal approximation of the current factorization (Sec. 2,
 * Eq. trBD): with alpha_i = d_i, beta_i = e_i and beta_0 = 0, keeps the r
 * indices i with the largest alpha_i^2 + beta_{i-1}^2 (on ties the lower i),
 * listed in increasing order in idx (1-based), and returns A_r = L R^T with
 * L(:, k) = alpha_i q_i + beta_{i-1} q_{i-1} (m x r) and R(:, k) = p_i (n x r),
 * column-major FP64 (in the mixed form from the FP32 factors), and in *err2
 * the exact error ||A - A_r||_F^2 = the sum of alpha_i^2 + beta_{i-1}^2 over
 * the other indices (Eq. errtrBD; exact for orthogonal Q and P).  For m < n
 * (L lower bidiagonal) the same applies to A^T: the kept indices are those of
 * the largest alpha_i^2 + beta_{i-1}^2 (rows of L), with L(:, k) = q_i and
 * R(:, k) = alpha_i p_i + beta_{i-1} p_{i-1}.  0 <= r <= min(m, n)
 * (BDU_EINVAL otherwise).  Host buffers, any may be NULL; completes deferred
 * work first and synchronizes. */
bdu_status bdu_read_truncated(bdu_handle h, int64_t r, double *L, double *R, int64_t *idx, double *err2);

/* The k largest singular values of the current bidiagonal Bd (those of A when
 * Q and P are orthogonal; Sec. 2), in descending order, computed on the device
 * by multisection with Sturm counts on the Golub-Kahan tridiagonal matrix of
 * Bd (absolute accuracy about 1e-15 of the largest).  0 <= k <= min(m, n)
 * (BDU_EINVAL otherwise); sv is a host buffer of k doubles.  Needs no deferred work to
 * complete (Bd is current after every update); synchronizes. */
bdu_status bdu_singular_values(bdu_handle h, int64_t k, double *sv);

/* Enqueues on the handle's stream every part of earlier updates that the
 * overlapped form defers (the application of the latest rank-1 column to Q
 * and P), so that work the caller enqueues afterwards on that stream sees the
 * updated factors.  Does not wait on the host.  A no-op without overlap. */
bdu_status bdu_flush(bdu_handle h);

/* Statistics since creation.  Synchronizes. */
bdu_status bdu_stats(bdu_handle h, bdu_stats_t *out);

/* Estimates ||Q^T Q - I||_2 and ||P^T P - I||_2 by power iteration (the
 * check the paper applies to long update streams, Sec. 4.2) and stores them
 * in the statistics; q_est / p_est may be NULL.  In the mixed form the same
 * check runs automatically every check_every updates and re-orthogonalizes a
 * factor (X <- X (3I - X^T X) / 2, FP64 products) whose estimate exceeds
 * reorth_tol.  The automatic check never makes an update wait: it is only
 * enqueued, and its result is acted on by the first later update (or batch)
 * that finds it finished, or else by the next call that synchronizes
 * (bdu_sync, bdu_read, bdu_stats, this call).  Synchronizes. */
bdu_status bdu_check_orthogonality(bdu_handle h, double *q_est, double *p_est);

/* Enables (on != 0) or disables per-kernel timing with CUDA events recorded
 * on the handle's stream around each kernel group; the accumulated device
 * times are reported by bdu_stats.  Off by default. */
bdu_status bdu_set_timing(bdu_handle h, int on);

/* Releases all device memory of the handle.  NULL is accepted. */
void bdu_destroy(bdu_handle h);

/* Message for the most recent failure on h (or of a failed bdu_create when
 * h is NULL; thread-local).  Never NULL. */
const char *bdu_last_error(bdu_handle h);

/* Replaces the device allocator used by handles created afterwards
 * (process-wide).  alloc(bytes, device, ctx) returns a device pointer or
 * NULL; release(ptr, device, ctx) frees it.  Passing NULL for both restores
 * cudaMalloc/cudaFree.  Lets a host framework (e.g. PyTorch's caching
 * allocator) own the memory, and lets tests inject allocation failures. */
typedef void *(*bdu_alloc_fn)(size_t bytes, int device, void *ctx);
typedef void (*bdu_free_fn)(void *ptr, int device, void *ctx);
void bdu_set_allocator(bdu_alloc_fn alloc, bdu_free_fn release, void *ctx);

/* Allocation-free FP64 rank-1 update of a factorization held in the caller's
 * own device memory.  The paper has no counterpart; this entry point exists
 * for callers that cannot allocate device memory: a host framework that
 * reserves the whole GPU for its own allocator and forbids foreign cudaMalloc
 * calls, a latency-critical loop in which an allocation (which may
 * synchronize the device) is not acceptable, or an embedding in which the
 * library may not own memory.
 *
 * All pointers are device pointers on the current device, FP64, column-major:
 * Q m*m, d n, e n-1 (may be NULL when n == 1), P n*n are read and replaced by
 * the factorization of A + b c^T; b (m) and c (n) are read.  The result is
 * bit-identical to bdu_update on a handle with the same data.  stream is a
 * cudaStream_t (NULL = the legacy default stream); the call returns after
 * the update has completed on it.
 *
 * Limits: m <= 1024 and n <= 256 (BDU_EINVAL beyond them, before any device
 * work), as well as m >= n >= 1.  Every intermediate lives in one fixed
 * __device__ array of the library (about 5.5 MB, held by every GPU that loads
 * the library until the process exits); no cudaMalloc, cudaFree or allocating
 * library routine is called by this entry point.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the device
 * current, so that first call should come before any stream capture.  Under
 * CUDA's lazy module loading that first call is also when the driver loads
 * the module and commits the array's memory on that device: a caller that
 * lets a host framework reserve the GPU's memory should make its first call
 * before the framework does (it can fail with BDU_ECUDA otherwise).  The
 * looked-up address is kept per device ordinal for the life of the process,
 * so the device's primary context must stay alive (no cudaDeviceReset between
 * calls).  Each call waits for its stream (cudaStreamSynchronize) before it
 * returns.  All calls share the array and each call clears what must start at
 * zero; calls that overlap on the GPU (from several host threads or unordered
 * streams) race on it.
 * Errors: BDU_EINVAL, BDU_ECUDA, BDU_ETIMEOUT (the chase's watchdog ran out),
 * BDU_EINTERNAL (a device invariant check failed) -- status codes only;
 * bdu_last_error is not updated.  After BDU_ETIMEOUT or BDU_EINTERNAL the
 * caller's Q, d, e and P are unchanged (the kernels that write them skip
 * their work when the chase has reported a failure); after BDU_ECUDA their
 * contents are undefined. */
bdu_status bdu_update_rank1_noalloc(int64_t m, int64_t n, double *Q, double *d, double *e,
                                    double *P, const double *b, const double *c, void *stream);

/* ---- Rank-k subspace tracking (Sec. 4, Eqs. lrup, defup, qrlr, equivlrup,
 * bdlrup) --------------------------------------------------------------------
 * A thin factorization A ~ Q1 B P1^T with Q1 (m x k) and P1 (n x k) of
 * orthonormal columns and B k x k upper bidiagonal (diagonal d, superdiagonal
 * e) is updated by A+ = Q1 B P1^T + b c^T and truncated back to rank k:
 *   b+ = Q1^T b, b_perp = b - Q1 b+, delta = ||b_perp|| (Eq. defup; classical
 *   Gram-Schmidt applied twice), likewise c+, c_perp, gamma; the middle matrix
 *   [B 0; 0 0] + [b+; delta][c+; gamma]^T (Eq. equivlrup) is reduced by the
 *   bidiagonal update of this library (Algorithm 2, FP64, on the device) to
 *   Q2 Bbar+ P2^T; then A+ = [Q1, b_perp/delta] Q2 Bbar+ ([P1, c_perp/gamma] P2)^T
 *   exactly (Eq. bdlrup).  The index i with the smallest column norm
 *   alpha_i^2 + beta_{i-1}^2 of Bbar+ (ties: the last such i) is removed with
 *   its row and column (the superdiagonal entry across it is zero) and
 *   Q1+ = [Q1, b_perp/delta] Q2(:, kept), P1+ likewise (cuBLAS GEMMs).
 *   When delta <= 2^-40 ||b|| (b in span(Q1)) delta is taken as 0 and the new
 *   column is the fixed vector z_i = frac(i * 0.6180339887498949) - 0.5
 *   orthogonalized against Q1 in the same way (likewise for c).
 * opt->precision: BDU_FP64, or BDU_MIXED: Q1, P1, Q2, P2 in FP32 (the middle
 * band and its rotations in FP64), FP32 products, one Newton-Schulz step on Q1
 * and P1 after every step, and b in span(Q1) below delta <= 2^-16 ||b||.
 * overlap, check_every and the re-orthogonalization options are not used for
 * the middle matrix (its factors start from the identity at every step).
 * Errors are status codes; the message of the most recent failure is returned by
 * bdu_thin_last_error (of NULL after a failed bdu_thin_create). */
typedef struct bdu_thin_ctx *bdu_thin_handle;

/* Q1: m*k, P1: n*k host doubles (column-major, orthonormal columns, not
 * checked), d: k, e: k-1 (may be NULL when k == 1).  1 <= k < min(m, n),
 * k < 16384.  Errors: BDU_EINVAL, BDU_ENOMEM, BDU_ECUDA. */
bdu_status bdu_thin_create(bdu_thin_handle *h, int64_t m, int64_t n, int64_t k, const double *Q1,
                           const double *d, const double *e, const double *P1, const bdu_options *opt);

/* One step with host vectors b (m) and c (n) (Eq. lrup); returns once it is
 * complete.  *dropped (may be NULL) receives the removed index i (0-based,
 * 0..k) and *err2 (may be NULL) the truncation error
 * ||A+ - Q1+ B+ P1+^T||_F^2 = alpha_i^2 + beta_{i-1}^2 + beta_i^2 (exact for
 * orthonormal factors).  Errors: BDU_EINVAL, BDU_EBUSY, BDU_EPOISONED,
 * BDU_ECUDA, BDU_ETIMEOUT, BDU_EINTERNAL. */
bdu_status bdu_thin_update(bdu_thin_handle h, const double *b, const double *c, int64_t *dropped, double *err2);

/* As bdu_thin_update with b and c in device memory (FP64). */
bdu_status bdu_thin_update_dev(bdu_thin_handle h, const double *db, const double *dc, int64_t *dropped,
                               double *err2);

/* Copies Q1 (m*k), d (k), e (k-1), P1 (n*k) to host buffers (any may be NULL). */
bdu_status bdu_thin_read(bdu_thin_handle h, double *Q1, double *d, double *e, double *P1);

/* Steps taken, and how many of them found b (c) inside span(Q1) (span(P1)). */
bdu_status bdu_thin_stats(bdu_thin_handle h, int64_t *updates, int64_t *in_span_b, int64_t *in_span_c);

const char *bdu_thin_last_error(bdu_thin_handle h);

/* Releases the handle's device memory.  NULL is accepted. */
void bdu_thin_destroy(bdu_thin_handle h);

/* ---- Failure injection ----------------------------------------------------
 * Drives the library's bounded device-side waits and its chase watchdog to
 * expiry without a GPU fault, for tests of failure detection (process-wide:
 * it applies to kernels launched after the call, on every handle and on
 * bdu_update_rank1_noalloc).  site:
 *   BDU_INJECT_NONE: off (the default; value ignored);
 *   BDU_INJECT_STEP_BUDGET: a chase launched with no step budget of its own
 *     (bdu_options.step_budget = 0, and the allocation-free entry point) stops
 *     after `value` synchronous steps per rank-1 column;
 *   BDU_INJECT_APPLY_STALL: the FP32 register-resident rotation apply (mixed
 *     form) starts no copy of rotation records, and its compute warps give up
 *     after `value` polls of a wait;
 *   BDU_INJECT_ROTVEC_STALL: likewise for the rotation of projected vectors
 *     (overlapped mixed form and mixed rank-r updates);
 *   BDU_INJECT_BHU_STALL: the first block of the BHU kernel (bdu_bhu_factor,
 *     bdu_update_bhu) leaves before its first grid barrier, and the other
 *     blocks give up a barrier wait after `value` polls.
 * In each case nothing is in flight when the waits give up; the expiry sets a
 * bit of the handle's device status word, the next synchronizing call reports
 * BDU_ETIMEOUT and the handle is poisoned.  Returns BDU_EINVAL for an unknown
 * site or value < 1 (the setting is then unchanged). */
enum {
  BDU_INJECT_NONE = 0,
  BDU_INJECT_STEP_BUDGET = 1,
  BDU_INJECT_APPLY_STALL = 2,
  BDU_INJECT_ROTVEC_STALL = 3,
  BDU_INJECT_BHU_STALL = 4
};
bdu_status bdu_set_fault_injection(int site, int64_t value);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int bdu_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BDU_H */
