// Internal declarations of libbdu (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bdu.h"

namespace bdu {

// Device-side error bits written to the status word.
enum : int {
  ERR_BAND = 1,      // a write outside the stored band, or a nonzero where the schedule leaves 0
  ERR_CAP = 2,       // a chase produced more rotations than its record slot holds
  ERR_STEPS = 4,     // the chase engine exceeded its step budget (no progress)
  ERR_SCHEDULE = 8,  // an op found a zero where the schedule guarantees a nonzero
  ERR_APPLY = 16,    // a bounded wait of the register-resident apply ran out
  ERR_ROTVEC = 32,   // a bounded wait of the vector rotation ran out
  ERR_RANGE = 64,    // a record named a pair outside the vector (skipped)
  ERR_GEMM = 128,    // a bounded wait of the tensor-core GEMM ran out
  ERR_BHU = 256,     // a grid barrier of the BHU kernel ran out
};

// Failure injection for tests of the bounded waits (bdu_set_fault_injection):
// the site set (BDU_INJECT_*) and its value; site BDU_INJECT_NONE when off.
struct Injection {
  int site;
  long long value;
};
Injection injection();

// The working core M = band + u v^T of one rank-1 step, in global memory.
// 1-based arrays.  dg[o+2][i] = M(i, i+o) for rows i >= 2 and offsets
// o = -2..3; row 1 is kept densely in r1[j] = M(1, j), j = 1..n, in every
// phase.  u has m+2 entries (the spike works on rows n+1..m), v has n+2.
struct BandPtrs {
  double *dg[6];
  double *r1;
  double *v;
  double *u;
};

// Layout of the band buffer: 6 diagonals of length N+2, r1 (n+2), v (n+2),
// u (m+2), all contiguous.
inline int64_t band_doubles(int64_t m, int64_t n) {
  int64_t N = (m > n) ? n + 1 : n;
  return 6 * (N + 2) + 2 * (n + 2) + (m + 2);
}
inline BandPtrs band_ptrs(double *base, int64_t m, int64_t n) {
  int64_t N = (m > n) ? n + 1 : n;
  BandPtrs b;
  for (int o = 0; o < 6; o++) b.dg[o] = base + o * (N + 2);
  b.r1 = base + 6 * (N + 2);
  b.v = b.r1 + (n + 2);
  b.u = b.v + (n + 2);
  return b;
}

// Rotation records of one rank-1 column, grouped by chase ("task") in the
// order in which they must be applied.  Task t's left rotations are
// Lc/Ls/La[t*cap + 0 .. Ln[t]-1] (pairs (a, a+1), 1-based), likewise right.
// The spike chain (m > n) precedes all tasks on the left side.
struct RotStream {
  int T;    // number of tasks
  int cap;  // record slots per task and side
  double *Lc, *Ls, *Rc, *Rs;
  int32_t *La, *Ra, *Ln, *Rn;
  double *Sc, *Ss;
  int32_t *Sa, *Sn;  // spike records; Sn[0] = count
  // FP32 copies (c, s) of the records for the mixed form; null in the FP64 form
  float2 *Lf, *Rf, *Sf;
  int p1;         // chases 0..p1-1 are phase-1 chases (pairs two columns apart)
  int4 *Lm, *Rm;  // per-chase descriptors for the register-resident FP32 apply (T each), or null
  void *tc_ws;    // workspace of the blocked tensor-core apply (mixed form), or null
  size_t tc_ws_bytes;
};

// Number of chases of the schedule for an m x n problem.
inline int num_tasks(int64_t m, int64_t n) {
  int64_t N = (m > n) ? n + 1 : n;
  int64_t p1 = N - 1;
  int64_t p2 = n > 2 ? n - 2 : 0;
  int64_t ilast = (N == n + 1) ? n : n - 1;
  return (int)(p1 + p2 + 2 * ilast);
}
inline int task_cap(int64_t n) { return (int)(n / 2 + 4); }

struct ChaseArgs {
  int m, n;
  BandPtrs band;      // global memory
  double *Ux;         // later columns of U (rx of them, leading dimension m), or null
  double *Vx;         // later columns of V (leading dimension n)
  int rx;
  RotStream st;
  int *status;        // device error word (ERR_* bits)
  unsigned long long *counters;  // [0..3] left by phase, [4..7] right by phase, [8] steps
  int fast;           // 1: fused multiply-add / Newton rotation arithmetic (mixed form)
  int engine;         // 0: by size, 1: one CTA, 2: thread-block cluster
  long long step_budget;  // bound on synchronous steps per column; 0: 64 (n + 16) + 4096
};

// One matrix (Q or P of one factorization) for the batched apply.
struct ApplyItem {
  void *X;
  int64_t ld;
  int nrow, ncol, R, csw, side, with_spike;
  RotStream st;
};

// One projection X^T B for the batched projection.
struct ProjItem {
  const void *X;
  int nrow, ncol, r;
  const double *B;
  double *U;
  int32_t *nz;  // nrow*r indices followed by r counts
};

// Launchers (return the launch error, if any).
cudaError_t launch_chase(const ChaseArgs &a, cudaStream_t s);
// The cluster chase engine keeps the band in its CTAs' shared memory; false
// when (m, n) is too large for that (n above about 48000).
bool chase_cluster_fits(int m, int n);

cudaError_t launch_project(int precision, const void *X, int64_t ld, int nrow, int ncol,
                           const double *B, int64_t ldb, int r, double *U, int64_t ldu,
                           cudaStream_t s);

// status: the device error word (needed by the register-resident FP32 path;
// null selects the shared-memory slab kernel).
// sm_reserve: SMs the register-resident path leaves free (for a chase that
// runs concurrently); desc_ready: the chase descriptors of st are current.
// variant (all give identical results): 0 = the library's choice; FP64 form:
// R > 0 = rows per thread block of the slab kernel (even, <= 64); mixed form:
// 1..4 = a register layout of launch_apply_reg, kSlabVariant = the slab
// kernel.  cudaErrorNotSupported when the variant does not cover the shape.
// gate (slab kernel only; may be null): a device error word; when an earlier
// kernel on the stream has made it nonzero, X is left untouched.
// Mixed form, variant 64, 96 or 128: the blocked tensor-core apply with blocks
// of that order (st.tc_ws must be set); variant 0 uses it (order 128) when no
// register layout covers the shape.
constexpr int kSlabVariant = 5;
// Mixed form: factors of order >= kBlockedFrom take the blocked tensor-core
// apply with blocks of order 128 whenever the variant is left to the library
// (single updates before and after tuning, batches alike), smaller ones a
// tuned FP32 variant; the two round differently, and a fixed rule keeps every
// path of one shape bit-identical.
constexpr int kBlockedFrom = 1024;
inline bool is_tc_variant(int v) { return v == 64 || v == 96 || v == 128; }
cudaError_t launch_apply(int precision, void *X, int64_t ld, int nrow, int ncol,
                         const RotStream &st, int side, bool with_spike, cudaStream_t s,
                         int *status = nullptr, int sm_reserve = 0, bool desc_ready = false,
                         int variant = 0, const int *gate = nullptr);

cudaError_t launch_chase_batch(const ChaseArgs *d_items, int count, int max_n, int max_band_doubles,
                               int fast, cudaStream_t s);
// In a batch, items with n at or above this size get a thread-block cluster each.
constexpr int kClusterBatchMinN = 512;
cudaError_t launch_chase_cluster_batch(const ChaseArgs *d_items, int count, int max_n, int fast,
                                       cudaStream_t s);
void apply_geometry(int precision, int ncol, size_t smem_cap, int *R, int *csw);
cudaError_t launch_apply_reg(float *X, int64_t ld, int nrow, int ncol, const RotStream &st, int side,
                             bool with_spike, int *status, int sm_reserve, bool desc_ready, int layout,
                             cudaStream_t s);
cudaError_t launch_chase_descriptors(const RotStream &st, int side, cudaStream_t s);
cudaError_t launch_apply_spike32(float *X, int64_t ld, int nrow, const RotStream &st, cudaStream_t s);
// The blocked tensor-core apply (mixed form): the rotations of nb/2
// consecutive chases accumulated into nb x nb orthogonal blocks and applied to
// the FP32 factor with tcgen05 3xTF32 MMAs.  nb in {64, 96, 128}; ws holds
// tc_workspace_bytes(ncol, T, nb) bytes.  cudaErrorNotSupported when the
// shape or nb is not covered (nothing launched then).
size_t tc_workspace_bytes(int ncol, int T, int nb);
cudaError_t launch_apply_tc(float *X, int64_t ld, int nrow, int ncol, const RotStream &st, int side,
                            bool with_spike, int *status, bool desc_ready, int nb, void *ws, size_t ws_bytes,
                            cudaStream_t s);
bool rotate_vectors_supported(int m, int n);
cudaError_t launch_rotate_vectors(const double *w_left, double *dst_left, int m, const double *w_right,
                                  double *dst_right, int n, const RotStream &st, bool with_spike, int *status,
                                  cudaStream_t s);
cudaError_t launch_rotate_vector_sets(const double *w_left, double *dst_left, int64_t ldl, int nl, int m,
                                      const double *w_right, double *dst_right, int64_t ldr, int nr, int n,
                                      const RotStream &st, bool with_spike, int *status, cudaStream_t s);
// L(:, k) = alpha[k] q_i + beta[k] q_{i-1} (just alpha[k] q_1 for i = 1) and
// R(:, k) = p_i, i = idx[k] (1-based), in FP64 (L m x r, R n x r, column-major).
cudaError_t launch_truncate(int precision, const void *Q, int64_t m, const void *P, int64_t n, const int32_t *idx,
                            const double *alpha, const double *beta, int r, double *L, double *R, cudaStream_t s);
// The k largest singular values (descending) of the bidiagonal whose
// Golub-Kahan off-diagonal entries squared are b2[0 .. 2n-2] (all on the device).
cudaError_t launch_bidiag_svals(const double *b2, int n, double hi, double pivmin, int k, double *sv,
                                cudaStream_t s);
cudaError_t launch_apply_batch(int precision, const ApplyItem *d_items, const int *d_first, int count,
                               int total_slabs, size_t smem, cudaStream_t s);
cudaError_t launch_project_batch(int precision, const ProjItem *d_items, int count, int max_nrow,
                                 int max_ncol, int max_r, cudaStream_t s);
cudaError_t launch_stage_batch(const ChaseArgs *d_items, const double *const *d_ucol,
                               const double *const *d_vcol, int count, cudaStream_t s);

cudaError_t launch_ortho_probe(int precision, const void *X, int k, double *ws, int iters, cudaStream_t s);
// One Newton-Schulz step with FP32 products and an FP64 diagonal of X^T X
// (E, W: k*k floats of workspace).
// One Newton-Schulz step X <- X - X E / 2, E = X^T X - I, on X (rows x k,
// FP32, column-major, leading dimension rows); E and W: workspace of the
// sizes reorth32_workspace gives (floats); status: the device error word
// (ERR_GEMM).
cudaError_t launch_reorth32(float *X, int64_t rows, int k, float *E, float *W, int *status, cudaStream_t s);
void reorth32_workspace(int64_t rows, int k, size_t *e_floats, size_t *w_floats);

// D = alpha A B + beta D (beta 0 or 1) for FP32 operands on the tensor cores
// (tcgen05, kind::tf32): passes = 3 is 3xTF32 (about FP32 accuracy), 1 plain
// TF32.  K-contiguous operands: A(m, k) at A[m * a_sr + k], B(k, n) at
// B[n * b_sr + k], row strides multiples of 4 and bases 16-byte aligned
// (cudaErrorInvalidValue otherwise); D(m, n) at D[m * d_sm + n * d_sn].
cudaError_t launch_gemm_tc(int passes, const float *A, int64_t a_sr, const float *B, int64_t b_sr, int M, int N,
                           int K, float *D, int64_t d_sm, int64_t d_sn, float alpha, int beta, int *status,
                           cudaStream_t s);
// XT[i + r * ldt] = X[r + i * rows] (X rows x k); Y[r + i * ldy] = X[r + i * rows]
cudaError_t launch_transpose32(const float *X, int64_t rows, int k, float *XT, int64_t ldt, cudaStream_t s);
cudaError_t launch_pad_copy32(const float *X, int64_t rows, int k, float *Y, int64_t ldy, cudaStream_t s);
cudaError_t launch_convert_f64_to_f32(const double *src, float *dst, int64_t count,
                                      cudaStream_t s);
cudaError_t launch_convert_f32_to_f64(const float *src, double *dst, int64_t count,
                                      cudaStream_t s);

// BHU, the bidiagonal Householder update (k_bhu.cu; Sec. 3.3, Algorithm 1).
// kl, kr: left and right reflectors after `steps` iterations; the workspace
// of launch_bhu: ws_doubles doubles and ws_counters zeroed counters.
struct BhuSizes {
  int64_t kl, kr, ws_doubles, ws_counters;
};
BhuSizes bhu_sizes(int64_t m, int64_t n, int64_t steps);
// status: the device status word (ERR_BHU when a grid barrier runs out).
// rk (1..BDU_BHU_MAX_RANK) columns of U (leading dimension ldu) and V (ldv).
cudaError_t launch_bhu(int m, int n, int steps, int rk, const double *d, const double *e, const double *u,
                       int64_t ldu, const double *v, int64_t ldv, double *alpha, double *beta, double *Y, double *W,
                       double *SL, double *SR, double *ws, unsigned *cnt, int *status, cudaStream_t s,
                       int64_t *launches);
// The symmetric variant: the tridiagonalization of T + rho u u^T (n x n; Y
// n x k, S k x k with k = bhu_sizes(n, n, steps).kr; the workspace of
// bhu_sizes(n, n, steps)).
cudaError_t launch_tri(int n, int steps, const double *a, const double *b, double rho, const double *u,
                       double *alpha, double *beta, double *Y, double *S, double *ws, unsigned *cnt, int *status,
                       cudaStream_t s);
cudaError_t launch_bhu_band_get(double *band, int m, int n, double *d, double *e, cudaStream_t s);
cudaError_t launch_bhu_band_put(double *band, int m, int n, const double *d, const double *e, cudaStream_t s);

}  // namespace bdu
