// Orthogonality control of the mixed form (Q, P stored in FP32), the
// periodic check the paper applies to its long update streams (Sec. 4.2:
// loss of orthogonality is monitored and the factors are re-orthogonalized
// a few times).
//
// Probe: ||X^T X - I||_2 for X = Q (m x m) or P (n x n), estimated by power
// iteration on the symmetric E = X^T X - I: z = X^T (X x) - x, x <- z/||z||.
// Each product reads X once, coalesced, with FP64 accumulation.
//
// Re-orthogonalization: one Newton-Schulz step towards the polar factor,
// X <- X (3I - X^T X) / 2 = X - X E / 2 with E = X^T X - I.  It changes the
// represented A by O(||E||) relative, and shrinks ||E|| to O(||E||^2).  E is
// small (~1e-5), so it only needs to be right in absolute terms: its
// off-diagonal entries are sums of products of nearly orthogonal columns whose
// partial sums stay ~1/sqrt(k), and a 3xTF32 tensor-core GEMM (FP32 accuracy,
// launch_gemm_tc) gets them to ~1e-7; the diagonal, where the partial sums
// grow to 1, is formed in FP64.  X E / 2 is a correction of relative size
// ||E||, so plain TF32 (relative error ~5e-4 of a value ~1e-5 |X|) stays far
// below X's FP32 rounding.  (FP64 GEMMs would cost ~0.25 s at k = 4096 on
// GB300's FP64 rate.)
#include "bdu_internal.cuh"

namespace bdu {
namespace {

// y = X x (X column-major k x k, FP32 or FP64; x, y FP64)
template <typename TX>
__global__ void k_xv(const TX *__restrict__ X, int64_t ld, int k, const double *__restrict__ x,
                     double *__restrict__ y) {
  __shared__ double xs[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  for (int j0 = 0; j0 < k; j0 += 256) {
    __syncthreads();
    if (j0 + threadIdx.x < k) xs[threadIdx.x] = x[j0 + threadIdx.x];
    __syncthreads();
    const int jn = min(256, k - j0);
    if (i < k)
      for (int jj = 0; jj < jn; jj++) acc = fma((double)X[(size_t)(j0 + jj) * ld + i], xs[jj], acc);
  }
  if (i < k) y[i] = acc;
}

// z = X^T y - x, and accumulators: acc[0] += ||z||^2 (one warp per column)
template <typename TX>
__global__ void k_xtv(const TX *__restrict__ X, int64_t ld, int k, const double *__restrict__ y,
                      const double *__restrict__ x, double *__restrict__ z, double *__restrict__ acc) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= k) return;
  const TX *col = X + (size_t)warp * ld;
  double s = 0.0;
  for (int i = lane; i < k; i += 32) s = fma((double)col[i], y[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const double v = s - x[warp];
    z[warp] = v;
    atomicAdd(&acc[0], v * v);
  }
}

__global__ void k_normalize(const double *__restrict__ z, double *__restrict__ x, int k,
                            const double *__restrict__ acc) {
  const double nrm = sqrt(acc[0]);
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) x[i] = z[i] * inv;
}

__global__ void k_start_vector(double *__restrict__ x, int k) {
  // a fixed vector with no special structure, norm 1
  const double scale = rsqrt((double)k);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    unsigned h = (unsigned)i * 2654435761u;
    h ^= h >> 15;
    x[i] = ((h & 1) ? 1.0 : -1.0) * scale * (1.0 + 0.25 * ((h >> 8) & 3));
  }
}

// E(i, i) = sum_r X(r, i)^2 - 1 in FP64 (X rows x k, E with leading
// dimension lde; one warp per column)
__global__ void k_diag_gram(const float *__restrict__ X, int64_t rows, int k, float *__restrict__ E, int64_t lde) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= k) return;
  const float *col = X + (size_t)warp * rows;
  double s = 0.0;
  for (int64_t i = lane; i < rows; i += 32) {
    const double v = (double)col[i];
    s = fma(v, v, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) E[(size_t)warp * lde + warp] = (float)(s - 1.0);
}

}  // namespace

// ws: 3*k+1 doubles of workspace (x, y, z, acc).  The estimate (||E x|| for the
// final unit x, a lower bound that converges to ||E||_2) is sqrt(ws[3*k]).
template <typename TX>
static cudaError_t probe(const TX *X, int k, double *ws, int iters, cudaStream_t s) {
  double *x = ws, *y = ws + k, *z = ws + 2 * k, *acc = ws + 3 * k;
  const int th = 256;
  const int bl = (k + th - 1) / th;
  k_start_vector<<<bl, th, 0, s>>>(x, k);
  for (int it = 0; it < iters; it++) {
    cudaMemsetAsync(acc, 0, sizeof(double), s);
    k_xv<TX><<<bl, th, 0, s>>>(X, k, k, x, y);
    k_xtv<TX><<<(k * 32 + th - 1) / th, th, 0, s>>>(X, k, k, y, x, z, acc);
    k_normalize<<<bl, th, 0, s>>>(z, x, k, acc);
  }
  return cudaGetLastError();
}

cudaError_t launch_ortho_probe(int precision, const void *X, int k, double *ws, int iters, cudaStream_t s) {
  if (precision == BDU_FP64) return probe<double>((const double *)X, k, ws, iters, s);
  return probe<float>((const float *)X, k, ws, iters, s);
}

// One Newton-Schulz step on X (rows x k, FP32, leading dimension rows; a
// square factor or the thin factor of rank-k tracking), with the workspace
// reorth32_workspace gives: E (k x k, leading dimension kp = k rounded up to
// a multiple of 4) and W (a padded copy of X when rows is not a multiple of
// 4, then X^T with leading dimension kp).
cudaError_t launch_reorth32(float *X, int64_t rows, int k, float *E, float *W, int *status, cudaStream_t s) {
  const int64_t kp = (k + 3) / 4 * 4, rp = (rows + 3) / 4 * 4;
  // E = X^T X (3xTF32): X's columns, k-contiguous rows of the product
  const float *A1 = X;
  int64_t s1 = rows;
  cudaError_t e = cudaSuccess;
  if (rows % 4 != 0 || (uintptr_t)X % 16 != 0) {
    e = launch_pad_copy32(X, rows, k, W, rp, s);
    A1 = W;
    s1 = rp;
  }
  if (e == cudaSuccess) e = launch_gemm_tc(3, A1, s1, A1, s1, k, k, (int)rows, E, 1, kp, 1.0f, 0, status, s);
  if (e != cudaSuccess) return e;
  // its diagonal in FP64, minus 1
  k_diag_gram<<<(k * 32 + 255) / 256, 256, 0, s>>>(X, rows, k, E, kp);
  // X <- X - X E / 2 (TF32), from X^T so that the contracted index is contiguous
  e = launch_transpose32(X, rows, k, W, kp, s);
  if (e == cudaSuccess) e = launch_gemm_tc(1, W, kp, E, kp, (int)rows, k, k, X, 1, rows, -0.5f, 1, status, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace bdu
