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
// partial sums stay ~1/sqrt(k), and an FP32 GEMM (two plain cuBLAS SGEMMs, no
// tensor-core rounding) gets them to ~1e-7; the diagonal, where the partial
// sums grow to 1, is formed in FP64.  X E / 2 is a correction of relative size
// ||E||, so its FP32 rounding is negligible.  (FP64 GEMMs would cost ~0.25 s at
// k = 4096 on GB300's FP64 rate; these take a few ms.)
#include <cublas_v2.h>

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

__global__ void k_minus_identity(double *__restrict__ E, int64_t ld, int k) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) E[(size_t)i * ld + i] -= 1.0;
}

// E(i, i) = sum_r X(r, i)^2 - 1 in FP64 (X rows x k, one warp per column)
__global__ void k_diag_gram(const float *__restrict__ X, int64_t rows, int k, float *__restrict__ E) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= k) return;
  const float *col = X + (size_t)warp * rows;
  double s = 0.0;
  for (int64_t i = lane; i < rows; i += 32) {
    const double v = (double)col[i];
    s = fma(v, v, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) E[(size_t)warp * k + warp] = (float)(s - 1.0);
}

// X = X - W / 2 (FP32 entries, the difference formed in FP64 and rounded once)
__global__ void k_finish_reorth32(const float *__restrict__ W, float *__restrict__ X, int64_t count) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x)
    X[q] = (float)((double)X[q] - 0.5 * (double)W[q]);
}

// X = (float)(Xd - W / 2)
__global__ void k_finish_reorth(const double *__restrict__ Xd, const double *__restrict__ W,
                                float *__restrict__ X, int64_t count) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x)
    X[q] = (float)(Xd[q] - 0.5 * W[q]);
}

__global__ void k_widen(const float *__restrict__ s, double *__restrict__ d, int64_t count) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x)
    d[q] = (double)s[q];
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

// One Newton-Schulz step on X (k x k, FP32) using three k*k FP64 buffers.
cudaError_t launch_reorth(float *X, int k, double *Xd, double *E, double *W, void *cublas_handle,
                          cudaStream_t s) {
  cublasHandle_t hb = (cublasHandle_t)cublas_handle;
  if (cublasSetStream(hb, s) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  const int64_t cnt = (int64_t)k * k;
  k_widen<<<1216, 256, 0, s>>>(X, Xd, cnt);
  const double one = 1.0, zero = 0.0;
  if (cublasDgemm(hb, CUBLAS_OP_T, CUBLAS_OP_N, k, k, k, &one, Xd, k, Xd, k, &zero, E, k) != CUBLAS_STATUS_SUCCESS)
    return cudaErrorUnknown;
  k_minus_identity<<<(k + 255) / 256, 256, 0, s>>>(E, k, k);
  if (cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, k, k, k, &one, Xd, k, E, k, &zero, W, k) != CUBLAS_STATUS_SUCCESS)
    return cudaErrorUnknown;
  k_finish_reorth<<<1216, 256, 0, s>>>(Xd, W, X, cnt);
  return cudaGetLastError();
}

// One Newton-Schulz step on X (rows x k, FP32, leading dimension rows; a
// square factor or the thin factor of rank-k tracking), E: k*k and W: rows*k
// floats of workspace.
cudaError_t launch_reorth32(float *X, int64_t rows, int k, float *E, float *W, void *cublas_handle,
                            cudaStream_t s) {
  cublasHandle_t hb = (cublasHandle_t)cublas_handle;
  if (cublasSetStream(hb, s) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  if (cublasSetMathMode(hb, CUBLAS_PEDANTIC_MATH) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  const float one = 1.0f, zero = 0.0f;
  const int r = (int)rows;
  // E = X^T X (FP32; its diagonal is replaced by the FP64 one minus 1)
  if (cublasSgemm(hb, CUBLAS_OP_T, CUBLAS_OP_N, k, k, r, &one, X, r, X, r, &zero, E, k) != CUBLAS_STATUS_SUCCESS)
    return cudaErrorUnknown;
  k_diag_gram<<<(k * 32 + 255) / 256, 256, 0, s>>>(X, rows, k, E);
  if (cublasSgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, r, k, k, &one, X, r, E, k, &zero, W, r) != CUBLAS_STATUS_SUCCESS)
    return cudaErrorUnknown;
  k_finish_reorth32<<<1216, 256, 0, s>>>(W, X, rows * k);
  return cudaGetLastError();
}

}  // namespace bdu
