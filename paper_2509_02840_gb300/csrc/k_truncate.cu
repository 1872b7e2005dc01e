// Read-side truncation of the bidiagonal factorization (Sec. 2, Eq. trBD):
// A_r = L R^T with L(:, k) = alpha_i q_i + beta_{i-1} q_{i-1} and R(:, k) = p_i
// for the kept indices i.  The host picks the indices; this kernel forms the
// columns of L and R in FP64 from the device-resident factors, with separately
// rounded products and sum (the operations of the definition), so that in the
// FP64 form L and R are exact copies of the definition's values.
#include "bdu_internal.cuh"

namespace bdu {
namespace {

template <typename T>
__global__ void k_truncate(const T *__restrict__ Q, int64_t m, const T *__restrict__ P, int64_t n,
                           const int32_t *__restrict__ idx, const double *__restrict__ alpha,
                           const double *__restrict__ beta, int r, double *__restrict__ L,
                           double *__restrict__ R) {
  const int64_t rows = m > n ? m : n;
  const int64_t total = rows * r;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(q / rows);
    const int64_t row = q - (int64_t)k * rows;
    const int i = idx[k] - 1;  // 0-based column of q_i, p_i
    if (row < m) {
      const double a = __dmul_rn(alpha[k], (double)Q[(size_t)i * m + row]);
      L[(size_t)k * m + row] = i == 0 ? a : __dadd_rn(a, __dmul_rn(beta[k], (double)Q[(size_t)(i - 1) * m + row]));
    }
    if (row < n) R[(size_t)k * n + row] = (double)P[(size_t)i * n + row];
  }
}

}  // namespace

cudaError_t launch_truncate(int precision, const void *Q, int64_t m, const void *P, int64_t n, const int32_t *idx,
                            const double *alpha, const double *beta, int r, double *L, double *R, cudaStream_t s) {
  if (r <= 0) return cudaSuccess;
  const int64_t total = (m > n ? m : n) * (int64_t)r;
  const int threads = 256;
  const int64_t want = (total + threads - 1) / threads;
  const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
  if (precision == BDU_FP64)
    k_truncate<double><<<blocks, threads, 0, s>>>((const double *)Q, m, (const double *)P, n, idx, alpha, beta, r, L, R);
  else
    k_truncate<float><<<blocks, threads, 0, s>>>((const float *)Q, m, (const float *)P, n, idx, alpha, beta, r, L, R);
  return cudaGetLastError();
}

}  // namespace bdu
