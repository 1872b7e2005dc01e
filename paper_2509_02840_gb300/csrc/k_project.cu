// K1: projection of the update onto the current factors,
//   U = Q^T B (m x r),  V = P^T C (n x r)          (Sec. 3.2, Eq. bidiagsubproblem).
//
// Column i of U is the dot product of column i of Q with B(:, k).  Each
// thread owns one column and accumulates over the rows in increasing order
// with separately rounded multiplies and adds, so that, for FP64 factors,
// the result is identical to the plain definition evaluated in that order.
// Zero entries of B are skipped: adding +0 or -0 to a running sum that
// started at +0 never changes it, so sparse updates (a ratings column, a
// unit vector) cost only their nonzeros.
#include "bdu_internal.cuh"

namespace bdu {
namespace {

template <typename TQ>
__global__ void k_project(const TQ *__restrict__ X, int64_t ld, int nrow, int ncol,
                          const int32_t *__restrict__ nzidx, const int32_t *__restrict__ nzcnt,
                          const double *__restrict__ B, int64_t ldb, int r,
                          double *__restrict__ U, int64_t ldu) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncol) return;
  const TQ *x = X + (size_t)i * ld;
  for (int k = 0; k < r; k++) {
    const double *b = B + (size_t)k * ldb;
    double acc = 0.0;
    const int cnt = nzcnt[k];
    const int32_t *idx = nzidx + (size_t)k * nrow;
    for (int q = 0; q < cnt; q++) {
      const int l = idx[q];
      acc = __dadd_rn(acc, __dmul_rn((double)x[l], b[l]));
    }
    U[(size_t)k * ldu + i] = acc;
  }
}

// Row indices of the nonzeros of each column of B (in increasing order).
__global__ void k_nonzeros(const double *__restrict__ B, int64_t ldb, int nrow, int r,
                           int32_t *__restrict__ nzidx, int32_t *__restrict__ nzcnt) {
  const int k = blockIdx.x;
  if (k >= r) return;
  const double *b = B + (size_t)k * ldb;
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  // chunked stream compaction preserving order
  for (int l0 = 0; l0 < nrow; l0 += blockDim.x) {
    const int l = l0 + threadIdx.x;
    const bool nz = (l < nrow) && (b[l] != 0.0);
    const unsigned mask = __ballot_sync(0xffffffffu, nz);
    __shared__ int warp_cnt[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_cnt[w] = __popc(mask);
    __syncthreads();
    int off = base;
    for (int q = 0; q < w; q++) off += warp_cnt[q];
    if (nz) nzidx[(size_t)k * nrow + off + __popc(mask & ((1u << lane) - 1))] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int q = 0; q < (int)(blockDim.x >> 5); q++) tot += warp_cnt[q];
      base += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) nzcnt[k] = base;
}

__global__ void k_f64_to_f32(const double *__restrict__ s, float *__restrict__ d, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    d[q] = (float)s[q];
}
__global__ void k_f32_to_f64(const float *__restrict__ s, double *__restrict__ d, int64_t n) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x)
    d[q] = (double)s[q];
}

// Batched: item blockIdx.y, column blockIdx.x (nonzero compaction) ...
__global__ void k_nonzeros_batch(const ProjItem *__restrict__ items) {
  const ProjItem it = items[blockIdx.y];
  const int k = blockIdx.x;
  if (k >= it.r) return;
  const double *b = it.B + (size_t)k * it.nrow;
  int32_t *nzidx = it.nz, *nzcnt = it.nz + (size_t)it.nrow * it.r;
  __shared__ int base;
  __shared__ int warp_cnt[32];
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int l0 = 0; l0 < it.nrow; l0 += blockDim.x) {
    const int l = l0 + threadIdx.x;
    const bool nzv = (l < it.nrow) && (b[l] != 0.0);
    const unsigned mask = __ballot_sync(0xffffffffu, nzv);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_cnt[w] = __popc(mask);
    __syncthreads();
    int off = base;
    for (int q = 0; q < w; q++) off += warp_cnt[q];
    if (nzv) nzidx[(size_t)k * it.nrow + off + __popc(mask & ((1u << lane) - 1))] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int q = 0; q < (int)(blockDim.x >> 5); q++) tot += warp_cnt[q];
      base += tot;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) nzcnt[k] = base;
}

// ... and the ordered projection, one thread per column of X (as k_project).
template <typename TQ>
__global__ void k_project_batch(const ProjItem *__restrict__ items) {
  const ProjItem it = items[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= it.ncol) return;
  const TQ *x = (const TQ *)it.X + (size_t)i * it.nrow;
  const int32_t *nzcnt = it.nz + (size_t)it.nrow * it.r;
  for (int k = 0; k < it.r; k++) {
    const double *b = it.B + (size_t)k * it.nrow;
    const int32_t *idx = it.nz + (size_t)k * it.nrow;
    double acc = 0.0;
    const int cnt = nzcnt[k];
    for (int q = 0; q < cnt; q++) {
      const int l = idx[q];
      acc = __dadd_rn(acc, __dmul_rn((double)x[l], b[l]));
    }
    it.U[(size_t)k * it.ncol + i] = acc;
  }
}

// Stage column k of U, V into each item's band buffer (u(1..m), v(1..n)).
__global__ void k_stage_batch(const ChaseArgs *__restrict__ items, const double *const *__restrict__ ucol,
                              const double *const *__restrict__ vcol) {
  const ChaseArgs a = items[blockIdx.x];
  const double *uc = ucol[blockIdx.x], *vc = vcol[blockIdx.x];
  for (int i = threadIdx.x; i < a.m; i += blockDim.x) a.band.u[i + 1] = uc[i];
  for (int j = threadIdx.x; j < a.n; j += blockDim.x) a.band.v[j + 1] = vc[j];
  for (int t = threadIdx.x; t < a.st.T; t += blockDim.x) { a.st.Ln[t] = 0; a.st.Rn[t] = 0; }
}

}  // namespace

cudaError_t launch_project_batch(int precision, const ProjItem *d_items, int count, int max_nrow,
                                 int max_ncol, int max_r, cudaStream_t s) {
  if (count <= 0 || max_r <= 0) return cudaSuccess;
  k_nonzeros_batch<<<dim3(max_r, count), 256, 0, s>>>(d_items);
  const dim3 g((max_ncol + 127) / 128, count);
  if (precision == BDU_FP64) k_project_batch<double><<<g, 128, 0, s>>>(d_items);
  else k_project_batch<float><<<g, 128, 0, s>>>(d_items);
  (void)max_nrow;
  return cudaGetLastError();
}

cudaError_t launch_stage_batch(const ChaseArgs *d_items, const double *const *d_ucol,
                               const double *const *d_vcol, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_stage_batch<<<count, 256, 0, s>>>(d_items, d_ucol, d_vcol);
  return cudaGetLastError();
}

// nz workspace: nrow * r int32 indices followed by r counts, provided by the
// caller through U's companion buffer (see bdu_api.cu).
cudaError_t launch_project_nz(int precision, const void *X, int64_t ld, int nrow, int ncol,
                              const double *B, int64_t ldb, int r, double *U, int64_t ldu,
                              int32_t *nz_ws, cudaStream_t s) {
  if (r <= 0) return cudaSuccess;
  int32_t *nzidx = nz_ws, *nzcnt = nz_ws + (size_t)nrow * r;
  k_nonzeros<<<r, 256, 0, s>>>(B, ldb, nrow, r, nzidx, nzcnt);
  const int th = 128, bl = (ncol + th - 1) / th;
  if (precision == BDU_FP64)
    k_project<double><<<bl, th, 0, s>>>((const double *)X, ld, nrow, ncol, nzidx, nzcnt, B, ldb, r, U, ldu);
  else
    k_project<float><<<bl, th, 0, s>>>((const float *)X, ld, nrow, ncol, nzidx, nzcnt, B, ldb, r, U, ldu);
  return cudaGetLastError();
}

cudaError_t launch_convert_f64_to_f32(const double *src, float *dst, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_f64_to_f32<<<1216, 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}
cudaError_t launch_convert_f32_to_f64(const float *src, double *dst, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_f32_to_f64<<<1216, 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

}  // namespace bdu
