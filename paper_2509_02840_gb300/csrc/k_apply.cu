// K3: application of the rotation stream to the columns of Q (left
// rotations, Q+ = Q * prod G^T) or P (right rotations, P+ = P * prod H)
// (Sec. 3.2, Eq. bidiagplus).
//
// Rows of Q and P are independent under column rotations, so each CTA owns a
// slab of rows, keeps it in shared memory for the whole rank-1 column and
// writes it back once: every element is read and written once per column.
// The rotations of one chase act on disjoint column pairs, so a chase is
// applied by all threads at once; consecutive chases are separated by a
// barrier.  The spike chain (m > n) is sequential and runs first, one thread
// per row.
//
// FP64: each pair update is c*x + s*y with separately rounded operations, the
// same operations a one-rotation-at-a-time evaluation performs.  FP32 (the
// mixed form): rotations are rounded to FP32 and applied with fused
// multiply-adds.
#include "bdu_internal.cuh"

namespace bdu {
namespace {

template <typename T> struct Arith;
template <> struct Arith<double> {
  static __device__ __forceinline__ void rot(double c, double s, double &x, double &y) {
    const double xo = x, yo = y;
    x = __dadd_rn(__dmul_rn(c, xo), __dmul_rn(s, yo));
    y = __dadd_rn(__dmul_rn(-s, xo), __dmul_rn(c, yo));
  }
};
template <> struct Arith<float> {
  static __device__ __forceinline__ void rot(float c, float s, float &x, float &y) {
    const float xo = x, yo = y;
    x = fmaf(c, xo, s * yo);
    y = fmaf(c, yo, -s * xo);
  }
};

template <typename T>
__global__ void __launch_bounds__(512) k_apply_slab(
    T *__restrict__ X, int64_t ld, int nrow, int ncol, int R,
    const double *__restrict__ Sc, const double *__restrict__ Ss, const int32_t *__restrict__ Sa,
    const int32_t *__restrict__ Sn,
    const double *__restrict__ Cc, const double *__restrict__ Cs, const int32_t *__restrict__ Ca,
    const int32_t *__restrict__ Cn, int ntask, int cap) {
  extern __shared__ unsigned char raw[];
  T *tile = reinterpret_cast<T *>(raw);
  const int ldt = ncol + 1;  // padded row length in shared memory
  const int r0 = blockIdx.x * R;
  const int rows = min(R, nrow - r0);
  if (rows <= 0) return;
  const int tid = threadIdx.x, nth = blockDim.x;

  for (int64_t q = tid; q < (int64_t)rows * ncol; q += nth) {
    const int col = (int)(q / rows), rr = (int)(q % rows);
    tile[rr * ldt + col] = X[(size_t)col * ld + r0 + rr];
  }
  __syncthreads();

  if (Sn != nullptr) {
    const int ns = Sn[0];
    if (tid < rows) {
      T *row = tile + tid * ldt - 1;  // 1-based column index
      for (int e = 0; e < ns; e++) {
        const int a = Sa[e];
        Arith<T>::rot((T)Sc[e], (T)Ss[e], row[a], row[a + 1]);
      }
    }
    __syncthreads();
  }

  for (int t = 0; t < ntask; t++) {
    const int cnt = Cn[t];
    const size_t base = (size_t)t * cap;
    for (int q = tid; q < cnt * rows; q += nth) {
      const int e = q / rows, rr = q - e * rows;
      const int a = Ca[base + e];
      T *row = tile + rr * ldt - 1;
      Arith<T>::rot((T)Cc[base + e], (T)Cs[base + e], row[a], row[a + 1]);
    }
    __syncthreads();
  }

  for (int64_t q = tid; q < (int64_t)rows * ncol; q += nth) {
    const int col = (int)(q / rows), rr = (int)(q % rows);
    X[(size_t)col * ld + r0 + rr] = tile[rr * ldt + col];
  }
}

}  // namespace

cudaError_t launch_apply(int precision, void *X, int64_t ld, int nrow, int ncol,
                         const RotStream &st, int side, bool with_spike, cudaStream_t s) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t esz = (precision == BDU_FP64) ? sizeof(double) : sizeof(float);
  const size_t row_bytes = esz * (size_t)(ncol + 1);
  int R = (int)((size_t)optin / row_bytes);
  if (R > 32) R = 32;
  if (R < 1) return cudaErrorInvalidValue;  // a single row does not fit
  const size_t smem = row_bytes * R;
  const int blocks = (nrow + R - 1) / R;
  const double *Cc = side == 0 ? st.Lc : st.Rc;
  const double *Cs = side == 0 ? st.Ls : st.Rs;
  const int32_t *Ca = side == 0 ? st.La : st.Ra;
  const int32_t *Cn = side == 0 ? st.Ln : st.Rn;
  const int32_t *Sn = with_spike ? st.Sn : nullptr;
  cudaError_t e;
  if (precision == BDU_FP64) {
    e = cudaFuncSetAttribute(k_apply_slab<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_apply_slab<double><<<blocks, 512, smem, s>>>((double *)X, ld, nrow, ncol, R, st.Sc, st.Ss, st.Sa,
                                                   Sn, Cc, Cs, Ca, Cn, st.T, st.cap);
  } else {
    e = cudaFuncSetAttribute(k_apply_slab<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_apply_slab<float><<<blocks, 512, smem, s>>>((float *)X, ld, nrow, ncol, R, st.Sc, st.Ss, st.Sa,
                                                  Sn, Cc, Cs, Ca, Cn, st.T, st.cap);
  }
  return cudaGetLastError();
}

}  // namespace bdu
