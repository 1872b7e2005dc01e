// K3: application of the rotation stream to the columns of Q (left
// rotations, Q+ = Q * prod G^T) or P (right rotations, P+ = P * prod H)
// (Sec. 3.2, Eq. bidiagplus).
//
// Rows of Q and P are independent under column rotations, so each CTA owns a
// slab of R rows, keeps it in shared memory for the whole rank-1 column and
// writes it back once: every element is read and written once per column.
// The slab is stored column by column, so that a rotation reaches 4 (FP32) or
// 2 (FP64) rows of both of its columns with each 16-byte shared access.
// The rotations of one chase act on disjoint column pairs, so a chase is
// applied by all threads at once -- one rotation per thread, looping over the
// slab's rows -- and consecutive chases are separated by a barrier; the next
// chase's rotations are prefetched into registers while the current one is
// applied.  The spike chain (m > n) is sequential and runs first, one thread
// per row.  R is chosen so that the grid fills whole waves of SMs.
//
// FP64: each pair update is c*x + s*y with separately rounded operations, the
// same operations a one-rotation-at-a-time evaluation performs.  FP32 (the
// mixed form): the generator's FP32 copies of (c, s) are applied with fused
// multiply-adds.
#include "bdu_internal.cuh"

namespace bdu {
namespace {

constexpr int kThreads = 512;
constexpr int kPer = 5;  // rotations per thread per chase held in registers

template <typename T> struct Coef;
template <> struct Coef<double> {
  double c, s;
  static __device__ __forceinline__ Coef load(const RotStream &st, int side, size_t i) {
    Coef k;
    k.c = side == 0 ? st.Lc[i] : st.Rc[i];
    k.s = side == 0 ? st.Ls[i] : st.Rs[i];
    return k;
  }
  static __device__ __forceinline__ Coef load_spike(const RotStream &st, int i) {
    Coef k; k.c = st.Sc[i]; k.s = st.Ss[i]; return k;
  }
  __device__ __forceinline__ void rot(double &x, double &y) const {
    const double xo = x, yo = y;
    x = __dadd_rn(__dmul_rn(c, xo), __dmul_rn(s, yo));
    y = __dadd_rn(__dmul_rn(-s, xo), __dmul_rn(c, yo));
  }
};
template <> struct Coef<float> {
  float c, s;
  static __device__ __forceinline__ Coef load(const RotStream &st, int side, size_t i) {
    const float2 v = side == 0 ? st.Lf[i] : st.Rf[i];
    Coef k; k.c = v.x; k.s = v.y; return k;
  }
  static __device__ __forceinline__ Coef load_spike(const RotStream &st, int i) {
    const float2 v = st.Sf[i];
    Coef k; k.c = v.x; k.s = v.y; return k;
  }
  __device__ __forceinline__ void rot(float &x, float &y) const {
    const float xo = x, yo = y;
    x = fmaf(c, xo, s * yo);
    y = fmaf(c, yo, -s * xo);
  }
};

// 16-byte vectors of the tile: 4 floats or 2 doubles
template <typename T> struct Vec;
template <> struct Vec<float> {
  using type = float4;
  static constexpr int V = 4;
  static __device__ __forceinline__ void rot(const Coef<float> &k, float4 &x, float4 &y) {
    k.rot(x.x, y.x); k.rot(x.y, y.y); k.rot(x.z, y.z); k.rot(x.w, y.w);
  }
};
template <> struct Vec<double> {
  using type = double2;
  static constexpr int V = 2;
  static __device__ __forceinline__ void rot(const Coef<double> &k, double2 &x, double2 &y) {
    k.rot(x.x, y.x); k.rot(x.y, y.y);
  }
};

// Shared-memory tile: column-major, column c's R rows at tile[c*csw ...],
// csw = V * (odd count of 16-byte vectors) >= R, so that the columns touched
// by a stride-3 chase fall in distinct 16-byte bank groups.
template <typename T>
__device__ __forceinline__ void apply_slab_body(T *__restrict__ X, int64_t ld, int nrow, int ncol, int R,
                                                int csw, const RotStream &st, int side, int with_spike,
                                                int slab) {
  using VT = typename Vec<T>::type;
  constexpr int V = Vec<T>::V;
  extern __shared__ __align__(16) unsigned char raw[];
  T *tile = reinterpret_cast<T *>(raw);
  const int r0 = slab * R;
  const int rows = min(R, nrow - r0);
  if (rows <= 0) return;
  const int tid = threadIdx.x;
  const int32_t *Ca = side == 0 ? st.La : st.Ra;
  const int32_t *Cn = side == 0 ? st.Ln : st.Rn;
  const int cap = st.cap, ntask = st.T;
  const int nv = R / V;  // vectors per column

  for (int64_t q = tid; q < (int64_t)R * ncol; q += kThreads) {
    const int col = (int)(q / R), rr = (int)(q % R);
    tile[(size_t)col * csw + rr] = (rr < rows) ? X[(size_t)col * ld + r0 + rr] : T(0);
  }
  __syncthreads();

  if (with_spike) {
    const int ns = st.Sn[0];
    if (tid < rows) {
      T *row = tile + tid;
      for (int e = 0; e < ns; e++) {
        const int a = st.Sa[e] - 1;  // 0-based first column of the pair
        Coef<T>::load_spike(st, e).rot(row[(size_t)a * csw], row[(size_t)(a + 1) * csw]);
      }
    }
    __syncthreads();
  }

  // the rotations of the current chase owned by this thread, in registers
  Coef<T> cf[kPer];
  int ca[kPer];
  int cnt = ntask > 0 ? Cn[0] : 0;
#pragma unroll
  for (int k = 0; k < kPer; k++) {
    const int e = tid + k * kThreads;
    ca[k] = -1;
    if (e < cnt) {
      cf[k] = Coef<T>::load(st, side, (size_t)e);
      ca[k] = Ca[e] - 1;
    }
  }
  for (int t = 0; t < ntask; t++) {
    // prefetch chase t+1
    Coef<T> nf[kPer];
    int na[kPer];
    const int ncnt = (t + 1 < ntask) ? Cn[t + 1] : 0;
    const size_t nbase = (size_t)(t + 1) * cap;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
      const int e = tid + k * kThreads;
      na[k] = -1;
      if (e < ncnt) {
        nf[k] = Coef<T>::load(st, side, nbase + e);
        na[k] = Ca[nbase + e] - 1;
      }
    }
    // apply chase t: each owned rotation to all rows of the slab, V rows per access
#pragma unroll
    for (int k = 0; k < kPer; k++) {
      if (ca[k] >= 0) {
        VT *pa = reinterpret_cast<VT *>(tile + (size_t)ca[k] * csw);
        VT *pb = reinterpret_cast<VT *>(tile + (size_t)(ca[k] + 1) * csw);
        for (int q = 0; q < nv; q++) {
          VT x = pa[q], y = pb[q];
          Vec<T>::rot(cf[k], x, y);
          pa[q] = x;
          pb[q] = y;
        }
      }
    }
    // chases longer than the register-held part
    const int ccnt = Cn[t];
    for (int e = tid + kPer * kThreads; e < ccnt; e += kThreads) {
      const size_t i = (size_t)t * cap + e;
      const Coef<T> k = Coef<T>::load(st, side, i);
      VT *pa = reinterpret_cast<VT *>(tile + (size_t)(Ca[i] - 1) * csw);
      VT *pb = reinterpret_cast<VT *>(tile + (size_t)Ca[i] * csw);
      for (int q = 0; q < nv; q++) {
        VT x = pa[q], y = pb[q];
        Vec<T>::rot(k, x, y);
        pa[q] = x;
        pb[q] = y;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPer; k++) {
      cf[k] = nf[k];
      ca[k] = na[k];
    }
  }

  for (int64_t q = tid; q < (int64_t)rows * ncol; q += kThreads) {
    const int col = (int)(q / rows), rr = (int)(q % rows);
    X[(size_t)col * ld + r0 + rr] = tile[(size_t)col * csw + rr];
  }
}

// gate (may be null): a device error word written by an earlier kernel on
// the stream; when it is nonzero the kernel leaves X untouched.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_apply_slab(T *__restrict__ X, int64_t ld, int nrow,
                                                         int ncol, int R, int csw, RotStream st,
                                                         int side, int with_spike, const int *gate) {
  if (gate && *(volatile const int *)gate) return;
  apply_slab_body<T>(X, ld, nrow, ncol, R, csw, st, side, with_spike, blockIdx.x);
}

// Many matrices of uneven sizes in one launch: block b works on the slab
// b - first[i] of item i, where first[] is the prefix sum of the items' slab
// counts (found by binary search).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_apply_batch(const ApplyItem *__restrict__ items,
                                                          const int *__restrict__ first, int count) {
  const int b = blockIdx.x;
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  const ApplyItem it = items[lo];
  apply_slab_body<T>((T *)it.X, it.ld, it.nrow, it.ncol, it.R, it.csw, it.st, it.side, it.with_spike,
                     b - first[lo]);
}

}  // namespace

// Rows per slab and column stride for an ncol-wide matrix within smem_cap
// bytes of shared memory, as many rows as fit (at most 64).
void apply_geometry(int precision, int ncol, size_t smem_cap, int *R, int *csw) {
  const int esz = (precision == BDU_FP64) ? 8 : 4;
  const int V = 16 / esz;
  int bestR = 0, bestc = 0;
  for (int r = V; r <= 64; r += V) {
    int w = r / V;
    if ((w & 1) == 0) w++;
    const int c = w * V;
    if ((size_t)esz * c * ncol > smem_cap) break;
    bestR = r; bestc = c;
  }
  *R = bestR; *csw = bestc;
}

cudaError_t launch_apply_batch(int precision, const ApplyItem *d_items, const int *d_first, int count,
                               int total_slabs, size_t smem, cudaStream_t s) {
  if (count <= 0 || total_slabs <= 0) return cudaSuccess;
  cudaError_t e;
  if (precision == BDU_FP64) {
    e = cudaFuncSetAttribute(k_apply_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_apply_batch<double><<<total_slabs, kThreads, smem, s>>>(d_items, d_first, count);
  } else {
    e = cudaFuncSetAttribute(k_apply_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_apply_batch<float><<<total_slabs, kThreads, smem, s>>>(d_items, d_first, count);
  }
  return cudaGetLastError();
}

cudaError_t launch_apply(int precision, void *X, int64_t ld, int nrow, int ncol,
                         const RotStream &st, int side, bool with_spike, cudaStream_t s, int *status,
                         int sm_reserve, bool desc_ready, int variant, const int *gate) {
  if (precision == BDU_MIXED && (st.Lf == nullptr || st.Rf == nullptr)) return cudaErrorInvalidValue;
  if (precision == BDU_MIXED && variant == 0 && ncol >= kBlockedFrom && st.tc_ws) variant = 128;
  if (precision == BDU_MIXED && is_tc_variant(variant))
    return launch_apply_tc((float *)X, ld, nrow, ncol, st, side, with_spike, status, desc_ready, variant, st.tc_ws,
                           st.tc_ws_bytes, s);
  if (precision == BDU_MIXED && variant != kSlabVariant) {
    cudaError_t e = launch_apply_reg((float *)X, ld, nrow, ncol, st, side, with_spike, status, sm_reserve,
                                     desc_ready, variant, s);
    if (e != cudaErrorNotSupported || variant != 0) return e;
    // no register layout covers the shape: the blocked tensor-core apply
    e = launch_apply_tc((float *)X, ld, nrow, ncol, st, side, with_spike, status, desc_ready, 128, st.tc_ws,
                        st.tc_ws_bytes, s);
    if (e != cudaErrorNotSupported) return e;
    cudaGetLastError();
  }
  int dev = 0, optin = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int esz = (precision == BDU_FP64) ? 8 : 4;
  const int V = 16 / esz;
  // rows per CTA: a multiple of V; the column stride is an odd number of
  // 16-byte vectors.  Pick the R that minimizes waves x (R + overhead).
  // (FP64 form: a positive variant fixes R instead)
  int best_R = 0, best_csw = 0;
  double best_cost = 1e300;
  const bool fixed = precision == BDU_FP64 && variant > 0;
  if (fixed && (variant % V != 0 || variant > 64)) return cudaErrorNotSupported;
  for (int R = V; R <= 64; R += V) {
    int w = R / V;
    if ((w & 1) == 0) w++;
    const int csw = w * V;
    const size_t smem = (size_t)esz * csw * ncol;
    if (smem > (size_t)optin) break;
    const int ctas = (nrow + R - 1) / R;
    const int waves = (ctas + sms - 1) / sms;
    const double cost = fixed ? (R == variant ? 0.0 : 1e299) : (double)waves * (R + 4);
    if (cost <= best_cost) { best_cost = cost; best_R = R; best_csw = csw; }
  }
  if (fixed && best_R != variant) return cudaErrorNotSupported;
  if (best_R == 0) return cudaErrorNotSupported;  // a single vector column does not fit
  const size_t smem = (size_t)esz * best_csw * ncol;
  const int blocks = (nrow + best_R - 1) / best_R;
  cudaError_t e;
  if (precision == BDU_FP64) {
    e = cudaFuncSetAttribute(k_apply_slab<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_apply_slab<double><<<blocks, kThreads, smem, s>>>((double *)X, ld, nrow, ncol, best_R, best_csw, st,
                                                        side, with_spike ? 1 : 0, gate);
  } else {
    e = cudaFuncSetAttribute(k_apply_slab<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_apply_slab<float><<<blocks, kThreads, smem, s>>>((float *)X, ld, nrow, ncol, best_R, best_csw, st,
                                                       side, with_spike ? 1 : 0, gate);
  }
  return cudaGetLastError();
}

}  // namespace bdu
