// bdu_update_rank1_noalloc: one FP64 rank-1 update of a factorization that the
// caller keeps in its own device memory, without any device allocation.
//
// Who needs it: callers that cannot allocate device memory -- a host framework
// that reserves the whole GPU for its own allocator and forbids foreign
// cudaMalloc calls, a latency-critical loop in which an allocation (which may
// synchronize the device) is not acceptable, or an embedding in which the
// library may not own memory at all.  Such a caller passes its inputs and
// outputs as device pointers; every intermediate (the working band, the
// projections, the rotation records, the status word) lives in one
// file-scope __device__ array below, of a fixed size.
//
// The array is shared by every call on a device and keeps the previous call's
// contents; each call clears what must start at zero.  Calls that overlap on
// the GPU (issued from several host threads or on several streams without
// ordering) race on the array.  Every GPU that loads the library holds the
// array until the process exits.
#include <cstdio>
#include <mutex>

#include "bdu_internal.cuh"

namespace bdu {
cudaError_t launch_project_nz(int precision, const void *X, int64_t ld, int nrow, int ncol,
                              const double *B, int64_t ldb, int r, double *U, int64_t ldu,
                              int32_t *nz_ws, cudaStream_t s);
}

using namespace bdu;

namespace {

constexpr int64_t kMaxM = 1024;  // largest m accepted
constexpr int64_t kMaxN = 256;   // largest n accepted

constexpr int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

// Byte layout of the scratch for an m x n problem.
struct Layout {
  int64_t band, nz_b, nz_c, Lc, Ls, Rc, Rs, La, Ra, Ln, Rn, Sc, Ss, Sa, Sn, status, counters, total;
};

constexpr Layout layout(int64_t m, int64_t n) {
  const int64_t N = (m > n) ? n + 1 : n;
  const int64_t p2 = n > 2 ? n - 2 : 0;
  const int64_t ilast = (N == n + 1) ? n : n - 1;
  const int64_t T = (N - 1) + p2 + 2 * ilast;
  const int64_t cap = n / 2 + 4;
  const int64_t tc = T * cap;
  const int64_t band = 6 * (N + 2) + 2 * (n + 2) + (m + 2);
  Layout L{};
  int64_t o = 0;
  L.band = o; o = align256(o + 8 * band);
  L.nz_b = o; o = align256(o + 4 * (m + 1));
  L.nz_c = o; o = align256(o + 4 * (n + 1));
  L.Lc = o; o = align256(o + 8 * tc);
  L.Ls = o; o = align256(o + 8 * tc);
  L.Rc = o; o = align256(o + 8 * tc);
  L.Rs = o; o = align256(o + 8 * tc);
  L.La = o; o = align256(o + 4 * tc);
  L.Ra = o; o = align256(o + 4 * tc);
  L.Ln = o; o = align256(o + 4 * (T + 1));
  L.Rn = o; o = align256(o + 4 * (T + 1));
  L.Sc = o; o = align256(o + 8 * (m + 1));
  L.Ss = o; o = align256(o + 8 * (m + 1));
  L.Sa = o; o = align256(o + 4 * (m + 1));
  L.Sn = o; o = align256(o + 16);
  L.status = o; o = align256(o + 16);
  L.counters = o; o = align256(o + 8 * 16);
  L.total = o;
  return L;
}

// The scratch: sized for the largest accepted problem (about 5.5 MB).
constexpr int64_t kScratchBytes = layout(kMaxM, kMaxN).total;
static_assert(kScratchBytes < 8 * 1024 * 1024, "scratch must stay modest");
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch, looked up once per device (with that device
// current).  In host code the symbol itself is only a host-side stand-in.
constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

void *scratch_address(int dev, cudaError_t *err) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_addr[dev]) return g_scratch_addr[dev];
  void *p = nullptr;
  *err = cudaGetSymbolAddress(&p, g_scratch);
  if (*err != cudaSuccess) return nullptr;
  g_scratch_addr[dev] = p;
  return p;
}

// The band buffer layout of BandPtrs (6 diagonals of length N+2, r1, v, u),
// evaluated on the device.
__device__ int64_t dev_band_doubles(int64_t m, int64_t n) {
  const int64_t N = (m > n) ? n + 1 : n;
  return 6 * (N + 2) + 2 * (n + 2) + (m + 2);
}
__device__ BandPtrs dev_band_ptrs(double *base, int64_t m, int64_t n) {
  const int64_t N = (m > n) ? n + 1 : n;
  BandPtrs b;
  for (int o = 0; o < 6; o++) b.dg[o] = base + o * (N + 2);
  b.r1 = base + 6 * (N + 2);
  b.v = b.r1 + (n + 2);
  b.u = b.v + (n + 2);
  return b;
}

// Band layout of the working core (see BandPtrs) from the caller's d, e.
__global__ void k_band_from_de(const double *__restrict__ d, const double *__restrict__ e,
                               double *__restrict__ band, int m, int n) {
  const int64_t total = dev_band_doubles(m, n);
  BandPtrs b = dev_band_ptrs(band, m, n);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x)
    band[q] = 0.0;
  __syncthreads();  // single block: zero before placing d, e
  for (int i = threadIdx.x + 1; i <= n; i += blockDim.x) {
    if (i == 1) b.r1[1] = d[0];
    else b.dg[2][i] = d[i - 1];
    if (i < n) {
      if (i == 1) b.r1[2] = e[0];
      else b.dg[3][i] = e[i - 1];
    }
  }
}

// Leaves d, e untouched when the status word reports a failure of the chase.
__global__ void k_de_from_band(const double *__restrict__ band, double *__restrict__ d,
                               double *__restrict__ e, int m, int n, const int *__restrict__ status) {
  if (*(volatile const int *)status) return;
  BandPtrs b = dev_band_ptrs(const_cast<double *>(band), m, n);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x + 1; i <= n; i += gridDim.x * blockDim.x) {
    d[i - 1] = (i == 1) ? b.r1[1] : b.dg[2][i];
    if (i < n) e[i - 1] = (i == 1) ? b.r1[2] : b.dg[3][i];
  }
}

bdu_status set_err(bdu_status code, const char *) { return code; }

}  // namespace

extern "C" bdu_status bdu_update_rank1_noalloc(int64_t m, int64_t n, double *Q, double *d, double *e,
                                               double *P, const double *b, const double *c,
                                               void *stream) {
  if (n < 1 || m < n) return set_err(BDU_EINVAL, "bdu_update_rank1_noalloc: need m >= n >= 1");
  if (m > kMaxM || n > kMaxN)
    return set_err(BDU_EINVAL, "bdu_update_rank1_noalloc: m or n exceeds the maximum (m <= 1024, n <= 256)");
  if (!Q || !d || !P || !b || !c || (n > 1 && !e))
    return set_err(BDU_EINVAL, "bdu_update_rank1_noalloc: NULL pointer");
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_err(BDU_ECUDA, "bdu_update_rank1_noalloc: no current CUDA device");
  unsigned char *base = (unsigned char *)scratch_address(dev, &ce);
  if (!base) return set_err(BDU_ECUDA, "bdu_update_rank1_noalloc: cudaGetSymbolAddress failed");

  const Layout L = layout(m, n);
  cudaStream_t s = (cudaStream_t)stream;
  double *band = (double *)(base + L.band);
  BandPtrs bp = band_ptrs(band, m, n);
  RotStream st{};  // FP32 copies stay null: this entry point is FP64 only
  st.T = num_tasks(m, n);
  st.cap = task_cap(n);
  st.Lc = (double *)(base + L.Lc); st.Ls = (double *)(base + L.Ls);
  st.Rc = (double *)(base + L.Rc); st.Rs = (double *)(base + L.Rs);
  st.La = (int32_t *)(base + L.La); st.Ra = (int32_t *)(base + L.Ra);
  st.Ln = (int32_t *)(base + L.Ln); st.Rn = (int32_t *)(base + L.Rn);
  st.Sc = (double *)(base + L.Sc); st.Ss = (double *)(base + L.Ss);
  st.Sa = (int32_t *)(base + L.Sa); st.Sn = (int32_t *)(base + L.Sn);
  int *status = (int *)(base + L.status);
  unsigned long long *counters = (unsigned long long *)(base + L.counters);

  // what must start at zero: status, counters, per-task record counts, spike count
  ce = cudaMemsetAsync(status, 0, 16, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(counters, 0, 8 * 16, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(st.Ln, 0, 4 * (st.T + 1), s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(st.Rn, 0, 4 * (st.T + 1), s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(st.Sn, 0, 16, s);
  if (ce != cudaSuccess) return set_err(BDU_ECUDA, cudaGetErrorString(ce));
  k_band_from_de<<<1, 256, 0, s>>>(d, e, band, (int)m, (int)n);
  ce = cudaGetLastError();
  // u = Q^T b and v = P^T c, written straight into the band's u, v (1-based)
  if (ce == cudaSuccess)
    ce = launch_project_nz(BDU_FP64, Q, m, (int)m, (int)m, b, m, 1, bp.u + 1, m,
                           (int32_t *)(base + L.nz_b), s);
  if (ce == cudaSuccess)
    ce = launch_project_nz(BDU_FP64, P, n, (int)n, (int)n, c, n, 1, bp.v + 1, n,
                           (int32_t *)(base + L.nz_c), s);
  if (ce == cudaSuccess) {
    ChaseArgs a{};  // exact arithmetic, engine chosen by size
    a.m = (int)m; a.n = (int)n; a.band = bp;
    a.Ux = nullptr; a.Vx = nullptr; a.rx = 0;
    a.st = st; a.status = status; a.counters = counters;
    ce = launch_chase(a, s);
  }
  // a failure of the chase (status word nonzero) leaves Q, P, d and e untouched
  if (ce == cudaSuccess) ce = launch_apply(BDU_FP64, Q, m, (int)m, (int)m, st, 0, m > n, s, status, 0, false, 0, status);
  if (ce == cudaSuccess) ce = launch_apply(BDU_FP64, P, n, (int)n, (int)n, st, 1, false, s, status, 0, false, 0, status);
  if (ce == cudaSuccess) {
    k_de_from_band<<<1, 256, 0, s>>>(band, d, e, (int)m, (int)n, status);
    ce = cudaGetLastError();
  }
  int hst = 0;
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return set_err(BDU_ECUDA, cudaGetErrorString(ce));
  if (hst & ERR_STEPS) return set_err(BDU_ETIMEOUT, "bdu_update_rank1_noalloc: chase engine step budget exceeded");
  if (hst) return set_err(BDU_EINTERNAL, "bdu_update_rank1_noalloc: device invariant check failed");
  return BDU_OK;
}
