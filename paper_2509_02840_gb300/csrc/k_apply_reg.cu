// K3, mixed form: register-resident application of the rotation stream of one
// rank-1 column to the FP32 columns of Q (left rotations) or P (right
// rotations) (Sec. 3.2, Eq. bidiagplus).
//
// Rows are independent under column rotations.  Each thread owns W = 12
// consecutive columns (c0 = W * thread) of V = 8 consecutive rows and keeps
// that V x W block in registers through all the chases of the column: every
// element is read from and written to global memory once, and a rotation costs
// four FP32 operations per row and no shared-memory traffic.  A persistent
// grid walks over the row groups.
//
// The rotations of one chase act on disjoint column pairs (a, a+1); their
// first columns a increase by a fixed step, 2 in phase 1 and 3 in phases 2
// and 3, unless a rotation was skipped because the entry it would eliminate
// was already zero.  Since W is a multiple of 6, where a gap-free chase's
// pairs fall inside a thread's block depends only on a mod step: five compiled
// variants cover every such chase, and a thread finds the records of its
// pairs by index arithmetic.  In two of the variants one pair straddles each
// edge of the block; both threads owning it compute their half from exchanged
// values (shuffles inside a warp, shared memory and one barrier across warps).
// A chase with a gap takes a general path that binary-searches its records.
// While chase t is applied, each thread copies the coefficients of its pairs
// in chase t+3 and the descriptor of chase t+6 into its own shared-memory
// rings with cp.async, so no load latency is exposed.
//
// Arithmetic: the generator's FP32 copies of (c, s), x' = fma(c, x, s*y),
// y' = fma(c, y, -s*x) -- the operations of the shared-memory slab kernel, so
// both kernels give identical results.  The spike chain (m > n) is sequential
// and runs before, one thread per row.
#include <climits>

#include "bdu_internal.cuh"

namespace bdu {
namespace {

constexpr int kMaxThreads = 384;  // threads per block: ceil(ncol / W) rounded to warps
constexpr int kDist = 3;          // chases between a coefficient copy and its use
constexpr int kDescRing = 8;      // descriptor ring slots (>= 2 kDist + 1, power of two)
constexpr int kCoefRing = 4;      // coefficient ring slots (>= kDist + 1, power of two)

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void rot32(float c, float s, float &x, float &y) {
  const float xo = x, yo = y;
  x = fmaf(c, xo, s * yo);
  y = fmaf(c, yo, -s * xo);
}

// Chase descriptor (one per chase, read by every thread):
//   x = e0, the record index of the pair starting at column phi (< 0 allowed):
//       a thread's first pair inside its block is record e0 + c0 / step;
//   y = count | code << 24, code = 0..4 for a gap-free progression with
//       (step, first column mod step) = (2,0), (2,1), (3,0), (3,1), (3,2),
//       5 for a chase with a gap, 7 for an empty one;
//   z, w = first columns of the chase's first and last pairs.
__global__ void k_chase_descriptors(const int32_t *__restrict__ Ca, const int32_t *__restrict__ Cn, int T,
                                    int cap, int p1, int4 *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const int cnt = min(max(Cn[t], 0), cap);
  if (cnt == 0) {
    out[t] = make_int4(0, 7 << 24, INT_MAX, INT_MIN);
    return;
  }
  const int step = t < p1 ? 2 : 3;
  const size_t b = (size_t)t * cap;
  const int first = Ca[b] - 1, last = Ca[b + cnt - 1] - 1;
  int code = 5, e0 = 0;
  if (last - first == (cnt - 1) * step) {
    const int phi = first % step;
    code = step == 2 ? phi : 2 + phi;
    e0 = (phi - first) / step;
  }
  out[t] = make_int4(e0, cnt | (code << 24), first, last);
}

// The spike chain: rotations on (a, a+1) with a descending; column a+1 of one
// rotation is column a of the previous one, kept in a register.  Column a has
// not been touched by earlier rotations of the chain, so its loads are issued
// ahead, eight records at a time.
__global__ void k_apply_spike32(float *__restrict__ X, int64_t ld, int nrow, const float2 *__restrict__ Sf,
                                const int32_t *__restrict__ Sa, const int32_t *__restrict__ Sn) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= nrow) return;
  const int ns = Sn[0];
  float *xr = X + row;
  int held = -1;
  float hv = 0.f;
  for (int e0 = 0; e0 < ns; e0 += 8) {
    int a[8];
    float2 g[8];
    float xa[8], xb[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
      a[q] = -2;
      if (e0 + q < ns) {
        a[q] = Sa[e0 + q] - 1;
        g[q] = Sf[e0 + q];
      }
    }
#pragma unroll
    for (int q = 0; q < 8; q++)
      if (a[q] >= 0) {
        xa[q] = xr[(size_t)a[q] * ld];
        xb[q] = xr[(size_t)(a[q] + 1) * ld];
      }
#pragma unroll
    for (int q = 0; q < 8; q++) {
      if (a[q] < 0) continue;
      float y;
      if (held == a[q] + 1) {
        y = hv;
      } else {
        if (held >= 0) xr[(size_t)held * ld] = hv;
        y = xb[q];
      }
      float x = xa[q];
      rot32(g[q].x, g[q].y, x, y);
      xr[(size_t)(a[q] + 1) * ld] = y;
      held = a[q];
      hv = x;
    }
  }
  if (held >= 0) xr[(size_t)held * ld] = hv;
}

// Exchange of the edge columns with the neighbouring threads: yr = column c0+W
// (the right neighbour's column 0), xl = column c0-1 (the left neighbour's
// column W-1), both as they were before this chase.
template <int W, int V>
__device__ __forceinline__ void exchange(const float (&x)[V][W], float (&xl)[V], float (&yr)[V], float *edge,
                                         int lane, int warp, int nwarps) {
#pragma unroll
  for (int r = 0; r < V; r++) {
    yr[r] = __shfl_down_sync(0xffffffffu, x[r][0], 1);
    xl[r] = __shfl_up_sync(0xffffffffu, x[r][W - 1], 1);
  }
  if (lane == 0)
#pragma unroll
    for (int r = 0; r < V; r++) edge[warp * V + r] = x[r][0];
  if (lane == 31)
#pragma unroll
    for (int r = 0; r < V; r++) edge[(nwarps + warp) * V + r] = x[r][W - 1];
  __syncthreads();
  if (lane == 31 && warp + 1 < nwarps)
#pragma unroll
    for (int r = 0; r < V; r++) yr[r] = edge[(warp + 1) * V + r];
  if (lane == 0 && warp > 0)
#pragma unroll
    for (int r = 0; r < V; r++) xl[r] = edge[(nwarps + warp - 1) * V + r];
}

// The halves of the straddling pairs this thread keeps: (c0+W-1, c0+W) gives
// the new column W-1, (c0-1, c0) the new column 0.
template <int W, int V>
__device__ __forceinline__ void right_half(float (&x)[V][W], float2 g, const float (&yr)[V]) {
#pragma unroll
  for (int r = 0; r < V; r++) x[r][W - 1] = fmaf(g.x, x[r][W - 1], g.y * yr[r]);
}
template <int W, int V>
__device__ __forceinline__ void left_half(float (&x)[V][W], float2 g, const float (&xl)[V]) {
#pragma unroll
  for (int r = 0; r < V; r++) x[r][0] = fmaf(g.x, x[r][0], -g.y * xl[r]);
}

// Where a gap-free chase of step S, pairs starting at columns = PHI (mod S),
// meets a block: K pairs inside, and with X one pair across each edge.  Ring
// slot k+1 holds the coefficients of the thread's k-th pair (record ef + k);
// k = -1 and k = K are the straddling pairs.
template <int W, int S, int PHI>
struct Geo {
  static constexpr int K = (W - 2 - PHI) / S + 1;
  static constexpr bool X = ((W - 1) % S) == PHI;
  static constexpr int kLo = X ? -1 : 0;
  static constexpr int kHi = X ? K : K - 1;
};

template <int W, int V, int S, int PHI>
__device__ __forceinline__ void apply_prog(float (&x)[V][W], const float2 *ring, int nth, int ef, int cnt,
                                           float *edge, int lane, int warp, int nwarps) {
  using G = Geo<W, S, PHI>;
  float xl[V], yr[V];
  if (G::X) exchange<W, V>(x, xl, yr, edge, lane, warp, nwarps);
#pragma unroll
  for (int k = 0; k < G::K; k++) {
    if ((unsigned)(ef + k) < (unsigned)cnt) {
      const float2 g = ring[(k + 1) * nth];
#pragma unroll
      for (int r = 0; r < V; r++) rot32(g.x, g.y, x[r][PHI + S * k], x[r][PHI + S * k + 1]);
    }
  }
  if (G::X) {
    if ((unsigned)(ef + G::K) < (unsigned)cnt) right_half<W, V>(x, ring[(G::K + 1) * nth], yr);
    if ((unsigned)(ef - 1) < (unsigned)cnt) left_half<W, V>(x, ring[0], xl);
  }
}

template <int W, int S, int PHI>
__device__ __forceinline__ void prefetch(float2 *dst, int nth, const float2 *src, int ef, int cnt) {
  using G = Geo<W, S, PHI>;
#pragma unroll
  for (int k = G::kLo; k <= G::kHi; k++) {
    const int e = ef + k;
    if ((unsigned)e < (unsigned)cnt) cp_async8(dst + (k + 1) * nth, src + e);
  }
}

// A chase with a gap: the thread's records are found by binary search (the
// pairs of a chase are recorded in increasing order).
template <int W, int V>
__device__ __forceinline__ void apply_general(float (&x)[V][W], const float2 *__restrict__ coef,
                                           const int32_t *__restrict__ Ca, size_t base, int cnt, int c0,
                                           float *edge, int lane, int warp, int nwarps) {
  float xl[V], yr[V];
  exchange<W, V>(x, xl, yr, edge, lane, warp, nwarps);
  int lo = 0, hi = cnt;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (Ca[base + mid] - 1 < c0 - 1) lo = mid + 1;
    else hi = mid;
  }
  for (int e = lo; e < cnt; e++) {
    const int p = Ca[base + e] - 1 - c0;
    if (p > W - 1) break;
    const float2 g = coef[base + e];
    if (p == -1) {
      left_half<W, V>(x, g, xl);
    } else if (p == W - 1) {
      right_half<W, V>(x, g, yr);
    } else {
#pragma unroll
      for (int q = 0; q < W - 1; q++)
        if (q == p)
#pragma unroll
          for (int r = 0; r < V; r++) rot32(g.x, g.y, x[r][q], x[r][q + 1]);
    }
  }
}

template <int W, int V>
__global__ void __launch_bounds__(kMaxThreads, 1)
    k_apply_reg(float *__restrict__ X, int64_t ld, int nrow, int ncol, const float2 *__restrict__ coef,
                const int32_t *__restrict__ Ca, const int4 *__restrict__ desc, int T, int cap) {
  constexpr int kSlots = W / 2 + 2;
  extern __shared__ __align__(16) unsigned char raw[];
  const int nth = blockDim.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
  int4 *dring = reinterpret_cast<int4 *>(raw) + tid;                                          // [kDescRing][nth]
  float2 *cring = reinterpret_cast<float2 *>(reinterpret_cast<int4 *>(raw) + kDescRing * nth) + tid;  // [kCoefRing][kSlots][nth]
  float *edge0 = reinterpret_cast<float *>(cring - tid + kCoefRing * kSlots * nth);          // [2][2 nwarps V]
  const int c0 = tid * W;
  // the warp has work in a chase whose pairs start at columns first..last iff
  // first <= wlast and last >= wfirst (pairs across the warp's edges included)
  const int wfirst = warp * 32 * W - 1, wlast = (warp + 1) * 32 * W - 1;
  const int groups = (nrow + V - 1) / V;
  int par = 0;  // edge buffer of the next exchange; alternates so that one barrier per exchange suffices

  for (int grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    const int r0 = grp * V;
    float x[V][W];
#pragma unroll
    for (int k = 0; k < W; k++) {
      const int col = c0 + k;
#pragma unroll
      for (int r = 0; r < V; r++) x[r][k] = (col < ncol && r0 + r < nrow) ? X[(size_t)col * ld + r0 + r] : 0.f;
    }
    for (int t = -2 * kDist; t < T; t++) {
      cp_wait<kDist - 1>();  // the group issued kDist chases ago has landed
      if (t >= 0) {
        const int4 d = dring[(t & (kDescRing - 1)) * nth];
        const int cnt = d.y & 0xffffff, code = d.y >> 24;
        if (code != 7) {
          const bool cross = code == 1 || code == 4 || code == 5;  // one barrier in this chase
          if (d.z <= wlast && d.w >= wfirst) {
            float *edge = edge0 + par * 2 * nwarps * V;
            const float2 *ring = cring + (size_t)(t & (kCoefRing - 1)) * kSlots * nth;
            switch (code) {
              case 0: apply_prog<W, V, 2, 0>(x, ring, nth, d.x + tid * (W / 2), cnt, edge, lane, warp, nwarps); break;
              case 1: apply_prog<W, V, 2, 1>(x, ring, nth, d.x + tid * (W / 2), cnt, edge, lane, warp, nwarps); break;
              case 2: apply_prog<W, V, 3, 0>(x, ring, nth, d.x + tid * (W / 3), cnt, edge, lane, warp, nwarps); break;
              case 3: apply_prog<W, V, 3, 1>(x, ring, nth, d.x + tid * (W / 3), cnt, edge, lane, warp, nwarps); break;
              case 4: apply_prog<W, V, 3, 2>(x, ring, nth, d.x + tid * (W / 3), cnt, edge, lane, warp, nwarps); break;
              default: apply_general<W, V>(x, coef, Ca, (size_t)t * cap, cnt, c0, edge, lane, warp, nwarps); break;
            }
          } else if (cross) {
            __syncthreads();  // the barrier of the exchange the other warps perform
          }
          if (cross) par ^= 1;
        }
      }
      // coefficients of chase t + kDist (its descriptor landed with the group awaited above)
      const int u = t + kDist;
      if (u >= 0 && u < T) {
        const int4 d = dring[(u & (kDescRing - 1)) * nth];
        const int cnt = d.y & 0xffffff, code = d.y >> 24;
        if (code < 5 && d.z <= wlast && d.w >= wfirst) {
          const float2 *src = coef + (size_t)u * cap;
          float2 *dst = cring + (size_t)(u & (kCoefRing - 1)) * kSlots * nth;
          switch (code) {
            case 0: prefetch<W, 2, 0>(dst, nth, src, d.x + tid * (W / 2), cnt); break;
            case 1: prefetch<W, 2, 1>(dst, nth, src, d.x + tid * (W / 2), cnt); break;
            case 2: prefetch<W, 3, 0>(dst, nth, src, d.x + tid * (W / 3), cnt); break;
            case 3: prefetch<W, 3, 1>(dst, nth, src, d.x + tid * (W / 3), cnt); break;
            default: prefetch<W, 3, 2>(dst, nth, src, d.x + tid * (W / 3), cnt); break;
          }
        }
      }
      const int v = t + 2 * kDist;
      if (v >= 0 && v < T) cp_async16(dring + (v & (kDescRing - 1)) * nth, desc + v);
      cp_commit();
    }
    cp_wait<0>();
#pragma unroll
    for (int k = 0; k < W; k++) {
      const int col = c0 + k;
#pragma unroll
      for (int r = 0; r < V; r++)
        if (col < ncol && r0 + r < nrow) X[(size_t)col * ld + r0 + r] = x[r][k];
    }
  }
}

template <int W, int V>
struct RegLaunch {
  static constexpr int kSlots = W / 2 + 2;
  int nth = 0, grid = 0;
  size_t smem = 0;
  // Geometry for an nrow x ncol matrix; false when it is not covered.
  bool plan(int nrow, int ncol) {
    nth = ((ncol + W - 1) / W + 31) / 32 * 32;
    if (nth > kMaxThreads) return false;
    smem = (size_t)kDescRing * nth * 16 + (size_t)kCoefRing * kSlots * nth * 8 + (size_t)2 * 2 * (nth / 32) * V * 4;
    if (cudaFuncSetAttribute(k_apply_reg<W, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return false;
    int dev = 0, sms = 1, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_reg<W, V>, nth, smem) != cudaSuccess ||
        per_sm < 1)
      return false;
    const int groups = (nrow + V - 1) / V;
    grid = groups < per_sm * sms ? groups : per_sm * sms;
    return true;
  }
  void launch(float *X, int64_t ld, int nrow, int ncol, const float2 *coef, const int32_t *Ca, const int4 *desc,
              int T, int cap, cudaStream_t s) const {
    k_apply_reg<W, V><<<grid, nth, smem, s>>>(X, ld, nrow, ncol, coef, Ca, desc, T, cap);
  }
};

}  // namespace

// Register-resident FP32 apply; cudaErrorNotSupported, before anything is
// launched, when the shape or the stream is not covered (the caller then uses
// the shared-memory slab kernel).
cudaError_t launch_apply_reg(float *X, int64_t ld, int nrow, int ncol, const RotStream &st, int side,
                             bool with_spike, cudaStream_t s) {
  const float2 *coef = side == 0 ? st.Lf : st.Rf;
  int4 *desc = side == 0 ? st.Lm : st.Rm;
  if (!coef || !desc) return cudaErrorNotSupported;
  RegLaunch<12, 8> narrow;
  RegLaunch<24, 4> wide;
  const bool use_narrow = narrow.plan(nrow, ncol);
  if (!use_narrow && !wide.plan(nrow, ncol)) {
    cudaGetLastError();
    return cudaErrorNotSupported;
  }
  const int32_t *Ca = side == 0 ? st.La : st.Ra;
  const int32_t *Cn = side == 0 ? st.Ln : st.Rn;
  if (st.T > 0) k_chase_descriptors<<<(st.T + 255) / 256, 256, 0, s>>>(Ca, Cn, st.T, st.cap, st.p1, desc);
  if (with_spike) k_apply_spike32<<<(nrow + 127) / 128, 128, 0, s>>>(X, ld, nrow, st.Sf, st.Sa, st.Sn);
  if (st.T > 0) {
    if (use_narrow) narrow.launch(X, ld, nrow, ncol, coef, Ca, desc, st.T, st.cap, s);
    else wide.launch(X, ld, nrow, ncol, coef, Ca, desc, st.T, st.cap, s);
  }
  return cudaGetLastError();
}

}  // namespace bdu
