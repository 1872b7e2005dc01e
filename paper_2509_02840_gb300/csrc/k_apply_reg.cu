// K3, mixed form: register-resident application of the rotation stream of one
// rank-1 column to the FP32 columns of Q (left rotations) or P (right
// rotations) (Sec. 3.2, Eq. bidiagplus).
//
// Rows are independent under column rotations.  Each compute thread owns W
// consecutive columns (c0 = W * thread) of V consecutive rows and keeps that
// V x W block in registers through all the chases of the column: every
// element is read from and written to global memory once, and a rotation
// costs four FP32 operations per row.  A persistent grid walks over the row
// groups.
//
// Records.  The rotations of one chase act on disjoint column pairs (a, a+1)
// whose first columns a increase by a fixed step, 2 in phase 1 and 3 in
// phases 2 and 3, unless a rotation was skipped because the entry it would
// eliminate was already zero.  A producer warp streams each chase's FP32
// coefficients into a ring of shared-memory slots with one bulk copy per
// chase (full/empty mbarriers per slot), so the compute warps run ahead of
// one another by up to the ring depth and never wait on global loads.
//
// Geometry.  W is a multiple of 6, so where a gap-free chase's pairs fall in a
// block depends only on a mod step: five compiled variants cover every such
// chase, and a thread finds its records by index arithmetic.  In two of the
// variants one pair straddles each edge of every block; both owners compute
// their half of it from exchanged values: shuffles inside a warp; across two
// warps, shared memory with a per-layer flag (no block-wide barrier).  A chase
// with a gap takes a general path that binary-searches its records.  A warp
// whose columns the chase does not reach skips it.
//
// Every wait is bounded; one that runs out sets ERR_APPLY in the status word
// (the result is then reported as invalid): the producer issues no further
// copies and waits for those in flight, a compute warp stops.  Failure
// injection (bdu_set_fault_injection) can keep the producer from issuing any
// copy and shorten the bound, so that a test drives these waits to expiry
// with nothing in flight.
//
// Arithmetic: the generator's FP32 copies of (c, s), x' = fma(c, x, s*y),
// y' = fma(c, y, -s*x) -- the operations of the shared-memory slab kernel, so
// both kernels give identical results.  The spike chain (m > n) is sequential
// and runs before, one thread per row.
#include <climits>

#include "async_copy.cuh"
#include "bdu_internal.cuh"

namespace bdu {
namespace {

using async::bulk_g2s;
using async::mbar_arrive;
using async::mbar_arrive_tx;
using async::mbar_init;
using async::mbar_wait;

constexpr int kMaxThreads = 384;  // compute warps + the producer warp
constexpr int kMaxCompute = 352;  // compute threads
constexpr size_t kSmemBudget = 200 * 1024;

__device__ __forceinline__ void rot32(float c, float s, float &x, float &y) {
  const float xo = x, yo = y;
  x = fmaf(c, xo, s * yo);
  y = fmaf(c, yo, -s * xo);
}

constexpr int kEmptyCode = 7;

// ---------------------------------------------------------------------------
// per-chase descriptors
// ---------------------------------------------------------------------------
// x = e0, the record index of the pair starting at column phi (< 0 allowed):
//     a thread's first pair inside its block is record e0 + c0 / step;
// y = count | code << 24, code = 0..4 for a gap-free progression with
//     (step, first column mod step) = (2,0), (2,1), (3,0), (3,1), (3,2),
//     5 for a chase with a gap, 7 for an empty one;
// z, w = first columns of the chase's first and last pairs.
__global__ void k_chase_descriptors(const int32_t *__restrict__ Ca, const int32_t *__restrict__ Cn, int T,
                                    int cap, int p1, int4 *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const int cnt = min(max(Cn[t], 0), cap);
  if (cnt == 0) {
    out[t] = make_int4(0, kEmptyCode << 24, INT_MAX, INT_MIN);
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

// ---------------------------------------------------------------------------
// the spike chain
// ---------------------------------------------------------------------------
// Rotations on (a, a+1) with a descending; column a+1 of one rotation is
// column a of the previous one, kept in a register.  Column a has not been
// touched by earlier rotations of the chain, so its loads are issued ahead,
// eight records at a time.
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

// ---------------------------------------------------------------------------
// the register-resident kernel
// ---------------------------------------------------------------------------
// Shared memory of one block, R ring slots:
//   slot s: the 16-byte chase descriptor, then the chase's records (float2),
//           the first at index (t * cap) & 1 (copies start on 16-byte units);
//   full[R], empty[R]: mbarriers;
//   edges: per slot and compute warp, its column 0 (side 0) and column W-1
//          (side 1) for the neighbouring warps, V floats each, and a flag per
//          side naming the layer they belong to.
struct Layout {
  int R, rshift, nwc;  // R = 1 << rshift
  size_t slot_bytes, full, empty, edge, flag, total;
  void make(int cap, int V, int nwc_) {
    nwc = nwc_;
    slot_bytes = 16 + (size_t)((cap + 3) / 2) * 16;  // up to cap + 2 records
    R = 0;
    for (int r = 8; r >= 2; r >>= 1) {
      const size_t edge_b = (size_t)r * nwc * 2 * V * 4, flag_b = (size_t)r * nwc * 2 * 4;
      const size_t tot = r * slot_bytes + 2 * r * 8 + edge_b + flag_b;
      if (tot <= kSmemBudget) {
        R = r;
        rshift = r == 8 ? 3 : (r == 4 ? 2 : 1);
        full = r * slot_bytes;
        empty = full + 8 * r;
        edge = empty + 8 * r;
        flag = edge + edge_b;
        total = flag + flag_b;
        break;
      }
    }
  }
};

// Values of the neighbouring columns before this chase: yr = column c0+W,
// xl = column c0-1.  Across warps through shared memory and flags: a warp
// publishes its edges before it waits for its neighbours', so no wait cycle
// can form.
// Returns false (for the whole warp) when a wait ran out.
template <int W, int V>
__device__ __forceinline__ bool exchange(const float (&x)[V][W], float (&xl)[V], float (&yr)[V], float *edge,
                                         volatile int *flag, int slot, int q, int lane, int warp, int nwc,
                                         bool lact, bool ract, int spin, int *status) {
  bool ok = true;
#pragma unroll
  for (int r = 0; r < V; r++) {
    yr[r] = __shfl_down_sync(0xffffffffu, x[r][0], 1);
    xl[r] = __shfl_up_sync(0xffffffffu, x[r][W - 1], 1);
  }
  const int base = slot * nwc + warp;  // this warp's entries in the slot
  if (lane == 0 && lact) {
#pragma unroll
    for (int r = 0; r < V; r++) edge[(base * 2 + 0) * V + r] = x[r][0];
    __threadfence_block();
    flag[base * 2 + 0] = q;
  }
  if (lane == 31 && ract) {
#pragma unroll
    for (int r = 0; r < V; r++) edge[(base * 2 + 1) * V + r] = x[r][W - 1];
    __threadfence_block();
    flag[base * 2 + 1] = q;
  }
  if (lane == 31 && ract) {
    const int nb = base + 1;  // the right neighbour's column 0
    int i = 0;
    while (flag[nb * 2 + 0] != q && i < spin) i++;
    if (i == spin) { atomicOr(status, ERR_APPLY); ok = false; }
    __threadfence_block();
#pragma unroll
    for (int r = 0; r < V; r++) yr[r] = edge[(nb * 2 + 0) * V + r];
  }
  if (lane == 0 && lact) {
    const int nb = base - 1;  // the left neighbour's column W-1
    int i = 0;
    while (flag[nb * 2 + 1] != q && i < spin) i++;
    if (i == spin) { atomicOr(status, ERR_APPLY); ok = false; }
    __threadfence_block();
#pragma unroll
    for (int r = 0; r < V; r++) xl[r] = edge[(nb * 2 + 1) * V + r];
  }
  return !__any_sync(0xffffffffu, !ok);
}

// The halves of the straddling pairs a thread keeps: (c0+W-1, c0+W) gives the
// new column W-1, (c0-1, c0) the new column 0.
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

// A gap-free chase of step S with pairs starting at columns = PHI (mod S):
// K pairs inside each block (records ef .. ef+K-1) and, with X, one pair
// across each edge (records ef-1 and ef+K).
template <int W, int V, int S, int PHI>
__device__ __forceinline__ void apply_prog(float (&x)[V][W], const float2 *rec, int ef, int cnt,
                                           const float (&xl)[V], const float (&yr)[V]) {
  constexpr int K = (W - 2 - PHI) / S + 1;
  constexpr bool X = ((W - 1) % S) == PHI;
#pragma unroll
  for (int k = 0; k < K; k++) {
    if ((unsigned)(ef + k) < (unsigned)cnt) {
      const float2 g = rec[ef + k];
#pragma unroll
      for (int r = 0; r < V; r++) rot32(g.x, g.y, x[r][PHI + S * k], x[r][PHI + S * k + 1]);
    }
  }
  if (X) {
    if ((unsigned)(ef + K) < (unsigned)cnt) right_half<W, V>(x, rec[ef + K], yr);
    if ((unsigned)(ef - 1) < (unsigned)cnt) left_half<W, V>(x, rec[ef - 1], xl);
  }
}

// A chase with a gap: the thread's records are found by binary search over
// the pair positions (recorded in increasing order).
template <int W, int V>
__device__ __forceinline__ void apply_general(float (&x)[V][W], const float2 *rec,
                                              const int32_t *__restrict__ Ca, size_t base, int cnt, int c0,
                                              const float (&xl)[V], const float (&yr)[V]) {
  int lo = 0, hi = cnt;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (Ca[base + mid] - 1 < c0 - 1) lo = mid + 1;
    else hi = mid;
  }
  for (int e = lo; e < cnt; e++) {
    const int p = Ca[base + e] - 1 - c0;
    if (p > W - 1) break;
    const float2 g = rec[e];
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
                const int32_t *__restrict__ Ca, const int4 *__restrict__ desc, int T, int cap, Layout L,
                int spin, int stall, int *__restrict__ status) {
  extern __shared__ __align__(128) unsigned char raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwc = L.nwc, R = L.R, rs = L.rshift, rmask = L.R - 1;
  uint64_t *full = reinterpret_cast<uint64_t *>(raw + L.full);
  uint64_t *empty = reinterpret_cast<uint64_t *>(raw + L.empty);
  float *edge = reinterpret_cast<float *>(raw + L.edge);
  volatile int *flag = reinterpret_cast<volatile int *>(raw + L.flag);
  const int groups = (nrow + V - 1) / V;
  const int my_groups = (int)blockIdx.x < groups ? (groups - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int layers = my_groups * T;  // chases this block goes through

  if (tid == 0) {
    for (int s = 0; s < R; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], nwc);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  for (int i = tid; i < R * nwc * 2; i += blockDim.x) flag[i] = -1;
  __syncthreads();

  if (warp == nwc) {
    // ---- producer warp: one bulk copy per chase into the ring; the
    // descriptors come 32 at a time, one per lane.  After a wait that ran out
    // it issues nothing more.  With stall set (failure injection) it issues
    // nothing at all, so that the compute warps' waits run out while no copy
    // is in flight.
    if (stall) return;
    const int4 none = make_int4(0, kEmptyCode << 24, INT_MAX, INT_MIN);
    int4 dcur = none;
    int issued = 0;
    for (int q = 0, u = 0; q < layers; q++, u = (u + 1 == T) ? 0 : u + 1) {
      if ((u & 31) == 0) dcur = (u + lane < T) ? desc[u + lane] : none;
      int4 d;
      d.x = __shfl_sync(0xffffffffu, dcur.x, u & 31);
      d.y = __shfl_sync(0xffffffffu, dcur.y, u & 31);
      d.z = __shfl_sync(0xffffffffu, dcur.z, u & 31);
      d.w = __shfl_sync(0xffffffffu, dcur.w, u & 31);
      bool ok = true;
      if (lane == 0) {
        const int s = q & rmask;
        if (q >= R && !mbar_wait(&empty[s], (unsigned)(((q >> rs) - 1) & 1), spin)) {
          atomicOr(status, ERR_APPLY);
          ok = false;
        } else {
          unsigned char *slot = raw + (size_t)s * L.slot_bytes;
          *reinterpret_cast<int4 *>(slot) = d;
          const int cnt = d.y & 0xffffff;
          const size_t first = (size_t)u * cap;  // the chase's first record
          const size_t start = first & ~(size_t)1;
          const unsigned bytes = cnt > 0 ? (unsigned)(((first - start + cnt + 1) / 2) * 16) : 0u;
          mbar_arrive_tx(&full[s], bytes);
          if (bytes) bulk_g2s(slot + 16, coef + start, bytes, &full[s]);
        }
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      issued = q + 1;
    }
    // the last copies issued have landed before the block may exit
    if (lane == 0)
      for (int q = issued > R ? issued - R : 0; q < issued; q++)
        if (!mbar_wait(&full[q & rmask], (unsigned)((q >> rs) & 1), spin)) atomicOr(status, ERR_APPLY);
    return;
  }

  // ---- compute warps
  const int c0 = tid * W;
  // the warp has work in a chase whose pairs start at columns z..w iff
  // z <= (warp + 1) * span - 1 and w >= warp * span - 1 (pairs across its
  // edges included)
  const int span = 32 * W;
  const int wlo = warp * span - 1, whi = (warp + 1) * span - 1;  // this warp's reach
  int q = 0;
  for (int grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    const int r0 = grp * V;
    float x[V][W];
#pragma unroll
    for (int k = 0; k < W; k++) {
      const int col = c0 + k;
#pragma unroll
      for (int r = 0; r < V; r++) x[r][k] = (col < ncol && r0 + r < nrow) ? X[(size_t)col * ld + r0 + r] : 0.f;
    }
    for (int t = 0; t < T; t++, q++) {
      const int s = q & rmask;
      // after a wait that ran out the warp stops (the result is reported invalid)
      if (__any_sync(0xffffffffu, !mbar_wait(&full[s], (unsigned)((q >> rs) & 1), spin))) {
        if (lane == 0) atomicOr(status, ERR_APPLY);
        return;
      }
      const unsigned char *slot = raw + (size_t)s * L.slot_bytes;
      const int4 d = *reinterpret_cast<const int4 *>(slot);
      const int cnt = d.y & 0xffffff, code = d.y >> 24;
      if (code != kEmptyCode && d.z <= whi && d.w >= wlo) {
        const float2 *rec = reinterpret_cast<const float2 *>(slot + 16) + (t & cap & 1);
        float xl[V], yr[V];
        if (code == 1 || code == 4 || code == 5) {
          // given this warp's part, the left (right) neighbour has one iff the
          // chase starts (ends) within its reach
          const bool lact = warp > 0 && d.z <= wlo;
          const bool ract = warp + 1 < nwc && d.w >= whi;
          if (!exchange<W, V>(x, xl, yr, edge, flag, s, q, lane, warp, nwc, lact, ract, spin, status)) return;
        }
        switch (code) {
          case 0: apply_prog<W, V, 2, 0>(x, rec, d.x + tid * (W / 2), cnt, xl, yr); break;
          case 1: apply_prog<W, V, 2, 1>(x, rec, d.x + tid * (W / 2), cnt, xl, yr); break;
          case 2: apply_prog<W, V, 3, 0>(x, rec, d.x + tid * (W / 3), cnt, xl, yr); break;
          case 3: apply_prog<W, V, 3, 1>(x, rec, d.x + tid * (W / 3), cnt, xl, yr); break;
          case 4: apply_prog<W, V, 3, 2>(x, rec, d.x + tid * (W / 3), cnt, xl, yr); break;
          default: apply_general<W, V>(x, rec, Ca, (size_t)t * cap, cnt, c0, xl, yr); break;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
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
  int nth = 0, grid = 0;
  Layout L{};
  // Geometry for an nrow x ncol matrix with record slots of cap; false when
  // it is not covered.
  bool plan(int nrow, int ncol, int cap, int sm_reserve) {
    const int nwc = ((ncol + W - 1) / W + 31) / 32;
    if (nwc * 32 > kMaxCompute) return false;
    nth = nwc * 32 + 32;
    L.make(cap, V, nwc);
    if (L.R == 0) return false;
    if (cudaFuncSetAttribute(k_apply_reg<W, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total) !=
        cudaSuccess)
      return false;
    int dev = 0, sms = 1, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply_reg<W, V>, nth, L.total) != cudaSuccess ||
        per_sm < 1)
      return false;
    const int usable = sms - sm_reserve > 0 ? sms - sm_reserve : 1;
    const int groups = (nrow + V - 1) / V;
    grid = groups < per_sm * usable ? groups : per_sm * usable;
    return true;
  }
  void launch(float *X, int64_t ld, int nrow, int ncol, const float2 *coef, const int32_t *Ca, const int4 *desc,
              int T, int cap, int *status, cudaStream_t s) const {
    const Injection inj = injection();
    const int stall = inj.site == BDU_INJECT_APPLY_STALL ? 1 : 0;
    const int spin = stall ? (int)(inj.value < async::kSpin ? inj.value : async::kSpin) : async::kSpin;
    k_apply_reg<W, V><<<grid, nth, L.total, s>>>(X, ld, nrow, ncol, coef, Ca, desc, T, cap, L, spin, stall, status);
  }
};

}  // namespace

// The spike chain (m > n) of st applied to the FP32 rows of X, one thread per row.
cudaError_t launch_apply_spike32(float *X, int64_t ld, int nrow, const RotStream &st, cudaStream_t s) {
  if (!st.Sf) return cudaErrorInvalidValue;
  k_apply_spike32<<<(nrow + 127) / 128, 128, 0, s>>>(X, ld, nrow, st.Sf, st.Sa, st.Sn);
  return cudaGetLastError();
}

// Per-chase descriptors of one side of st (see k_chase_descriptors).
cudaError_t launch_chase_descriptors(const RotStream &st, int side, cudaStream_t s) {
  int4 *desc = side == 0 ? st.Lm : st.Rm;
  if (!desc || st.T <= 0) return cudaSuccess;
  k_chase_descriptors<<<(st.T + 255) / 256, 256, 0, s>>>(side == 0 ? st.La : st.Ra, side == 0 ? st.Ln : st.Rn,
                                                           st.T, st.cap, st.p1, desc);
  return cudaGetLastError();
}

// Register-resident FP32 apply; cudaErrorNotSupported, before anything is
// launched, when the shape or the stream is not covered (the caller then uses
// the shared-memory slab kernel).  layout: 0 = the first of (W, V) = (12, 8),
// (24, 4) that covers the columns; 1 = (12, 8), 2 = (24, 4), 3 = (6, 16),
// 4 = (18, 4) (columns per thread W, rows per thread V; all give identical
// results).  Records are copied in 16-byte units up to one entry past the last
// chase's slot, so Lf and Rf hold T*cap + 2 entries.
cudaError_t launch_apply_reg(float *X, int64_t ld, int nrow, int ncol, const RotStream &st, int side,
                             bool with_spike, int *status, int sm_reserve, bool desc_ready, int layout,
                             cudaStream_t s) {
  const float2 *coef = side == 0 ? st.Lf : st.Rf;
  int4 *desc = side == 0 ? st.Lm : st.Rm;
  if (!coef || !desc || !status || layout < 0 || layout > 4) return cudaErrorNotSupported;
  RegLaunch<12, 8> l1;
  RegLaunch<24, 4> l2;
  RegLaunch<6, 16> l3;
  RegLaunch<18, 4> l4;
  int use = 0;
  if (layout == 0) {
    use = l1.plan(nrow, ncol, st.cap, sm_reserve) ? 1 : (l2.plan(nrow, ncol, st.cap, sm_reserve) ? 2 : 0);
  } else {
    const bool ok = layout == 1   ? l1.plan(nrow, ncol, st.cap, sm_reserve)
                    : layout == 2 ? l2.plan(nrow, ncol, st.cap, sm_reserve)
                    : layout == 3 ? l3.plan(nrow, ncol, st.cap, sm_reserve)
                                  : l4.plan(nrow, ncol, st.cap, sm_reserve);
    use = ok ? layout : 0;
  }
  if (use == 0) {
    cudaGetLastError();
    return cudaErrorNotSupported;
  }
  const int32_t *Ca = side == 0 ? st.La : st.Ra;
  const int32_t *Cn = side == 0 ? st.Ln : st.Rn;
  if (st.T > 0 && !desc_ready)
    k_chase_descriptors<<<(st.T + 255) / 256, 256, 0, s>>>(Ca, Cn, st.T, st.cap, st.p1, desc);
  if (with_spike) k_apply_spike32<<<(nrow + 127) / 128, 128, 0, s>>>(X, ld, nrow, st.Sf, st.Sa, st.Sn);
  if (st.T > 0) {
    if (use == 1) l1.launch(X, ld, nrow, ncol, coef, Ca, desc, st.T, st.cap, status, s);
    else if (use == 2) l2.launch(X, ld, nrow, ncol, coef, Ca, desc, st.T, st.cap, status, s);
    else if (use == 3) l3.launch(X, ld, nrow, ncol, coef, Ca, desc, st.T, st.cap, status, s);
    else l4.launch(X, ld, nrow, ncol, coef, Ca, desc, st.T, st.cap, status, s);
  }
  return cudaGetLastError();
}

}  // namespace bdu
