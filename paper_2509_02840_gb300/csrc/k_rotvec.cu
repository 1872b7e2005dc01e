// Rotation of projected vectors by a finished rotation stream, for the
// overlapped mixed form.
//
// After rank-1 column j-1 has generated its rotations G (left) and H (right),
// Q_j = Q_{j-1} G and P_j = P_{j-1} H (Sec. 3.2, Eq. bidiagplus), so the
// projections of the next column satisfy u_j = Q_j^T b = G^T (Q_{j-1}^T b) and
// v_j = H^T (P_{j-1}^T c).  They can therefore be formed from the factors as
// they were before column j-1 was applied, and then rotated here: a rotation
// of columns (a, a+1) of Q acts on entries (a, a+1) of Q^T b exactly as on the
// two entries of one row of Q.  This lets the application of column j-1 to Q
// and P run concurrently with the chase of column j.
//
// One block per vector; the vector sits in shared memory.  The spike chain
// (left side, m > n) is sequential: its records are staged in shared memory a
// chunk at a time and one thread runs through them.  The chases' rotations
// then come as the FP32 coefficients the apply uses and the per-chase
// descriptors: a producer warp cuts each chase into chunks of up to kRecs
// records and streams them into a ring of shared-memory slots with bulk copies
// (full/empty mbarriers, bounded waits), so that many copies are in flight at
// once; the compute threads apply a chunk's rotations, which act on disjoint
// pairs, all at once (kPerThread each), and meet at a barrier only where a
// chase ends.  A chunk holds a whole chase of up to kRecs records, so the
// barriers, not the data, set the pace: about one per chase.  A pair's
// first column comes from the chase's progression (first + step * index), or
// from the recorded positions for a chase with a gap.
//
// Arithmetic: FP32 with fused multiply-adds, the operations the mixed form
// applies to the rows of Q and P with the same coefficients -- so u = G^T w
// carries the rounding that Q_j^T b carries when Q_j is rotated in FP32.  (In
// FP64 the rotations would be bound by one SM's FP64 rate: about 4 x 12.5M
// operations per side at n = 4096, some 12 ms.)
#include "async_copy.cuh"
#include "bdu_internal.cuh"

namespace bdu {
namespace {

constexpr int kCompute = 512;            // compute threads
constexpr int kThreads = kCompute + 32;  // + the producer warp
constexpr int kRecs = 2048;              // records per chunk (a chase holds at most n/2 + 4)
constexpr int kPerThread = kRecs / kCompute;
constexpr int kSpike = 512;              // spike records staged at a time
constexpr size_t kSmemBudget = 220 * 1024;
constexpr size_t kSlot = 16 + (kRecs + 2) * 8;  // header + coefficients (from a 16-byte boundary)

__device__ __forceinline__ void rot32(float c, float s, float &x, float &y) {
  const float xo = x, yo = y;
  x = fmaf(c, xo, s * yo);
  y = fmaf(c, yo, -s * xo);
}

__host__ __device__ inline size_t round16(size_t b) { return (b + 15) / 16 * 16; }
constexpr size_t kStaging = 16 * ((kSpike * 4 + 15) / 16) + kSpike * 8;

// Shared memory: the vector, full[R] and empty[R], then R chunk slots (the
// spike's staging area before they are used).
struct RvLayout {
  int R, rmask, rshift;
  size_t vec, full, empty, ring, total;
  bool make(int len) {
    vec = round16((size_t)len * 4);
    R = 0;
    for (int r = 32, sh = 5; r >= 4; r >>= 1, sh--) {
      const size_t ring_b = (size_t)r * kSlot > kStaging ? (size_t)r * kSlot : kStaging;
      const size_t tot = vec + 16 * r + ring_b;
      if (tot <= kSmemBudget) {
        R = r; rmask = r - 1; rshift = sh;
        full = vec;
        empty = full + 8 * r;
        ring = empty + 8 * r;
        total = tot;
        return true;
      }
    }
    return false;
  }
};

// Chunk header: x = index within its chase of the chunk's first record;
// y = count | last << 12 | gap << 13 | shift << 14 | stop << 15;
// z = first column of the chase's first pair; w = step, or for a chase with a
// gap the index of its first record in the record arrays.
constexpr int kCountMask = (1 << 12) - 1, kLast = 1 << 12, kGap = 1 << 13, kShift = 1 << 14, kStop = 1 << 15;
static_assert(kRecs <= kCountMask && kRecs % kCompute == 0, "chunk layout");

// Blocks 0 .. nl-1: vector b of w_left (m entries, stride ldl) by the left
// stream into the same place of dst_left; blocks nl .. nl+nr-1: vector b-nl of
// w_right (n entries, stride ldr) by the right stream into dst_right.  A
// vector is read whole into shared memory before it is written, so w and dst
// may coincide.
__global__ void __launch_bounds__(kThreads) k_rotate_vectors(const double *w_left, double *dst_left, int64_t ldl,
                                                             int nl, int m, const double *w_right, double *dst_right,
                                                             int64_t ldr, int n,
                                                             RotStream st, int with_spike, RvLayout L,
                                                             int spin, int stall, int *__restrict__ status) {
  extern __shared__ __align__(128) unsigned char raw[];
  const bool left = (int)blockIdx.x < nl;
  const int vec = left ? (int)blockIdx.x : (int)blockIdx.x - nl;
  const int len = left ? m : n;
  const int tid = threadIdx.x;
  const double *w = left ? w_left + (size_t)vec * ldl : w_right + (size_t)vec * ldr;
  double *dst = left ? dst_left + (size_t)vec * ldl : dst_right + (size_t)vec * ldr;
  float *v = reinterpret_cast<float *>(raw);
  uint64_t *full = reinterpret_cast<uint64_t *>(raw + L.full);
  uint64_t *empty = reinterpret_cast<uint64_t *>(raw + L.empty);
  for (int i = tid; i < len; i += blockDim.x) v[i] = (float)w[i];
  if (tid == 0) {
    for (int q = 0; q < L.R; q++) {
      async::mbar_init(&full[q], 1);
      async::mbar_init(&empty[q], kCompute / 32);
    }
    async::mbar_init_fence();
  }
  __syncthreads();
  if (left && with_spike) {
    // staged in the ring, before the producer starts
    int *sa = reinterpret_cast<int *>(raw + L.ring);
    float2 *sg = reinterpret_cast<float2 *>(raw + L.ring + round16((size_t)kSpike * 4));
    const int ns = st.Sn[0];
    for (int e0 = 0; e0 < ns; e0 += kSpike) {
      const int k = min(kSpike, ns - e0);
      for (int i = tid; i < k; i += blockDim.x) {
        sa[i] = st.Sa[e0 + i] - 1;
        sg[i] = st.Sf[e0 + i];
      }
      __syncthreads();
      if (tid == 0)
        for (int i = 0; i < k; i++) {
          if (sa[i] < 0 || sa[i] + 1 >= len) { atomicOr(status, ERR_RANGE); continue; }
          rot32(sg[i].x, sg[i].y, v[sa[i]], v[sa[i] + 1]);
        }
      __syncthreads();
    }
  }
  const int32_t *Ca = left ? st.La : st.Ra;
  const float2 *Cf = left ? st.Lf : st.Rf;
  const int4 *desc = left ? st.Lm : st.Rm;
  const int cap = st.cap, T = st.T;

  if (tid >= kCompute) {
    // ---- producer warp: descriptors 32 at a time, one bulk copy per chunk.
    // After a wait that ran out it issues nothing more; with stall set
    // (failure injection) nothing at all, so that the compute threads' waits
    // run out while no copy is in flight.
    if (stall) return;
    const int lane = tid - kCompute;
    int q = 0;  // chunks issued
    bool dead = false;
    for (int t0 = 0; t0 < T && !dead; t0 += 32) {
      const int4 mine = (t0 + lane < T) ? desc[t0 + lane] : make_int4(0, 7 << 24, 0, 0);
      for (int i = 0; i < 32 && t0 + i < T; i++) {
        const int dy = __shfl_sync(0xffffffffu, mine.y, i);
        const int dz = __shfl_sync(0xffffffffu, mine.z, i);
        const int cnt = dy & 0xffffff, code = dy >> 24;
        if (cnt == 0 || code == 7) continue;  // uniform across the warp
        const int t = t0 + i;
        const bool gap = code == 5;
        const int step = code < 2 ? 2 : 3;
        if (lane == 0) {
          for (int e0 = 0; e0 < cnt; e0 += kRecs, q++) {
            const int k = min(kRecs, cnt - e0);
            const int s = q & L.rmask;
            if (q >= L.R && !async::mbar_wait(&empty[s], (unsigned)(((q >> L.rshift) - 1) & 1), spin)) {
              atomicOr(status, ERR_ROTVEC);
              dead = true;
              break;
            }
            unsigned char *slot = raw + L.ring + (size_t)s * kSlot;
            const size_t first = (size_t)t * cap + e0;
            const int sh = (int)(first & 1);
            const unsigned bytes = (unsigned)(((sh + k + 1) / 2) * 16);
            const int flags = k | (e0 + k == cnt ? kLast : 0) | (gap ? kGap : 0) | (sh ? kShift : 0);
            *reinterpret_cast<int4 *>(slot) = make_int4(e0, flags, dz, gap ? t * cap : step);
            async::mbar_arrive_tx(&full[s], bytes);
            async::bulk_g2s(slot + 16, Cf + (first - sh), bytes, &full[s]);
          }
        }
        q = __shfl_sync(0xffffffffu, q, 0);
        dead = __shfl_sync(0xffffffffu, dead, 0);
        if (dead) break;
      }
    }
    if (lane == 0) {
      // the end marker (unless a wait ran out), then the last copies issued
      // have landed before the block may exit
      const int s = q & L.rmask;
      if (!dead && q >= L.R && !async::mbar_wait(&empty[s], (unsigned)(((q >> L.rshift) - 1) & 1), spin)) {
        atomicOr(status, ERR_ROTVEC);
        dead = true;
      }
      if (!dead) {
        *reinterpret_cast<int4 *>(raw + L.ring + (size_t)s * kSlot) = make_int4(0, kStop, 0, 0);
        async::mbar_arrive_tx(&full[s], 0u);
      }
      // (chunk q - R shared its slot with the end marker: it was consumed before)
      for (int p = q - L.R + 1 > 0 ? q - L.R + 1 : 0; p < q; p++)
        if (!async::mbar_wait(&full[p & L.rmask], (unsigned)((p >> L.rshift) & 1), spin))
          atomicOr(status, ERR_ROTVEC);
    }
    return;
  }

  // ---- compute threads
  for (int q = 0;; q++) {
    const int s = q & L.rmask;
    if (!async::mbar_wait(&full[s], (unsigned)((q >> L.rshift) & 1), spin)) {
      atomicOr(status, ERR_ROTVEC);
      break;
    }
    const unsigned char *slot = raw + L.ring + (size_t)s * kSlot;
    const int4 hd = *reinterpret_cast<const int4 *>(slot);
    if (hd.y & kStop) break;
    const int k = min(hd.y & kCountMask, kRecs);
    const float2 *cf = reinterpret_cast<const float2 *>(slot + 16) + ((hd.y & kShift) ? 1 : 0);
    // records tid, tid + kCompute, ... of the chunk: disjoint pairs of one
    // chase, so all are loaded before any is stored
    int a4[kPerThread];
    float2 g4[kPerThread];
    float x4[kPerThread], y4[kPerThread];
#pragma unroll
    for (int u = 0; u < kPerThread; u++) {
      const int j = tid + u * kCompute;
      a4[u] = -1;
      if (j < k) {
        const int ri = hd.x + j;  // index of the record within its chase
        const int a = (hd.y & kGap) ? Ca[(size_t)hd.w + ri] - 1 : hd.z + hd.w * ri;
        if (a >= 0 && a + 1 < len) {
          a4[u] = a;
          g4[u] = cf[j];
          x4[u] = v[a];
          y4[u] = v[a + 1];
        } else {
          atomicOr(status, ERR_RANGE);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kPerThread; u++)
      if (a4[u] >= 0) {
        rot32(g4[u].x, g4[u].y, x4[u], y4[u]);
        v[a4[u]] = x4[u];
        v[a4[u] + 1] = y4[u];
      }
    if (hd.y & kLast) async::named_sync(1, kCompute);  // the chase done by all: its values visible
    __syncwarp();
    if ((tid & 31) == 0) async::mbar_arrive(&empty[s]);
  }
  async::named_sync(1, kCompute);
  for (int i = tid; i < len; i += kCompute) dst[i] = (double)v[i];
}

}  // namespace

// Whether the vector rotation of an m x n factorization fits one block's
// shared memory.
bool rotate_vectors_supported(int m, int n) {
  RvLayout L{};
  return L.make(m > n ? m : n);
}

// dst_left = G^T w_left (m entries), dst_right = H^T w_right (n entries) for
// the rotation stream st, whose chase descriptors (Lm, Rm) are current;
// with_spike when the left stream starts with a spike chain (m > n).  The
// FP32 coefficients are read in 16-byte units, up to one entry past the last
// chase's slot (Lf, Rf hold T*cap + 2 entries).
cudaError_t launch_rotate_vectors(const double *w_left, double *dst_left, int m, const double *w_right,
                                  double *dst_right, int n, const RotStream &st, bool with_spike, int *status,
                                  cudaStream_t s) {
  return launch_rotate_vector_sets(w_left, dst_left, m, 1, m, w_right, dst_right, n, 1, n, st, with_spike, status, s);
}

// The same for count vectors on each side: column j of w_left (leading
// dimension ldl) into column j of dst_left, likewise on the right; one block
// per vector, all at once.
cudaError_t launch_rotate_vector_sets(const double *w_left, double *dst_left, int64_t ldl, int nl, int m,
                                      const double *w_right, double *dst_right, int64_t ldr, int nr, int n,
                                      const RotStream &st, bool with_spike, int *status, cudaStream_t s) {
  RvLayout L{};
  if (!st.Lf || !st.Rf || !st.Sf || !st.Lm || !st.Rm || !L.make(m > n ? m : n) || nl < 0 || nr < 0)
    return cudaErrorNotSupported;
  if (nl + nr == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_rotate_vectors, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
  if (e != cudaSuccess) return e;
  const Injection inj = injection();
  const int stall = inj.site == BDU_INJECT_ROTVEC_STALL ? 1 : 0;
  const int spin = stall ? (int)(inj.value < async::kSpin ? inj.value : async::kSpin) : async::kSpin;
  k_rotate_vectors<<<nl + nr, kThreads, L.total, s>>>(w_left, dst_left, ldl, nl, m, w_right, dst_right, ldr, n, st,
                                                     with_spike ? 1 : 0, L, spin, stall, status);
  return cudaGetLastError();
}

}  // namespace bdu
