// K4, mixed form: blocked application of the rotation stream of one rank-1
// column on the tensor cores (Sec. 3.2, Eq. bidiagplus: Q+ = Q Q1, P+ = P P1,
// with Q1, P1 the products of the left and right rotations).
//
// Tiling.  Chase t's rotations act on disjoint column pairs (a, a+1), and a
// rotation of chase t depends only on rotations of earlier chases that share
// a column with it (|a - a'| <= 1).  The chases are cut into bands of K
// consecutive chases; inside a band, the rotation of local chase i on the pair
// starting at column a belongs to tile j = floor((a + i + 1) / W): a window of
// W pair starts that moves one column to the left per chase (a
// parallelogram).  With that slope every rotation's predecessors lie in its
// own tile or in tiles to its left, and no rotation of tile j+1 precedes one
// of tile j, so applying the tiles left to right, each tile's rotations in
// chase order, gives the sequential result (the argument holds for a grid
// shifted by any o columns, tile j = floor((a + i + 1 + o) / W); the shift
// changes from band to band, below).  Tile j touches the NB = W + K
// columns [j W - K - o, j W + W - o); its rotations compose into an NB x NB
// orthogonal block G_j (formed by applying them, in order, to the identity),
// and the tile is applied as the product X(:, cols) <- X(:, cols) G_j.
// Consecutive tiles of a band overlap in K columns: the last K columns of one
// product are the first K inputs of the next, and the first W are final.
//
// Kernels, per band: k_tc_form builds the band's blocks (one thread block per
// tile, four threads per row of G, in shared memory) and writes each as the
// tensor cores' B operand, split into two TF32 parts; k_tc_apply then gives
// each panel of 128 rows of X to one thread block, which walks the band's
// tiles left to right: a row thread per TMEM lane holds its row's inputs
// [carry | W new columns], split into TF32 hi and lo parts, in tensor memory
// (the A operand), one thread issues tcgen05.mma (kind::tf32, M = 128,
// N = NB, accumulator in tensor memory) with B streamed into shared memory by
// bulk copies, and the row threads read the accumulator back (tcgen05.ld),
// store its first W columns and carry the last K into the next tile.
//
// Arithmetic: 3xTF32 with FP32 accumulation, D = A_hi B_hi + (A_hi B_lo +
// A_lo B_hi), where x_hi = x rounded to TF32 (nearest) and x_lo = x - x_hi,
// also rounded to TF32; the two terms accumulate separately in tensor memory
// (the accumulation truncates toward zero, so the large term sees only one
// truncation per 8-deep MMA) and are added in FP32; the blocks themselves are formed in FP32 with the
// generator's FP32 coefficients (x' = fma(c, x, s y), y' = fma(c, y, -s x)).
// Each output row is then scaled back to its input norm over the tile (G is
// orthogonal; the tensor cores' accumulation truncates toward zero, a bias
// that would otherwise add up over the bands).  Results agree with the
// rotation-by-rotation FP32 apply to FP32 rounding (not bit for bit).
//
// Every wait is bounded; one that runs out sets ERR_APPLY, the kernel stops
// issuing work, waits (bounded) for what it has in flight, frees its tensor
// memory and returns.
#include <climits>

#include "async_copy.cuh"
#include "bdu_internal.cuh"
#include "tcgen05.cuh"

namespace bdu {
namespace {

using namespace tc;

constexpr int kRows = 128;          // rows of a panel: the MMA's M and the TMEM lanes
constexpr uint32_t kTmemCols = 512;
// TMEM columns: the main accumulator (A_hi B_hi), A hi, A lo, the correction
// accumulator (A_hi B_lo + A_lo B_hi)
constexpr uint32_t kColD = 0, kColAH = 128, kColAL = 256, kColDC = 384;
constexpr int kEmpty = 7;           // descriptor code of a chase without rotations
constexpr unsigned kCopyChunk = 16384;

// first index e in [0, cnt) with v[e] >= key (v ascending)
__device__ __forceinline__ int lower_bound(const int32_t *__restrict__ v, int cnt, int key) {
  int lo = 0, hi = cnt;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The tile grid of band b is shifted by o_b columns (tile j covers
// [j W - K - o_b, j W + W - o_b)); the tiling argument holds for any shift.
// Shifting it from band to band moves each column of X through every
// position in a tile, so that the accumulation's residual error, which
// depends on the position, does not pile up on the same columns.
__host__ __device__ __forceinline__ int band_offset(int b, int W) { return (int)(((long long)b * 37) % W); }

// ---------------------------------------------------------------------------
// per-band tile ranges
// ---------------------------------------------------------------------------
// ranges[b] = (first, last) tile of band b, or (0, -1) when the band has no
// rotation.  desc: the per-chase descriptors (z, w = first columns of the
// chase's first and last pairs, 0-based).
// A band whose range would exceed max_tiles (only possible with corrupt
// descriptors) is reported (ERR_RANGE) and skipped.
__global__ void k_tc_band_ranges(const int4 *__restrict__ desc, int T, int K, int W, int nbands, int max_tiles,
                                 int2 *__restrict__ ranges, int *__restrict__ status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbands) return;
  const int o = band_offset(b, W);
  int lo = INT_MAX, hi = INT_MIN;
  for (int i = 0; i < K; i++) {
    const int t = b * K + i;
    if (t >= T) break;
    const int4 d = desc[t];
    if ((d.y >> 24) == kEmpty) continue;
    lo = min(lo, (d.z + i + 1 + o) / W);
    hi = max(hi, (d.w + i + 1 + o) / W);
  }
  if (lo <= hi && (lo < 0 || hi - lo + 1 > max_tiles)) {
    atomicOr(status, ERR_RANGE);
    lo = 0;
    hi = -1;
  }
  ranges[b] = lo <= hi ? make_int2(lo, hi) : make_int2(0, -1);
}

// ---------------------------------------------------------------------------
// the structure of a block
// ---------------------------------------------------------------------------
// In tile coordinates, local chase i may rotate pairs starting at columns
// [K - 1 - i, K - 2 - i + W]: a value moves at most one column per chase,
// and only inside that window, which slides one column to the left per
// chase.  So G(k, c) = 0 unless output column c is reachable from input
// column k, whatever the rotations are; the reachable range of each k is an
// interval, computed here by following its ends through the K chases.  The
// B operand keeps, for each 8-row k-step s of the MMA, only the output
// columns [n0[s], n1[s]) reachable from its rows (rounded out to 16, the
// MMA's N granularity): about 62% of the block at NB = 128.  Layout of one
// part (hi or lo) of a blob: step s at byte off[s], K-major without swizzle,
// its two 4-column K chunks one after the other, each (n1 - n0) / 8 core
// matrices of 8 rows x 16 bytes (leading-dimension offset (n1 - n0) / 8 *
// 128 bytes, stride-dimension offset 128).
template <int NB>
struct Cone {
  static constexpr int K = NB / 2, W = NB / 2, S = NB / 8;
  int n0[S], n1[S], off[S + 1];
  __host__ __device__ constexpr Cone() : n0(), n1(), off() {
    for (int s = 0; s < S; s++) {
      int lo = NB, hi = -1;
      for (int k = 8 * s; k < 8 * s + 8; k++) {
        int a = k, b = k;  // the reachable interval
        for (int i = 0; i < K; i++) {
          const int ps0 = K - 1 - i, ps1 = K - 2 - i + W;
          const int r = b < ps1 ? b : ps1;  // rightmost position that can move right
          if (r >= (a > ps0 ? a : ps0) && r + 1 > b) b = r + 1;
          const int l = a > ps0 + 1 ? a : ps0 + 1;  // leftmost position that can move left
          if (l <= (b < ps1 + 1 ? b : ps1 + 1) && l - 1 < a) a = l - 1;
        }
        if (b > NB - 1) b = NB - 1;
        if (a < lo) lo = a;
        if (b > hi) hi = b;
      }
      n0[s] = lo / 16 * 16;
      n1[s] = (hi / 16 + 1) * 16;
    }
    off[0] = 0;
    for (int s = 0; s < S; s++) off[s + 1] = off[s] + 2 * (n1[s] - n0[s]) * 16;
  }
};
template <int NB>
__host__ __device__ constexpr uint32_t blob_part_bytes() { return (uint32_t)Cone<NB>().off[NB / 8]; }

// The table as a kernel parameter (filled on the host from Cone<NB>).
struct ConeTable {
  int n0[16], n1[16], off[17];
};
template <int NB>
ConeTable cone_table() {
  constexpr Cone<NB> c{};
  ConeTable t{};
  for (int s = 0; s < NB / 8; s++) {
    t.n0[s] = c.n0[s];
    t.n1[s] = c.n1[s];
    t.off[s] = c.off[s];
  }
  t.off[NB / 8] = c.off[NB / 8];
  return t;
}

// ---------------------------------------------------------------------------
// the blocks of one band
// ---------------------------------------------------------------------------
// Block x forms tile j = first + x of band b with kFormThreads threads: thread
// (g, r) = (tid / NB, tid % NB) works on row r of G, G(r, c) at Gs[c * S + r]
// (the rows of one column contiguous: a warp's accesses are conflict-free),
// starting from the identity.  First the tile's rotations are gathered into
// shared memory, chase by chase (rec = (column of the pair in the tile,
// c, s)); then the chases are applied in order, separated by barriers, each
// chase's rotations -- disjoint pairs -- dealt to the kFormGroups groups of
// threads.  Output: blob x = [hi | lo], each the block as the MMA's B operand
// (K = the row index of G, N = its column index) in the compact layout of
// Cone, written in order of its 16-byte chunks.
constexpr int kFormThreads = 512;

struct FormRec {
  int l;
  float c, s;
};

template <int NB>
__host__ __device__ constexpr size_t form_smem_bytes() {
  // G, the per-chase record offsets (K + 1 ints) and the records (at most
  // W / 2 + 1 per chase: pair starts W apart, two columns apart at least)
  return (size_t)NB * (NB + 4) * 4 + 16 * ((4 * (NB / 2 + 1) + 15) / 16) +
         (size_t)(NB / 2) * (NB / 4 + 1) * sizeof(FormRec);
}

template <int NB>
__global__ void __launch_bounds__(kFormThreads) k_tc_form(const int32_t *__restrict__ Ca, const float2 *__restrict__ Cf,
                                                          const int4 *__restrict__ desc, int T, int cap, int b0,
                                                          int max_tiles, const int2 *__restrict__ ranges,
                                                          float *__restrict__ blobs, const ConeTable cone,
                                                          int *__restrict__ status) {
  constexpr int K = NB / 2, W = NB / 2, S = NB + 4, G = kFormThreads / NB;
  extern __shared__ __align__(16) float Gs[];
  int *off = reinterpret_cast<int *>(Gs + NB * S);  // K + 1 offsets into rec
  FormRec *rec = reinterpret_cast<FormRec *>(reinterpret_cast<unsigned char *>(off) + 16 * ((4 * (K + 1) + 15) / 16));
  __shared__ int cnt_s[K], e0_s[K];
  // block (band b0 + i, tile t) at i * max_tiles + t; its blob at the same index
  const int b = b0 + (int)blockIdx.x / max_tiles;
  const int2 rg = ranges[b];
  const int j = rg.x + (int)blockIdx.x % max_tiles;
  if (j > rg.y) return;
  const int tid = threadIdx.x, r = tid % NB, g = tid / NB;
  const int o = band_offset(b, W);
  const int base = j * W - K - o;  // column of X that is column 0 of the tile
  for (int q = tid; q < NB * NB; q += kFormThreads) {
    const int c = q / NB, rr = q % NB;
    Gs[c * S + rr] = (c == rr) ? 1.f : 0.f;
  }
  // each chase's records in this tile: [e0, e0 + cnt)
  if (tid < K) {
    const int i = tid, t = b * K + i;
    int e0 = 0, e1 = 0;
    if (t < T) {
      const int4 d = desc[t];
      const int cnt = d.y & 0xffffff, code = d.y >> 24;
      const int lo = j * W - 1 - i - o, hi = lo + W;  // this tile's pair starts in chase t
      if (code != kEmpty && d.w >= lo && d.z < hi) {
        if (code < 5) {
          // gap-free: record e starts at column d.z + step * e
          const int step = code < 2 ? 2 : 3;
          e0 = lo <= d.z ? 0 : (lo - d.z + step - 1) / step;
          e1 = min(cnt, (hi - d.z + step - 1) / step);
        } else {
          const size_t rb = (size_t)t * cap;
          e0 = lower_bound(Ca + rb, cnt, lo + 1);  // Ca holds 1-based pair starts
          e1 = lower_bound(Ca + rb, cnt, hi + 1);
        }
      }
    }
    e0_s[i] = e0;
    cnt_s[i] = max(0, min(e1 - e0, W / 2 + 1));
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int i = 0; i < K; i++) {
      off[i] = acc;
      acc += cnt_s[i];
    }
    off[K] = acc;
  }
  __syncthreads();
  // gather: warp w takes chases w, w + 16, ...
  for (int i = tid >> 5; i < K; i += kFormThreads / 32) {
    const int t = b * K + i, n = cnt_s[i];
    if (n == 0) continue;
    const int4 d = desc[t];
    const int code = d.y >> 24, step = code < 2 ? 2 : 3;
    const size_t rb = (size_t)t * cap;
    for (int q = tid & 31; q < n; q += 32) {
      const int e = e0_s[i] + q;
      int l = (code < 5 ? d.z + step * e : Ca[rb + e] - 1) - base;
      const float2 cs = Cf[rb + e];
      if (l < 0 || l > NB - 2) {
        atomicOr(status, ERR_RANGE);
        l = -1;  // skipped below
      }
      rec[off[i] + q] = FormRec{l, cs.x, cs.y};
    }
  }
  __syncthreads();
  // apply, chase by chase
  const bool active = g < G;  // threads beyond G whole groups of NB (NB = 96) idle here
  for (int i = 0; i < K; i++) {
    const int r0 = off[i], r1 = off[i + 1];
#pragma unroll 2
    for (int q = r0 + g; active && q < r1; q += G) {
      const FormRec f = rec[q];
      if (f.l < 0) continue;
      float *px = Gs + f.l * S + r;
      const float x = px[0], y = px[S];
      px[0] = fmaf(f.c, x, f.s * y);
      px[S] = fmaf(f.c, y, -f.s * x);
    }
    __syncthreads();
  }
  constexpr uint32_t part = blob_part_bytes<NB>();
  unsigned char *oh = reinterpret_cast<unsigned char *>(blobs) + (size_t)blockIdx.x * 2 * part;
  unsigned char *ol = oh + part;
#pragma unroll
  for (int s = 0; s < NB / 8; s++) {
    const int ngn = (cone.n1[s] - cone.n0[s]) / 8, ng0 = cone.n0[s] / 8;
    // 16-byte chunks of step s in order: (K chunk, core, row of the core)
    for (int idx = tid; idx < 2 * ngn * 8; idx += kFormThreads) {
      const int r8 = idx & 7, core = (idx >> 3) % ngn, kc = 2 * s + (idx >> 3) / ngn;
      const float4 v = *reinterpret_cast<const float4 *>(Gs + ((ng0 + core) * 8 + r8) * S + 4 * kc);
      uint4 h, l;
      split_tf32(v.x, h.x, l.x);
      split_tf32(v.y, h.y, l.y);
      split_tf32(v.z, h.z, l.z);
      split_tf32(v.w, h.w, l.w);
      *reinterpret_cast<uint4 *>(oh + cone.off[s] + (size_t)idx * 16) = h;
      *reinterpret_cast<uint4 *>(ol + cone.off[s] + (size_t)idx * 16) = l;
    }
  }
}

// ---------------------------------------------------------------------------
// the products of one band
// ---------------------------------------------------------------------------
// v (N columns of this thread's row) into A hi / A lo at column col0
template <int N>
__device__ __forceinline__ void st_split_cols(uint32_t tm, uint32_t lane_off, int col0, const float (&v)[N]) {
#pragma unroll
  for (int c = 0; c < N; c += 16) {
    uint32_t h[16], l[16];
#pragma unroll
    for (int q = 0; q < 16; q++) split_tf32(v[c + q], h[q], l[q]);
    tmem_st16(tm + lane_off + kColAH + col0 + c, h);
    tmem_st16(tm + lane_off + kColAL + col0 + c, l);
  }
}

template <int NB>
__host__ __device__ constexpr size_t apply_smem_bytes() {
  // two B blobs, one buffer of the panel's new columns
  return (size_t)2 * 2 * blob_part_bytes<NB>() + (size_t)(NB / 2) * 128 * 4;
}

// Warps 0-7 are row warps: warp w serves TMEM lanes (panel rows)
// 32 (w % 4) .. + 31, one row per thread, and half h = w / 4 of the work:
// h = 0 the first W outputs (final after the tile), h = 1 the last K outputs,
// which are the next tile's first K inputs (the carry); each half also takes
// part of the W new input columns (32 + 32, 32 + 16 or 16 + 16).  The two warps of a lane quarter combine
// their squared norms through shared memory (named barrier 1 + quarter).
// Warp 8 issues the copies and MMAs.  Tensor memory: D (the main
// accumulator) at columns [0, NB), A hi at [128, 128 + NB), A lo at
// [256, 256 + NB), the correction accumulator at [384, 384 + NB); A's
// columns [0, K) hold the carry, [K, NB) the new columns.  The MMAs of k-step
// s cover only the output columns of Cone, so both accumulators are cleared
// (tcgen05.st of zeros) before a tile's MMAs.  Shared memory: two B blobs
// (tile q in buffer q & 1, loaded one tile ahead, while the previous tile's
// MMAs run), then one buffer of the panel's W new columns (column-major, 128
// rows), loaded by bulk copies while the previous tile's MMAs run when the
// panel is whole and the leading dimension a multiple of 4 (16-byte aligned
// columns), else read by the row threads themselves.  Barriers: bar_b[2] (a
// blob has landed; one phase per use), bar_a (the eight row warps have
// written A), bar_m (the tile's MMAs have completed: frees A, its blob
// buffer and the accumulators' contents for reading), bar_n (the new columns
// have landed), one phase per tile each.  (Nine warps: a sub-partition of the
// SM holds three, which bounds the kernel at 168 registers a thread.)
constexpr int kRowWarps = 8;
constexpr int kApplyThreads2 = (kRowWarps + 1) * 32;

// Bands in flight.  One launch applies a chunk of bands: the block of band
// b0 + i and panel p (index i * panels + p) runs beside the blocks of the
// bands before it, a couple of tiles behind band b - 1's block of the same
// panel.  Each row warp of a block publishes a progress word, a column bound
// (offset by kBias, INT_MAX when the block is done) below which X's columns
// of its rows are final for its band: the four warps that store finals
// during the band (half 0) publish the minimum of what they have stored and
// of band b - 1's words, so that the least of a block's eight words holds for
// every earlier band too; the carry warps (half 1) store only at the end.  A
// block reads a column of X only once band b - 1's eight words have passed
// it.  It waits only on a block of a lower index, which starts no later than
// itself.
constexpr int kBias = 1 << 24;
__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
// the least of band b - 1's eight progress words (INT_MAX without one)
__device__ __forceinline__ int pred_bound(const int *pred) {
  if (!pred) return INT_MAX;
  int mn = INT_MAX;
#pragma unroll
  for (int w = 0; w < kRowWarps; w++) mn = min(mn, ld_acquire(pred + w));
  return mn;
}
// waits (bounded) until band b - 1's columns below `need` (biased) are final
__device__ __forceinline__ bool wait_pred(const int *pred, int need) {
  if (!pred) return true;
  for (int it = 0; it < async::kSpin; it++) {
    if (pred_bound(pred) >= need) return true;
    __nanosleep(100);
  }
  return false;
}

// 16 columns of this thread's row into A hi / A lo at column col
__device__ __forceinline__ void st_split16(uint32_t tm, uint32_t lane_off, int col, const float (&v)[16]) {
  uint32_t h[16], l[16];
#pragma unroll
  for (int q = 0; q < 16; q++) split_tf32(v[q], h[q], l[q]);
  tmem_st16(tm + lane_off + kColAH + col, h);
  tmem_st16(tm + lane_off + kColAL + col, l);
}

template <int NB>
__global__ void __launch_bounds__(kApplyThreads2, 1)
    k_tc_apply(float *__restrict__ X, int64_t ld, int nrow, int ncol, const unsigned char *__restrict__ blobs,
               const int2 *__restrict__ ranges, int b0, int panels, int max_tiles, int *__restrict__ progress,
               const ConeTable cone, int *__restrict__ status) {
  constexpr int K = NB / 2, W = NB / 2, H = NB / 2;  // H: outputs per row warp
  // the W new columns are split between the two halves in multiples of 16
  // (the width of a tcgen05.st): half 0 takes kNw0, half 1 the rest
  constexpr int kNw0 = (W / 2 + 15) / 16 * 16, kNw1 = W - kNw0;
  static_assert(K % 16 == 0 && H % 16 == 0 && kNw0 % 16 == 0 && kNw1 % 16 == 0 && kNw1 > 0, "16-column groups");
  constexpr uint32_t kPart = blob_part_bytes<NB>(), kBlob = 2 * kPart;
  constexpr uint32_t kNvCol = kRows * 4u;  // bytes of one new column of the panel
  extern __shared__ __align__(1024) unsigned char sB[];  // [2][kBlob], then the new columns
  float *nvbuf = reinterpret_cast<float *>(sB + 2 * kBlob);  // [W][kRows]
  __shared__ uint64_t bar_b[2], bar_a, bar_m, bar_n;
  __shared__ uint32_t tmem_s;
  __shared__ volatile int dead;
  __shared__ float2 xchg[2][kRows];  // per half and row: (squared output norm, squared input norm)
  const int bi = (int)blockIdx.x / panels, panel = (int)blockIdx.x % panels, b = b0 + bi;
  const int2 rg = ranges[b];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int *prog = progress + ((size_t)bi * panels + panel) * kRowWarps;  // this block's words
  const int *pred = bi > 0 ? progress + ((size_t)(bi - 1) * panels + panel) * kRowWarps : nullptr;
  if (rg.y < rg.x) {
    // no rotation in this band (the same for the whole block): done once band b - 1 is
    if (tid < kRowWarps) {
      if (!wait_pred(pred, INT_MAX)) atomicOr(status, ERR_APPLY);
      st_release(prog + tid, INT_MAX);
    }
    return;
  }
  blobs += (size_t)bi * max_tiles * (2 * blob_part_bytes<NB>());
  const int ntiles = rg.y - rg.x + 1;
  const int row0 = panel * kRows;
  const bool bulk = (ld % 4) == 0 && row0 + kRows <= nrow;  // the same for the whole block
  const int o = band_offset(b, W);
  if (warp == 0) {
    tmem_alloc(&tmem_s, kTmemCols);
    tmem_relinquish();
  }
  if (tid == 32) {
    async::mbar_init(&bar_b[0], 1);
    async::mbar_init(&bar_b[1], 1);
    async::mbar_init(&bar_a, kRowWarps);
    async::mbar_init(&bar_m, 1);
    async::mbar_init(&bar_n, 1);
    async::mbar_init_fence();
    dead = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = tmem_s;

  if (warp == kRowWarps) {
    // ---- MMA warp (one thread)
    if (lane == 0) {
      auto issue_blob = [&](int q) {
        uint64_t *bar = &bar_b[q & 1];
        unsigned char *dst = sB + (size_t)(q & 1) * kBlob;
        const unsigned char *src = blobs + (size_t)q * kBlob;
        async::mbar_arrive_tx(bar, kBlob);
        for (uint32_t off = 0; off < kBlob; off += kCopyChunk)
          async::bulk_g2s(dst + off, src + off, kBlob - off < kCopyChunk ? kBlob - off : kCopyChunk, bar);
      };
      // new columns of tile q (columns outside X are not copied), once band
      // b - 1 is done with them
      auto issue_nv = [&](int q) {
        const int c0 = (rg.x + q) * W - o;
        if (!wait_pred(pred, c0 + W + kBias)) {
          atomicOr(status, ERR_APPLY);
          dead = 1;
        }
        asm volatile("fence.proxy.async.global;\n" ::: "memory");  // the copies read what band b - 1 stored
        const int lo = max(c0, 0), hi = min(c0 + W, ncol);
        async::mbar_arrive_tx(&bar_n, hi > lo ? (unsigned)(hi - lo) * kNvCol : 0u);
        for (int col = lo; col < hi; col++)
          async::bulk_g2s(nvbuf + (size_t)(col - c0) * kRows, X + (size_t)col * ld + row0, kNvCol, &bar_n);
      };
      int committed = 0, blobs_issued = 1, nv_issued = 0;
      issue_blob(0);
      if (bulk) {
        issue_nv(0);
        nv_issued = 1;
      }
      for (int q = 0; q < ntiles && !dead; q++) {
        // tile q + 1's blob into the buffer of tile q - 1, free once its MMAs are done
        if (q > 0 && !async::mbar_wait(&bar_m, (unsigned)((q - 1) & 1))) {
          atomicOr(status, ERR_APPLY);
          dead = 1;
          break;
        }
        if (q + 1 < ntiles) {
          issue_blob(q + 1);
          blobs_issued = q + 2;
        }
        if (!async::mbar_wait(&bar_b[q & 1], (unsigned)((q >> 1) & 1)) ||
            !async::mbar_wait(&bar_a, (unsigned)(q & 1))) {
          atomicOr(status, ERR_APPLY);
          dead = 1;
          break;
        }
        // the row warps have read the new columns of tile q: the buffer takes tile q + 1's
        if (bulk && q + 1 < ntiles) {
          issue_nv(q + 1);
          nv_issued = q + 2;
        }
        tc_fence_after();
        const uint32_t bh = su32(sB + (size_t)(q & 1) * kBlob), bl = bh + kPart;
#pragma unroll
        for (int s = 0; s < NB / 8; s++) {
          const uint32_t n = cone.n1[s] - cone.n0[s];
          const uint32_t idesc = idesc_tf32(kRows, (int)n);
          const uint64_t dh = smem_desc(bh + cone.off[s], n / 8 * 128, 128u);
          const uint64_t dl = smem_desc(bl + cone.off[s], n / 8 * 128, 128u);
          mma_tf32(tm + kColD + cone.n0[s], tm + kColAH + 8 * s, dh, idesc, 1u);
          mma_tf32(tm + kColDC + cone.n0[s], tm + kColAH + 8 * s, dl, idesc, 1u);
          mma_tf32(tm + kColDC + cone.n0[s], tm + kColAL + 8 * s, dh, idesc, 1u);
        }
        mma_commit(&bar_m);
        committed = q + 1;
      }
      if (dead) {
        // nothing of this thread stays in flight: its copies and MMAs
        for (int q = committed; q < blobs_issued; q++) async::mbar_wait(&bar_b[q & 1], (unsigned)((q >> 1) & 1));
        if (nv_issued > 0) async::mbar_wait(&bar_n, (unsigned)((nv_issued - 1) & 1));
        if (committed > 0) async::mbar_wait(&bar_m, (unsigned)((committed - 1) & 1));
      }
    }
  } else {
    // ---- row warps
    const int quarter = warp & 3, half = warp >> 2;
    const int r = quarter * 32 + lane;  // panel row <-> TMEM lane
    const int row = row0 + r;
    const bool rv = row < nrow;
    const float *xr = X + (rv ? row : 0);  // read: columns no earlier tile of the band has written
    float *xw = X + (rv ? row : 0);
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const uint32_t dcol = tm + lane_off + kColD + half * H;  // this warp's half of the outputs
    const uint32_t zero16[16] = {};
    float in2 = 0.f;  // squared norm of this thread's share of the inputs to the tile in flight
    float keep[H];    // finals (half 0) or carry (half 1) of the previous tile, scaled
    // Reads this warp's half of the previous tile's outputs (the two
    // accumulators added in FP32) into keep, clears them for the next tile,
    // and scales keep to restore the row's norm.  G is orthogonal, so each
    // row's 2-norm over the tile's NB columns is the same before and after
    // the product; the tensor cores' FP32 accumulation truncates toward zero
    // and shrinks it by about one unit in the last place per MMA step.  The
    // factor (both halves' sums combined) is 1 up to that bias, which would
    // otherwise add up over the bands of every update.
    auto take_outputs = [&]() {
      float o2a = 0.f, o2b = 0.f;
#pragma unroll
      for (int c = 0; c < H; c += 16) {
        uint32_t v[16], w[16];
        tmem_ld16(dcol + c, v);
        tmem_ld16(dcol + (kColDC - kColD) + c, w);
        tc_wait_ld();
#pragma unroll
        for (int qq = 0; qq < 16; qq += 2) {
          keep[c + qq] = __uint_as_float(v[qq]) + __uint_as_float(w[qq]);
          keep[c + qq + 1] = __uint_as_float(v[qq + 1]) + __uint_as_float(w[qq + 1]);
          o2a = fmaf(keep[c + qq], keep[c + qq], o2a);
          o2b = fmaf(keep[c + qq + 1], keep[c + qq + 1], o2b);
        }
      }
      const float o2 = o2a + o2b;
      xchg[half][r] = make_float2(o2, in2);
      async::named_sync(1 + quarter, 64);
      const float2 other = xchg[half ^ 1][r];
      const float out2 = o2 + other.x, inp2 = in2 + other.y;
      const float sc = (out2 > 0.f && inp2 > 0.f) ? sqrtf(inp2 / out2) : 1.f;
#pragma unroll
      for (int c = 0; c < H; c++) keep[c] *= sc;
      // both halves have read xchg before either writes it again: the next
      // write follows the next tile's MMAs, which wait for both (bar_a)
    };
    auto clear_outputs = [&]() {
#pragma unroll
      for (int c = 0; c < H; c += 16) {
        tmem_st16(dcol + c, zero16);
        tmem_st16(dcol + (kColDC - kColD) + c, zero16);
      }
    };
    auto store_keep = [&](int g0) {
      float *p = xw + (int64_t)g0 * ld;  // walks the columns (an address, dereferenced only inside X)
#pragma unroll
      for (int c = 0; c < H; c++, p += ld) {
        const int col = g0 + c;
        if (rv && col >= 0 && col < ncol) *p = keep[c];
      }
    };
    // this warp's progress word: its rows' columns below `bound` (unbiased)
    // are final for this band and band b - 1 (the warp's stores ordered
    // before the word by the warp barrier and lane 0's release)
    auto publish = [&](int bound) {
      __syncwarp();
      if (lane == 0) {
        __threadfence();
        st_release(prog + warp, min(bound + kBias, pred_bound(pred)));
      }
    };
    // half 1 writes X only at the end, the columns from the last tile's carry on
    if (half == 1 && lane == 0) st_release(prog + warp, rg.y * W - o + kBias);
    for (int q = 0; q < ntiles; q++) {
      if (dead) break;
      const int j = rg.x + q;
      if (q > 0) {
        if (!async::mbar_wait(&bar_m, (unsigned)((q - 1) & 1))) {
          if (lane == 0) atomicOr(status, ERR_APPLY);
          dead = 1;
          break;
        }
        tc_fence_after();
        take_outputs();
      }
      clear_outputs();
      float sa = 0.f, sb = 0.f;
      // columns of X this tile reads directly: the band's first carry (half 1)
      // and, without bulk copies, the new columns
      if ((q == 0 && half == 1) || !bulk) {
        const int need = bulk ? j * W - o : j * W + W - o;
        bool ok = true;
        if (lane == 0) ok = wait_pred(pred, need + kBias);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        __syncwarp();  // the warp's reads of X follow lane 0's acquire
        if (!ok) {
          if (lane == 0) atomicOr(status, ERR_APPLY);
          dead = 1;
          break;
        }
      }
      if (half == 1) {
        // the carry: the previous tile's last K outputs, or X's columns
        // [j W - K - o, j W - o) for the band's first tile
        if (q == 0) {
          const int g0 = j * W - K - o;
          const float *p = xr + (int64_t)g0 * ld;
#pragma unroll
          for (int c = 0; c < K; c++, p += ld) {
            const int col = g0 + c;
            keep[c] = (rv && col >= 0 && col < ncol) ? *p : 0.f;
          }
        }
#pragma unroll
        for (int c = 0; c < K; c += 16) {
          float v[16];
#pragma unroll
          for (int qq = 0; qq < 16; qq += 2) {
            v[qq] = keep[c + qq];
            v[qq + 1] = keep[c + qq + 1];
            sa = fmaf(v[qq], v[qq], sa);
            sb = fmaf(v[qq + 1], v[qq + 1], sb);
          }
          st_split16(tm, lane_off, c, v);
        }
      }
      // this half's share of the W new columns [j W - o, j W - o + W):
      // columns [cb, cb + nw) of them
      const int c0 = j * W - o;
      if (bulk && !async::mbar_wait(&bar_n, (unsigned)(q & 1))) {
        if (lane == 0) atomicOr(status, ERR_APPLY);
        dead = 1;
        break;
      }
      {
        const int cb = half ? kNw0 : 0, nw = half ? kNw1 : kNw0;
        const float *nb_ = nvbuf + r;
        const float *p = xr + (int64_t)(c0 + cb) * ld;
#pragma unroll
        for (int c = 0; c < kNw0; c += 16) {
          if (c >= nw) break;  // (uniform per warp)
          float v[16];
#pragma unroll
          for (int qq = 0; qq < 16; qq++, p += ld) {
            const int col = c0 + cb + c + qq;
            const bool in = col >= 0 && col < ncol;
            v[qq] = bulk ? (in ? nb_[(cb + c + qq) * kRows] : 0.f) : ((rv && in) ? *p : 0.f);
          }
#pragma unroll
          for (int qq = 0; qq < 16; qq += 2) {
            sa = fmaf(v[qq], v[qq], sa);
            sb = fmaf(v[qq + 1], v[qq + 1], sb);
          }
          st_split16(tm, lane_off, K + cb + c, v);
        }
      }
      in2 = sa + sb;
      tc_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) async::mbar_arrive(&bar_a);
      // the previous tile's finals, while this tile's MMAs run
      if (q > 0 && half == 0) store_keep((j - 1) * W - K - o);
      if (half == 0) publish(q > 0 ? (j - 1) * W - o : rg.x * W - K - o);
    }
    if (!dead) {
      if (!async::mbar_wait(&bar_m, (unsigned)((ntiles - 1) & 1))) {
        if (lane == 0) atomicOr(status, ERR_APPLY);
        dead = 1;
      } else {
        tc_fence_after();
        take_outputs();
        store_keep(rg.y * W - K - o + half * H);  // the last tile's columns, all final
      }
    }
    // done: once band b - 1 is (also after a failure, so that later bands end)
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      if (!wait_pred(pred, INT_MAX)) atomicOr(status, ERR_APPLY);
      st_release(prog + warp, INT_MAX);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tm, kTmemCols);
}

constexpr int kChunkBands = 16;  // bands per launch pair (form, apply)

template <int NB>
cudaError_t run_bands(float *X, int64_t ld, int nrow, int ncol, const RotStream &st, int side, int *status,
                      int2 *ranges, float *blobs, int *progress, int nbands, int max_tiles, cudaStream_t s) {
  const int32_t *Ca = side == 0 ? st.La : st.Ra;
  const float2 *Cf = side == 0 ? st.Lf : st.Rf;
  const int4 *desc = side == 0 ? st.Lm : st.Rm;
  const size_t form_smem = form_smem_bytes<NB>();
  const size_t apply_smem = apply_smem_bytes<NB>();
  cudaError_t e = cudaFuncSetAttribute(k_tc_form<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)form_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_apply<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)apply_smem);
  if (e != cudaSuccess) return e;
  const int panels = (nrow + kRows - 1) / kRows;
  const ConeTable cone = cone_table<NB>();
  for (int b0 = 0; b0 < nbands; b0 += kChunkBands) {
    const int nb = min(kChunkBands, nbands - b0);
    e = cudaMemsetAsync(progress, 0, sizeof(int) * (size_t)nb * panels * kRowWarps, s);
    if (e != cudaSuccess) return e;
    k_tc_form<NB><<<nb * max_tiles, kFormThreads, form_smem, s>>>(Ca, Cf, desc, st.T, st.cap, b0, max_tiles, ranges,
                                                                  blobs, cone, status);
    k_tc_apply<NB><<<nb * panels, kApplyThreads2, apply_smem, s>>>(
        X, ld, nrow, ncol, reinterpret_cast<const unsigned char *>(blobs), ranges, b0, panels, max_tiles, progress,
        cone, status);
  }
  return cudaGetLastError();
}

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

// Workspace of the blocked apply: the band ranges, the progress words of a
// chunk of bands, then the chunk's blobs.
// A band's tiles j run over floor((a + i + 1 + o) / W) for pair starts a in
// [0, ncol - 2], i < K and o < W: at most (ncol + K + W) / W + 1 of them.
static int tc_max_tiles(int ncol, int nb) { return (ncol + nb) / (nb / 2) + 2; }
static size_t blob_bytes(int nb) {
  return nb == 64 ? 2 * blob_part_bytes<64>() : nb == 96 ? 2 * blob_part_bytes<96>() : 2 * blob_part_bytes<128>();
}
static size_t tc_progress_bytes(int nrow) {
  return align256(sizeof(int) * (size_t)kChunkBands * ((nrow + kRows - 1) / kRows) * kRowWarps);
}
size_t tc_workspace_bytes(int ncol, int T, int nb) {
  const int K = nb / 2;
  const int nbands = (T + K - 1) / K;
  const int max_tiles = tc_max_tiles(ncol, nb);
  // (nrow <= ncol + 1 for every factor the apply serves: Q is m x m, P n x n)
  return align256((size_t)(nbands + 1) * sizeof(int2)) + tc_progress_bytes(ncol + 1) +
         (size_t)kChunkBands * max_tiles * blob_bytes(nb);
}

cudaError_t launch_apply_tc(float *X, int64_t ld, int nrow, int ncol, const RotStream &st, int side,
                            bool with_spike, int *status, bool desc_ready, int nb, void *ws, size_t ws_bytes,
                            cudaStream_t s) {
  const int4 *desc = side == 0 ? st.Lm : st.Rm;
  const float2 *coef = side == 0 ? st.Lf : st.Rf;
  if ((nb != 64 && nb != 96 && nb != 128) || !desc || !coef || !status || !ws || nrow < 1 || ncol < 2 ||
      ws_bytes < tc_workspace_bytes(ncol, st.T, nb))
    return cudaErrorNotSupported;
  cudaError_t e = cudaSuccess;
  if (st.T > 0 && !desc_ready) e = launch_chase_descriptors(st, side, s);
  if (e == cudaSuccess && with_spike) e = launch_apply_spike32(X, ld, nrow, st, s);
  if (e != cudaSuccess || st.T <= 0) return e;
  const int K = nb / 2, W = nb / 2;
  const int nbands = (st.T + K - 1) / K;
  const int max_tiles = tc_max_tiles(ncol, nb);
  int2 *ranges = reinterpret_cast<int2 *>(ws);
  int *progress = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(ws) +
                                          align256((size_t)(nbands + 1) * sizeof(int2)));
  float *blobs = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(progress) + tc_progress_bytes(nrow));
  if (nrow > ncol + 1) return cudaErrorNotSupported;  // the workspace is sized for nrow <= ncol + 1
  k_tc_band_ranges<<<(nbands + 127) / 128, 128, 0, s>>>(desc, st.T, K, W, nbands, max_tiles, ranges, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (nb == 64) return run_bands<64>(X, ld, nrow, ncol, st, side, status, ranges, blobs, progress, nbands, max_tiles, s);
  if (nb == 96) return run_bands<96>(X, ld, nrow, ncol, st, side, status, ranges, blobs, progress, nbands, max_tiles, s);
  return run_bands<128>(X, ld, nrow, ncol, st, side, status, ranges, blobs, progress, nbands, max_tiles, s);
}

}  // namespace bdu
