// K2: rotation generation and bulge chasing for one rank-1 column
// (Sec. 3.4, Algorithm 2), in FP64.
//
// The reduction of the core M = Bd + u v^T is a sequence of "chases": each
// starts with one rotation and pushes the bulge it creates down the band.
// Chases are generated in a fixed order (the schedule below) and every chase
// moves monotonically down the band, so chase t may run concurrently with
// chase t-1 as long as it stays a few positions behind it.  The engine gives
// each chase to one thread and advances all runnable chases by one rotation
// per synchronous step; a chase runs only when the nearest earlier unfinished
// chase is at least D positions ahead (D = 3 between phase-1 chases, 2 from
// the last phase-2 chase to a phase-3 one, 4 otherwise).  This keeps every
// band cell's read/write order identical to the sequential algorithm, so the
// result equals a one-rotation-at-a-time execution.
//
// Two engines share the chase logic:
//   * one CTA (small n): the band sits in that CTA's shared memory when it
//     fits, else in global memory; steps are separated by __syncthreads;
//   * a thread-block cluster of 16 CTAs (large n): the band's rows are
//     partitioned over the CTAs' shared memories and reached through
//     distributed shared memory; chases are dealt round-robin to the CTAs, and
//     steps are separated by cluster barriers.  This multiplies the FP64
//     throughput available to the chases (GB300 issues about two FP64 FMAs
//     per SM per clock).
//
// Schedule (1-based; N = n+1 if m > n else n):
//   spike:    j = m..n+2: left (j-1, j) zeroing u(j)             [one thread]
//   phase 1:  chase P1(j), j = N..2: left (j-1, j) zeroing u(j); then for
//             i = j-1, j+1, ...: right (i+1, i+2) zeroing M(i, i+2), left
//             (i+2, i+3) zeroing M(i+3, i+1), while the bulge exists
//   fold:     row 1 += u(1) v^T                                   [all threads]
//   phase 2:  chase P2(j), j = n..3: right (j-1, j) zeroing M(1, j), then
//             chase_lower(j-1)
//   phase 3:  chases P3b(i), P3c(i), i = 1..n-1 (and n when N = n+1):
//             P3b: left (i, i+1) zeroing M(i+1, i); right (i+2, i+3)
//                  zeroing M(i, i+3); chase_lower(i+2)
//             P3c: right (i+1, i+2) zeroing M(i, i+2); chase_lower(i+1)
//   chase_lower(k): left (k+1, k+2) zeroing M(k+2, k); right (k+3, k+4)
//             zeroing M(k+1, k+4); k += 3, while the bulge exists.
//
// Arithmetic.  Exact (FP64 form): every multiply, add, divide and square root
// is a separately rounded IEEE operation (__dmul_rn, __dadd_rn, __ddiv_rn,
// __dsqrt_rn), never a fused multiply-add, so each value is fully determined
// by its inputs.  Fast (mixed form, where Q and P are FP32 anyway): fused
// multiply-adds, and 1/sqrt(f^2 + g^2) from an FP32 seed refined by one
// third-order Newton step in FP64 (error well below an FP64 ulp), which
// avoids the long-latency FP64 division and square-root sequences.
#include <climits>
#include <cooperative_groups.h>
#include <cstdio>

#include "bdu_internal.cuh"

namespace cg = cooperative_groups;

namespace bdu {
namespace {

constexpr int kMaxThreads = 256;
// A placeholder address for band entries outside the stored diagonals: such
// entries read as zero and their new values are checked (a nonzero one is
// reported) instead of stored, so it is never read or written.
__device__ double g_zero_sink[1];
constexpr int kMaxCluster = 16;
// Ops a chase may run in one step, each while it stays within the lag of the
// chase ahead as that chase stood at the start of the step (which only moves
// further ahead during the step), so any value gives the same results.  Two
// cut the steps at n = 4096 by a third (45k -> 31k) but made a step 1.66x
// longer (a warp runs the whole op again for whichever lanes can go on), so
// the chase took 13% longer: one op per step.
constexpr int kOpsPerStep = 1;

enum Kind : int { P1 = 0, P2 = 1, P3B = 2, P3C = 3 };
enum : int { S_L0 = 0, S_R1 = 1, S_L1 = 2, S_A = 3, S_B = 4, S_C = 5, S_CL = 6, S_CR = 7, S_P2 = 8 };

// ----------------------------------------------------------------------------
// rotation arithmetic
// ----------------------------------------------------------------------------
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
// x != 0 and |x| compared through the bit pattern, on the integer pipes
__device__ __forceinline__ bool nz(double x) { return (__double_as_longlong(x) << 1) != 0; }
__device__ __forceinline__ unsigned long long absbits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }

// Rotation generator (Eqs. giv, giv1, zero handling of Sec. 3.4):
// [c s; -s c][f; g] = [r; 0], c >= 0, r = sign(f) hypot(f, g).  Returns false
// when g == 0 (no rotation); f == 0 gives c = 0, s = 1, r = g.  hypot uses
// power-of-two safe scaling.  Written without branches on the common path so
// that the lanes of a warp share its (long-latency) FP64 instructions.
__device__ __forceinline__ bool rotg_exact(double f, double g, double &c, double &s, double &r) {
  const unsigned long long bf = absbits(f), bg = absbits(g);
  const unsigned long long bm = bf > bg ? bf : bg;  // |x| order = bit-pattern order
  const double sigma = bm > 0x5F30000000000000ULL ? 0x1p-600 : (bm < 0x20B0000000000000ULL ? 0x1p600 : 1.0);
  const double fs = mul(f, sigma), gs = mul(g, sigma);
  const double h = __dsqrt_rn(add(mul(fs, fs), mul(gs, gs)));
  const double rs = copysign(h, f);
  const bool fz = bf == 0;
  const double den = fz ? 1.0 : rs;
  c = fz ? 0.0 : __ddiv_rn(fs, den);
  s = fz ? 1.0 : __ddiv_rn(gs, den);
  r = fz ? g : __ddiv_rn(rs, sigma);
  return bg != 0;
}

// FP32 value of x (|x| <= 2, or NaN), rounded to nearest even, formed from
// the bit pattern on the integer pipes: on GB300 an FP64 <-> FP32 conversion
// instruction holds the SM sub-partition's FP64 unit for about 90 cycles.
// Magnitudes below 2^-126 (under FP32's normal range) become signed zero.
__device__ __forceinline__ float f32_of(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = b & 0x7fffffffffffffffULL;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  unsigned long long t = mag >> 29;  // exponent and the top 23 mantissa bits
  const unsigned rem = (unsigned)(mag & 0x1fffffffULL);
  t += (rem > 0x10000000u || (rem == 0x10000000u && (t & 1))) ? 1 : 0;
  unsigned r = (unsigned)(t - (896ULL << 23));  // exponent bias 1023 -> 127
  r = mag < (897ULL << 52) ? 0u : r;
  r = mag >= 0x7ff0000000000000ULL ? 0x7fc00000u : r;
  return __uint_as_float(r | sign);
}

// Same rotation from y ~ 1/sqrt(f^2 + g^2): both inputs are scaled exactly by
// the power of two that brings the larger into [0.5, 1), so q = f^2 + g^2 lies
// in [0.25, 2); y0 = rsqrtf(q) (q truncated to FP32 and y0 widened back
// through the bit patterns, about 22 correct bits) is refined by
// y = y0 (1 + e/2 + 3e^2/8) with e = 1 - q y0^2 (third-order Newton step,
// error about e^3).  Inputs outside [2^-1021, 2^1022), subnormal, or with a
// ratio below 2^-1021 take the exact path.  Results are those of the same
// formulas with the scalings done as FP64 multiplies (which are exact).
__device__ __forceinline__ bool rotg_fast(double f, double g, double &c, double &s, double &r) {
  const unsigned long long bf = absbits(f), bg = absbits(g);
  const unsigned long long bm = bf > bg ? bf : bg, bn = bf > bg ? bg : bf;
  const int ex = (int)(bm >> 52), en = (int)(bn >> 52);
  // the exact path when the scalings below would leave the normal range: the
  // larger input's exponent outside [2, 2044], or the smaller input subnormal
  // or more than 2^1021 below the larger
  if (bg != 0 && (ex < 2 || ex > 2044 || (bn != 0 && (en == 0 || en + 1021 < ex)))) return rotg_exact(f, g, c, s, r);
  // fs = f 2^(1022-ex), gs = g 2^(1022-ex) and r = |r_s| 2^(ex-1022): exact
  // power-of-two scalings, done on the exponent field (integer pipes)
  const long long dk = (long long)(1022 - ex) << 52;
  const double fs = bf == 0 ? 0.0 : __longlong_as_double(__double_as_longlong(f) + dk);
  const double gs = bg == 0 ? 0.0 : __longlong_as_double(__double_as_longlong(g) + dk);
  const double q = fma(fs, fs, gs * gs);
  const unsigned qf = (unsigned)(((unsigned long long)__double_as_longlong(q) >> 29) - (896ULL << 23));
  double y = __longlong_as_double((long long)(((unsigned long long)__float_as_uint(rsqrtf(__uint_as_float(qf))) << 29) +
                                              (896ULL << 52)));
  const double e = fma(-(q * y), y, 1.0);
  y = fma(y * e, fma(0.375, e, 0.5), y);
  const bool fz = bf == 0;
  const long long sf = __double_as_longlong(f) & (long long)0x8000000000000000ULL;  // sign(f)
  const double fa = __longlong_as_double((long long)absbits(fs));                  // |fs|
  const double gsg = __longlong_as_double(__double_as_longlong(gs) ^ sf);          // sign(f) gs
  const double qy = q * y;                                                         // |r| scaled, in [0.5, 1.5)
  c = fz ? 0.0 : fa * y;
  s = fz ? 1.0 : gsg * y;
  r = fz ? g : __longlong_as_double((__double_as_longlong(qy) - dk) ^ sf);
  return bg != 0;
}

template <bool FAST> struct Arith;
template <> struct Arith<false> {
  static __device__ __forceinline__ bool rot(double f, double g, double &c, double &s, double &r) {
    return rotg_exact(f, g, c, s, r);
  }
  static __device__ __forceinline__ double px(double c, double s, double x, double y) { return add(mul(c, x), mul(s, y)); }
  static __device__ __forceinline__ double py(double c, double s, double x, double y) { return add(mul(-s, x), mul(c, y)); }
};
template <> struct Arith<true> {
  static __device__ __forceinline__ bool rot(double f, double g, double &c, double &s, double &r) {
    return rotg_fast(f, g, c, s, r);
  }
  static __device__ __forceinline__ double px(double c, double s, double x, double y) { return fma(c, x, s * y); }
  static __device__ __forceinline__ double py(double c, double s, double x, double y) { return fma(c, y, -(s * x)); }
};

// ----------------------------------------------------------------------------
// cell stores.  Band cells: dg[j-i+2] at row i >= 2 (offsets -2..3); row 1 is
// dense (r1[j]); u(1..N), v(1..n).
// ----------------------------------------------------------------------------
struct LocalStore {
  double *dg0;  // diagonal o starts at dg0 + (o+2) * ld
  int ld;
  double *r1, *u, *v;
  __device__ __forceinline__ double *cell(int i, int j) const {
    return (i == 1) ? r1 + j : dg0 + (size_t)(j - i + 2) * ld + i;
  }
  static __device__ __forceinline__ double load(const double *p) { return *p; }
  __device__ __forceinline__ double *uptr(int i) const { return u + i; }
  __device__ __forceinline__ double *vptr(int j) const { return v + j; }
  // cell handles of the uniform op: offsets from dg0 (one contiguous buffer)
  using H = int;
  __device__ __forceinline__ H h_band(int diag, int i) const { return diag * ld + i; }
  __device__ __forceinline__ H h_r1(int j) const { return (int)(r1 - dg0) + j; }
  __device__ __forceinline__ H h_v(int j) const { return (int)(v - dg0) + j; }
  __device__ __forceinline__ H h_u(int i) const { return (int)(u - dg0) + i; }
  __device__ __forceinline__ double ld_h(H h) const { return dg0[h]; }
  __device__ __forceinline__ void st_h(H h, double x) const { dg0[h] = x; }
};

// The band of a thread-block cluster, in distributed shared memory: nine
// arrays indexed 0..N+1 (the six diagonals by row, row 1 and v by column, u by
// row), index i of every array held by CTA i % 16 at slot i / 16 of its slice
// (the same shared-memory offset in every CTA; interleaved, so that the rows
// the chases are working on are spread over all the CTAs).  An op's cells are
// reached by their shared::cluster addresses (mapa), the general path's by
// generic pointers into the cluster's shared-memory window; the cluster
// barrier between steps orders every CTA's stores before the next step's
// loads.
struct DsmStore {
  double *loc;          // this CTA's slice (generic address)
  const uint32_t *rb;   // shared::cluster address of every CTA's slice (rb[r] for rank r; in shared memory)
  int B;                // indices per array and CTA
  using H = uint32_t;   // a cell's shared::cluster address
  // (plans also form handles of cells they never touch -- pairs past the
  // matrix edge, unused slots: harmless, the rank is masked into range and
  // such a handle is never dereferenced)
  __device__ __forceinline__ H h_at(int arr, int idx) const {
    return rb[idx & (kMaxCluster - 1)] + (uint32_t)(arr * B + (idx >> 4)) * 8u;
  }
  __device__ __forceinline__ H h_band(int diag, int i) const { return h_at(diag, i); }
  __device__ __forceinline__ H h_r1(int j) const { return h_at(6, j); }
  __device__ __forceinline__ H h_v(int j) const { return h_at(7, j); }
  __device__ __forceinline__ H h_u(int i) const { return h_at(8, i); }
  __device__ __forceinline__ double ld_h(H h) const {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];\n" : "=d"(v) : "r"(h) : "memory");
    return v;
  }
  __device__ __forceinline__ void st_h(H h, double v) const {
    asm volatile("st.shared::cluster.f64 [%0], %1;\n" ::"r"(h), "d"(v) : "memory");
  }
  __device__ __forceinline__ double *gp(int arr, int idx) const {
    return static_cast<double *>(__cluster_map_shared_rank(loc + arr * B + (idx >> 4), (unsigned)(idx & (kMaxCluster - 1))));
  }
  __device__ __forceinline__ double *cell(int i, int j) const { return (i == 1) ? gp(6, j) : gp(j - i + 2, i); }
  __device__ __forceinline__ double *uptr(int i) const { return gp(8, i); }
  __device__ __forceinline__ double *vptr(int j) const { return gp(7, j); }
  static __device__ __forceinline__ double load(const double *p) { return *p; }
};
// Slice of the cluster band per CTA: B indices of each array, 16 B >= N + 2.
__host__ __device__ inline int dsm_slice(int N) { return (N + 2 + kMaxCluster - 1) / kMaxCluster; }

struct Rec {
  double *c, *s;
  int32_t *a;
  float2 *f;  // FP32 copy of (c, s), or null
  int cnt, cap;
  int *err;
  __device__ __forceinline__ void push(double cc, double ss, int aa) {
    if (cnt < cap) {
      a[cnt] = aa;
      if (c) { c[cnt] = cc; s[cnt] = ss; }
      if (f) f[cnt] = make_float2(f32_of(cc), f32_of(ss));
    } else {
      atomicOr(err, ERR_CAP);
    }
    cnt++;
  }
};

struct Task {
  int t;      // task id (>= T: slot exhausted)
  int kind, p;
  int st;     // state
  int ii;     // i (phase 1) or k (chase_lower)
  int pos;    // position of the next op
  bool started, done;
  int phase;  // 1..3, for the rotation counters
};

__device__ __forceinline__ void task_init(Task &k, int t, int T, int N, int n) {
  k.t = t;
  k.started = false;
  k.done = (t >= T);
  if (k.done) { k.pos = INT_MAX; return; }
  int p1 = N - 1, p2 = n > 2 ? n - 2 : 0;
  if (t < p1) {
    k.kind = P1; k.p = N - t; k.st = S_L0; k.pos = k.p - 1; k.phase = 1;
  } else if (t < p1 + p2) {
    k.kind = P2; k.p = n - (t - p1); k.st = S_P2; k.pos = k.p - 1; k.phase = 2;
  } else {
    int q = t - p1 - p2;
    k.p = q / 2 + 1;
    k.phase = 3;
    if ((q & 1) == 0) { k.kind = P3B; k.st = S_A; k.pos = k.p; }
    else { k.kind = P3C; k.st = S_C; k.pos = k.p + 1; }
  }
}

// Geometry of each op kind (the plan in Chaser::run_op), fixed at compile time
// for the interior of the band.  A row op rotates rows (a, a+1) over columns
// lo..lo+W-1, a column op columns (a, a+1) over rows lo..lo+W-1; SRC 0: the
// entry eliminated is the first pair's second, 1: u(a+1) against u(a),
// 2: row 1's (1, a+1) against (1, a); S_R1 also rotates v(a), v(a+1).  The
// diagonal (j - i + 2, in 0..5) of the pair's first cell is C + q (rows) or
// C - q (columns); the second cell's is one less (rows) or one more (columns).
// Every cell of every kind falls on one of the six stored diagonals.
struct Geo { bool rows; int w, src; bool withv; int c; };
__host__ __device__ constexpr Geo geo_of(int st) {
  return st == S_L0 ? Geo{true, 3, 1, false, 2}
       : st == S_R1 ? Geo{false, 4, 0, true, 3}
       : st == S_L1 ? Geo{true, 4, 0, false, 1}
       : st == S_P2 ? Geo{false, 4, 2, false, 3}
       : st == S_A  ? Geo{true, 4, 0, false, 2}
       : st == S_B  ? Geo{false, 5, 0, false, 4}
       : st == S_C  ? Geo{false, 4, 0, false, 3}
       : st == S_CL ? Geo{true, 5, 0, false, 1}
       :              Geo{false, 5, 0, false, 4};  // S_CR
}

// ----------------------------------------------------------------------------
// the chase logic, shared by both engines
// ----------------------------------------------------------------------------
template <class Store, bool FAST>
struct Chaser {
  using A = Arith<FAST>;
  Store S;
  int N, n, m;
  int *err;
  double *Ux, *Vx;
  int rx;
  double *zero;  // placeholder address of entries outside the band (never dereferenced)

  __device__ __forceinline__ bool inband(int i, int j) const {
    if (i < 1 || i > N || j < 1 || j > n) return false;
    if (i == 1) return true;
    const int o = j - i;
    return o >= -2 && o <= 3;
  }
  // an entry outside the band reads as zero without a memory access (a chase's
  // end test at the bottom of the band would otherwise wait on an L2 round trip)
  __device__ __forceinline__ double get(int i, int j) const { return inband(i, j) ? Store::load(S.cell(i, j)) : 0.0; }
  // The later columns of U (V) of a rank-r update: entries (a, a+1) of each
  // rotated like the band's pair.  Loads of four columns are issued together,
  // so that they share one L2 round trip.
  __device__ __forceinline__ void rotate_extra(double *X, int ld, int a, double c, double s) {
    for (int t0 = 0; t0 < rx; t0 += 4) {
      double xu[4], yu[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const double *U = X + (size_t)(t0 + q) * ld - 1;
        xu[q] = t0 + q < rx ? Store::load(U + a) : 0.0;
        yu[q] = t0 + q < rx ? Store::load(U + a + 1) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 4; q++) {
        if (t0 + q < rx) {
          double *U = X + (size_t)(t0 + q) * ld - 1;
          U[a] = A::px(c, s, xu[q], yu[q]);
          U[a + 1] = A::py(c, s, xu[q], yu[q]);
        }
      }
    }
  }

  // One rotation, described by its geometry:
  //   rows (left rotation on rows a, a+1) over columns lo..lo+w-1, or
  //   cols (right rotation on columns a, a+1) over rows lo..lo+w-1;
  //   src 0: the entry eliminated is the second of the first pair, i.e.
  //          (a+1, lo) or (lo, a+1); src 1: u(a+1) against u(a); src 2: row
  //          1's (1, a+1) against (1, a) (row 1 rotates besides the w rows);
  //   withv: v(a), v(a+1) rotate too (phase-1 right rotations).
  // The extra pair (u, row 1 or v) takes the last of the five pair slots,
  // which these ops leave free (w <= 4 whenever one is needed).  Every lane of
  // a warp runs the same instruction sequence whatever its op -- on GB300 each
  // FP64 warp instruction occupies its SM sub-partition's FP64 unit for tens of
  // cycles however many lanes are active, so lanes must share them: addresses
  // are formed first (entries outside the band read as zero and their new
  // values are checked, not stored), all loads are issued together, and the
  // rotation and the pair updates are branch-free.  Returns false (nothing written) when the entry to
  // eliminate is already zero; last receives the new value of (a, lo+w-1)
  // (rows) or (lo+w-1, a) (cols), the bulge the chase looks at next.
  __device__ __forceinline__ bool exec(bool isrows, int a, int lo, int w, int src, bool withv, Rec &recL,
                                       Rec &recR, double &last) {
    // each cell's band test and address are formed once, for its load and its store
    double *pa[5], *pb[5];
    bool ia[5], ib[5];  // the cell is stored (inside the band)
    double x[5], y[5];
    const bool extra = (src != 0) || withv;
#pragma unroll
    for (int q = 0; q < 5; q++) {
      const bool in = q < w;
      const int i0 = isrows ? a : lo + q, j0 = isrows ? lo + q : a;
      const int i1 = isrows ? a + 1 : lo + q, j1 = isrows ? lo + q : a + 1;
      ia[q] = in && inband(i0, j0);
      ib[q] = in && inband(i1, j1);
      pa[q] = ia[q] ? S.cell(i0, j0) : zero;
      pb[q] = ib[q] ? S.cell(i1, j1) : zero;
    }
    if (extra) {
      if (src == 1) { pa[4] = S.uptr(a); pb[4] = S.uptr(a + 1); }
      else if (src == 2) { pa[4] = S.cell(1, a); pb[4] = S.cell(1, a + 1); }
      else { pa[4] = S.vptr(a); pb[4] = S.vptr(a + 1); }
      ia[4] = ib[4] = true;
    }
#pragma unroll
    for (int q = 0; q < 5; q++) {
      x[q] = ia[q] ? Store::load(pa[q]) : 0.0;
      y[q] = ib[q] ? Store::load(pb[q]) : 0.0;
    }
    const double f = src == 0 ? x[0] : x[4], g = src == 0 ? y[0] : y[4];
    double c, s, r;
    if (!A::rot(f, g, c, s, r)) return false;
#pragma unroll
    for (int q = 0; q < 5; q++) {
      const double nx = A::px(c, s, x[q], y[q]), ny = A::py(c, s, x[q], y[q]);
      x[q] = nx; y[q] = ny;
    }
    if (src == 0) { x[0] = r; y[0] = 0.0; }
    else { x[4] = r; y[4] = 0.0; }
    // a value that lands outside the band must be zero (reported otherwise)
    bool outside = false;
#pragma unroll
    for (int q = 0; q < 5; q++) {
      if (ia[q]) *pa[q] = x[q];
      else outside |= nz(x[q]);
      if (ib[q]) *pb[q] = y[q];
      else outside |= nz(y[q]);
    }
    if (outside) atomicOr(err, ERR_BAND);
    if (isrows) {
      rotate_extra(Ux, m, a, c, s);
      recL.push(c, s, a);
    } else {
      rotate_extra(Vx, n, a, c, s);
      recR.push(c, s, a);
    }
    last = w == 3 ? x[2] : (w == 4 ? x[3] : x[4]);
    return true;
  }

  // exec for an op of kind ST away from row 1 (rows a, a+1 >= 2 for a row
  // op, lo >= 2 for a column op) whose rotated pair lies inside the matrix:
  // the same arithmetic on the same values as exec, with the geometry fixed
  // at compile time.  Cell addresses are a base row plus constant diagonal
  // offsets; a cell is read and written only inside the matrix (column
  // lo + q <= n for a row op, row lo + q <= N for a column op), since both
  // cells of a pair lie on the same side of that bound; pairs whose results
  // are replaced by (r, 0) are not rotated.
  template <int ST>
  __device__ __forceinline__ bool exec_st(int a, int lo, Rec &recL, Rec &recR, double &last) {
    constexpr Geo G = geo_of(ST);
    constexpr int W = G.w;
    constexpr bool EXTRA = G.src != 0 || G.withv;
    const int lim = (G.rows ? n : N) - lo;  // cell q is inside iff q <= lim
    double *const base = S.dg0 + (G.rows ? a : lo);
    const size_t ld = (size_t)S.ld;
    double *pa[W], *pb[W];
    double x[W], y[W];
#pragma unroll
    for (int q = 0; q < W; q++) {
      const int oa = G.rows ? G.c + q : G.c - q;
      const int ob = G.rows ? oa - 1 : oa + 1;
      pa[q] = base + oa * ld + (G.rows ? 0 : q);
      pb[q] = base + ob * ld + (G.rows ? 1 : q);
    }
    double *pe = nullptr;
    double xe = 0.0, ye = 0.0;
    if (EXTRA) pe = G.src == 1 ? S.uptr(a) : (G.src == 2 ? S.cell(1, a) : S.vptr(a));
#pragma unroll
    for (int q = 0; q < W; q++) {
      const bool in = q <= lim;
      x[q] = in ? Store::load(pa[q]) : 0.0;
      y[q] = in ? Store::load(pb[q]) : 0.0;
    }
    if (EXTRA) { xe = Store::load(pe); ye = Store::load(pe + 1); }
    const double f = G.src == 0 ? x[0] : xe, g = G.src == 0 ? y[0] : ye;
    double c, s, r;
    if (!A::rot(f, g, c, s, r)) return false;
#pragma unroll
    for (int q = (G.src == 0 ? 1 : 0); q < W; q++) {
      const double nx = A::px(c, s, x[q], y[q]), ny = A::py(c, s, x[q], y[q]);
      x[q] = nx; y[q] = ny;
    }
    if (G.src == 0) { x[0] = r; y[0] = 0.0; }
    if (G.withv) {
      const double nx = A::px(c, s, xe, ye), ny = A::py(c, s, xe, ye);
      xe = nx; ye = ny;
    } else if (G.src != 0) {
      xe = r; ye = 0.0;
    }
#pragma unroll
    for (int q = 0; q < W; q++) {
      if (q <= lim) { *pa[q] = x[q]; *pb[q] = y[q]; }
    }
    if (EXTRA) { pe[0] = xe; pe[1] = ye; }
    if (G.rows) {
      rotate_extra(Ux, m, a, c, s);
      recL.push(c, s, a);
    } else {
      rotate_extra(Vx, n, a, c, s);
      recR.push(c, s, a);
    }
    last = x[W - 1];
    return true;
  }

  __device__ __forceinline__ void chase_start(Task &k, int kk, double bulge) {
    k.ii = kk;
    if (kk + 2 <= N && nz(bulge)) {
      k.st = S_CL;
      k.pos = kk + 1;
    } else {
      k.done = true;
    }
  }

  // Geometry of the next op of task k (integer logic): the pair (a, a+1) it
  // rotates, its first row or column lo, width w, source and whether v
  // rotates too; doit is false when the op does not exist (the state then
  // only advances).
  __device__ __forceinline__ void op_geometry(const Task &k, bool &isrows, int &a, int &lo, int &w, int &src,
                                              bool &withv, bool &doit) const {
    isrows = false; withv = false; doit = true;
    a = 0; lo = 0; w = 4; src = 0;
    switch (k.st) {
      case S_L0: isrows = true; a = k.p - 1; lo = a; w = 3; src = 1; break;                    // left (j-1, j) on u
      case S_R1: a = k.ii + 1; lo = k.ii; w = 4; withv = true; break;                            // right (i+1, i+2)
      case S_L1: isrows = true; a = k.ii + 2; lo = k.ii + 1; w = 4; break;                       // left (i+2, i+3)
      case S_P2: a = k.p - 1; if (a - 1 == 1) { lo = 1; } else { lo = a - 1; src = 2; } w = 4; break;  // right (j-1, j), row 1
      case S_A: isrows = true; a = k.p; lo = a; w = 4; doit = (k.p + 1 <= N); break;             // left (i, i+1)
      case S_B: a = k.p + 2; lo = k.p; w = 5; break;                                             // right (i+2, i+3)
      case S_C: a = k.p + 1; lo = k.p; w = 4; doit = (k.p + 2 <= n); break;                      // right (i+1, i+2)
      case S_CL: isrows = true; a = k.ii + 1; lo = k.ii; w = 5; break;                           // left (k+1, k+2)
      case S_CR: a = k.ii + 3; lo = k.ii + 1; w = 5; break;                                      // right (k+3, k+4)
    }
  }

  // Runs one op of task k: the geometry of its next rotation (integer logic),
  // the rotation itself, then the chase's next state.  Left rotations go to
  // recL, right ones to recR.
  __device__ __forceinline__ void run_op(Task &k, Rec &recL, Rec &recR, int &nl, int &nr) {
    bool isrows, withv, doit;
    int a, lo, w, src;
    op_geometry(k, isrows, a, lo, w, src, withv, doit);
    double b = 0.0;
    bool ok = false;
    if (doit) {
      const bool interior = isrows ? (a >= 2 && a + 1 <= N) : (lo >= 2 && a + 1 <= n);
      if (!interior) {
        ok = exec(isrows, a, lo, w, src, withv, recL, recR, b);
      } else {
        switch (k.st) {
          case S_L0: ok = exec_st<S_L0>(a, lo, recL, recR, b); break;
          case S_R1: ok = exec_st<S_R1>(a, lo, recL, recR, b); break;
          case S_L1: ok = exec_st<S_L1>(a, lo, recL, recR, b); break;
          case S_P2: ok = exec_st<S_P2>(a, lo, recL, recR, b); break;
          case S_A: ok = exec_st<S_A>(a, lo, recL, recR, b); break;
          case S_B: ok = exec_st<S_B>(a, lo, recL, recR, b); break;
          case S_C: ok = exec_st<S_C>(a, lo, recL, recR, b); break;
          case S_CL: ok = exec_st<S_CL>(a, lo, recL, recR, b); break;
          default: ok = exec_st<S_CR>(a, lo, recL, recR, b); break;
        }
      }
    }
    // Keeps the band loads of the advance step (the next bulge) from being
    // scheduled into the rotation above (measured: ~15% of the step time).
    asm volatile("" ::: "memory");
    if (ok) { if (isrows) nl++; else nr++; }
    advance(k, ok, b);
  }

  // The chase's next state after an op that rotated (ok) and left the bulge b.
  __device__ __forceinline__ void advance(Task &k, bool ok, double b) {
    switch (k.st) {
      case S_L0: {
        const int i = k.p - 1;
        k.ii = i; k.st = S_R1;
        if (!ok || !(i + 2 <= n && nz(b))) { k.done = true; return; }
        k.pos = i + 1;
        return;
      }
      case S_R1: {
        int i = k.ii;
        if (!ok) { atomicOr(err, ERR_SCHEDULE); k.done = true; return; }
        if (i + 3 <= N && nz(b)) { k.st = S_L1; k.pos = i + 2; return; }
        i += 2; k.ii = i;
        if (!(i + 2 <= n && nz(get(i, i + 2)))) { k.done = true; return; }
        k.pos = i + 1;
        return;
      }
      case S_L1: {
        if (!ok) { atomicOr(err, ERR_SCHEDULE); k.done = true; return; }
        const int i = k.ii + 2;
        k.ii = i; k.st = S_R1;
        if (!(i + 2 <= n && nz(b))) { k.done = true; return; }
        k.pos = i + 1;
        return;
      }
      case S_P2: chase_start(k, k.p - 1, ok ? b : 0.0); return;
      case S_A:
        k.st = S_B;
        if (k.p + 3 <= n) { k.pos = k.p + 2; return; }
        k.done = true;
        return;
      case S_B:
        if (!ok) { k.done = true; return; }
        chase_start(k, k.p + 2, b);
        return;
      case S_C:
        if (!ok) { k.done = true; return; }
        chase_start(k, k.p + 1, b);
        return;
      case S_CL: {
        const int kk = k.ii;
        if (!ok) { atomicOr(err, ERR_SCHEDULE); k.done = true; return; }
        if (kk + 4 <= n && nz(b)) { k.st = S_CR; k.pos = kk + 3; return; }
        chase_start(k, kk + 3, get(kk + 5, kk + 3));
        return;
      }
      case S_CR:
        if (!ok) { atomicOr(err, ERR_SCHEDULE); k.done = true; return; }
        chase_start(k, k.ii + 3, b);
        return;
    }
  }

  // Geometry of an interior op by state, for the plan: bit 0 rows, bits 1-3
  // w, bits 4-5 src, bit 6 withv, bit 7 a counts from ii (else p), bits 8-10
  // a's offset + 1, bits 11-12 lo's distance below a, bits 13-14 the op's
  // existence test (1: p + 1 <= N, 2: p + 2 <= n).  The same values as
  // op_geometry (which the general path keeps).
  static __device__ __forceinline__ unsigned geo_word(int st) {
    switch (st) {  // (the compiler turns the constant table into selects)
      case S_L0: return 1u | 3u << 1 | 1u << 4 | 0u << 8 | 0u << 11;
      case S_R1: return 0u | 4u << 1 | 1u << 6 | 1u << 7 | 2u << 8 | 1u << 11;
      case S_L1: return 1u | 4u << 1 | 1u << 7 | 3u << 8 | 1u << 11;
      case S_A: return 1u | 4u << 1 | 1u << 8 | 0u << 11 | 1u << 13;
      case S_B: return 0u | 5u << 1 | 3u << 8 | 2u << 11;
      case S_C: return 0u | 4u << 1 | 2u << 8 | 1u << 11 | 2u << 13;
      case S_CL: return 1u | 5u << 1 | 1u << 7 | 2u << 8 | 1u << 11;
      case S_CR: return 0u | 5u << 1 | 1u << 7 | 4u << 8 | 2u << 11;
      default: return 0u | 4u << 1 | 2u << 4 | 0u << 8 | 1u << 11;  // S_P2
    }
  }

  // ---- one instruction sequence for the interior ops of every kind
  //
  // An interior op (the exec_st cases) is the pair (f, g) that defines the
  // rotation plus three or four pairs rotated with it: the band pairs after
  // the first when the first is the source, all w band pairs otherwise, then
  // v(a), v(a+1) when v rotates.  The plan holds their addresses (the
  // store's cell handles), so that the lanes of a warp whose chases are in
  // different states run one sequence of FP64 instructions (which on GB300
  // cost the same for 1 or 32 lanes) instead of one per state.  Same
  // operations on the same values as exec_st.
  enum : unsigned char { kNoOp = 0, kUniform = 1, kGeneric = 2 };
  using H = typename Store::H;
  struct Plan {
    H xs, ys;        // the pair (f, g); becomes (r, 0)
    H xo[4], yo[4];  // the rotated pairs
    int a, lo, w, src;
    unsigned char kind, nrot, inmask;  // inmask bit q: rotated pair q lies inside the matrix
    bool rows, withv;
  };
  __device__ __forceinline__ void make_plan(const Task &k, Plan &P) const {
    P.kind = kNoOp;
    P.nrot = 0;
    P.inmask = 0;
    if (k.done) return;
    const unsigned gw = geo_word(k.st);
    const unsigned chk = (gw >> 13) & 3;
    if ((chk == 1 && k.p + 1 > N) || (chk == 2 && k.p + 2 > n)) return;  // the op does not exist
    P.rows = gw & 1;
    P.w = (gw >> 1) & 7;
    P.src = (gw >> 4) & 3;
    P.withv = (gw >> 6) & 1;
    P.a = ((gw >> 7) & 1 ? k.ii : k.p) + (int)((gw >> 8) & 7) - 1;
    P.lo = P.a - (int)((gw >> 11) & 3);
    const int a = P.a, lo = P.lo;
    if (!(P.rows ? (a >= 2 && a + 1 <= N) : (lo >= 2 && a + 1 <= n))) {
      bool doit;
      op_geometry(k, P.rows, P.a, P.lo, P.w, P.src, P.withv, doit);  // the general path's exact geometry
      P.kind = kGeneric;
      return;
    }
    P.kind = kUniform;
    // band pair q: rows (a, a+1) at column lo+q, diagonals c+q and c+q-1; or
    // columns (a, a+1) at row lo+q, diagonals c-q and c-q+1 (geo_of(st).c)
    const int c = P.rows ? lo - a + 2 : a - lo + 2;
    const int lim = (P.rows ? n : N) - lo;  // band pair q lies inside iff q <= lim
    const int q0 = P.src == 0 ? 1 : 0;
    const int nb = P.w - q0;
    if (P.src == 0) {
      P.xs = P.rows ? S.h_band(c, a) : S.h_band(c, lo);
      P.ys = P.rows ? S.h_band(c - 1, a + 1) : S.h_band(c + 1, lo);
    } else {
      P.xs = P.src == 1 ? S.h_u(a) : S.h_r1(a);
      P.ys = P.src == 1 ? S.h_u(a + 1) : S.h_r1(a + 1);
    }
    unsigned mask = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int qq = q0 + q;
      H xo = P.rows ? S.h_band(c + qq, a) : S.h_band(c - qq, lo + qq);
      H yo = P.rows ? S.h_band(c + qq - 1, a + 1) : S.h_band(c - qq + 1, lo + qq);
      bool in = q < nb && qq <= lim;
      if (P.withv && q == nb) { xo = S.h_v(a); yo = S.h_v(a + 1); in = true; }
      P.xo[q] = xo; P.yo[q] = yo;
      mask |= in ? (1u << q) : 0u;
    }
    P.inmask = (unsigned char)mask;
    P.nrot = (unsigned char)(nb + (P.withv ? 1 : 0));
  }
  // The loads of a uniform op (zeros for lanes without one), issued together.
  __device__ __forceinline__ void load_plan(const Plan &P, double &f, double &g, double (&x)[4], double (&y)[4]) const {
    const bool u = P.kind == kUniform;
    f = u ? S.ld_h(P.xs) : 0.0;
    g = u ? S.ld_h(P.ys) : 0.0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const bool in = u && ((P.inmask >> q) & 1);
      x[q] = in ? S.ld_h(P.xo[q]) : 0.0;
      y[q] = in ? S.ld_h(P.yo[q]) : 0.0;
    }
  }
  // Every lane of the warp calls this (the fourth pair is skipped when no
  // active lane has one); lanes with act store.  Returns act && rotated.
  __device__ __forceinline__ bool exec_uniform(const Plan &P, bool act, double f, double g, double (&x)[4],
                                               double (&y)[4], double &c, double &s, double &last) {
    f = act ? f : 0.0;
    g = act ? g : 0.0;
    double r;
    const bool ok = A::rot(f, g, c, s, r) && act;
#pragma unroll
    for (int q = 0; q < 3; q++) {
      const double nx = A::px(c, s, x[q], y[q]), ny = A::py(c, s, x[q], y[q]);
      x[q] = nx; y[q] = ny;
    }
    if (__any_sync(0xffffffffu, act && P.nrot == 4)) {
      const double nx = A::px(c, s, x[3], y[3]), ny = A::py(c, s, x[3], y[3]);
      x[3] = nx; y[3] = ny;
    }
    if (ok) {
      S.st_h(P.xs, r);
      S.st_h(P.ys, 0.0);
#pragma unroll
      for (int q = 0; q < 4; q++) {
        if ((P.inmask >> q) & 1) { S.st_h(P.xo[q], x[q]); S.st_h(P.yo[q], y[q]); }
      }
      if (rx) rotate_extra(P.rows ? Ux : Vx, P.rows ? m : n, P.a, c, s);
    }
    last = (P.nrot == 4 && !P.withv) ? x[3] : x[2];
    return ok;
  }
};

// Required lead of chase u over chase t (u < t) in positions.
__device__ __forceinline__ int lag(int ku, int kt, bool adjacent) {
  if (!adjacent) return 4;
  if (ku == P1 && kt == P1) return 3;
  if (ku == P2 && kt == P3B) return 2;
  return 4;
}
__device__ __forceinline__ int kind_of(int t, int p1, int p2) {
  if (t < p1) return P1;
  if (t < p1 + p2) return P2;
  return ((t - p1 - p2) & 1) ? P3C : P3B;
}

// Logical slot l (chases t with (t / CS) % S == l) lives on thread l: the
// running chases, a window of consecutive ids, stay packed in few warps.  On
// GB300 an SM's FP64 unit is shared by all its warps and each FP64 warp
// instruction holds it for about 16 cycles whatever the number of active
// lanes, so the cost of a step grows with the number of warps that have a
// running chase, not with the number of chases.
__device__ __forceinline__ int thread_slot(int th, int) { return th; }

// status word of a slot: x = task id held, y = pos << 2 | started << 1 | done
__device__ __forceinline__ int2 enc(const Task &k) {
  int pos = k.done ? 0 : (k.pos > (INT_MAX >> 3) ? (INT_MAX >> 3) : k.pos);
  return make_int2(k.t, (pos << 2) | (k.started ? 2 : 0) | (k.done ? 1 : 0));
}

// The spike (m > n): one sequential chain on u in global memory.
template <bool FAST>
__device__ void run_spike(const ChaseArgs &Ar, unsigned long long *cnt0) {
  using A = Arith<FAST>;
  const int m = Ar.m, n = Ar.n;
  int ns = 0;
  double *u = Ar.band.u;
  for (int j = m; j >= n + 2; j--) {
    double c, s, r;
    if (!A::rot(u[j - 1], u[j], c, s, r)) continue;
    u[j - 1] = r;
    u[j] = 0.0;
    for (int t = 0; t < Ar.rx; t++) {
      double *U = Ar.Ux + (size_t)t * m - 1;
      const double x = U[j - 1], y = U[j];
      U[j - 1] = A::px(c, s, x, y);
      U[j] = A::py(c, s, x, y);
    }
    Ar.st.Sc[ns] = c; Ar.st.Ss[ns] = s; Ar.st.Sa[ns] = j - 1;
    if (Ar.st.Sf) Ar.st.Sf[ns] = make_float2(f32_of(c), f32_of(s));
    ns++;
  }
  Ar.st.Sn[0] = ns;
  *cnt0 = ns;
}

__device__ __forceinline__ void bind_rec(const ChaseArgs &Ar, const Task &k, Rec &recL, Rec &recR) {
  const int cap = Ar.st.cap;
  if (k.t < Ar.st.T) {
    const size_t o = (size_t)k.t * cap;
    recL.a = Ar.st.La + o;
    recR.a = Ar.st.Ra + o;
    recL.c = Ar.st.Lc ? Ar.st.Lc + o : nullptr; recL.s = Ar.st.Ls ? Ar.st.Ls + o : nullptr;
    recR.c = Ar.st.Rc ? Ar.st.Rc + o : nullptr; recR.s = Ar.st.Rs ? Ar.st.Rs + o : nullptr;
    recL.f = Ar.st.Lf ? Ar.st.Lf + o : nullptr;
    recR.f = Ar.st.Rf ? Ar.st.Rf + o : nullptr;
    recL.cnt = recR.cnt = 0;
  }
}

// ----------------------------------------------------------------------------
// engine 1: one CTA
// ----------------------------------------------------------------------------
template <bool FAST>
__device__ __forceinline__ void engine_cta(const ChaseArgs &Ar, int use_smem) {
  extern __shared__ double sh[];
  __shared__ int2 st[2][kMaxThreads];
  __shared__ int front[3];
  __shared__ int p1done, ndone;
  __shared__ unsigned long long cnt[9];

  const int m = Ar.m, n = Ar.n, N = (m > n) ? n + 1 : n;
  const int S = blockDim.x, me = threadIdx.x;
  const int T = Ar.st.T;
  const int p1 = N - 1, p2 = n > 2 ? n - 2 : 0;

  if (me < 9) cnt[me] = 0;
  __syncthreads();
  if (me == 0) run_spike<FAST>(Ar, &cnt[0]);
  __syncthreads();

  __shared__ double zero_cell;
  if (me == 0) zero_cell = 0.0;
  Chaser<LocalStore, FAST> K;
  K.zero = &zero_cell;
  K.N = N; K.n = n; K.m = m; K.err = Ar.status;
  K.Ux = Ar.Ux; K.Vx = Ar.Vx; K.rx = Ar.rx;
  const int64_t nband = 6 * (int64_t)(N + 2) + 2 * (int64_t)(n + 2) + (N + 2);
  K.S.ld = N + 2;
  if (use_smem) {
    double *p = sh;
    K.S.dg0 = p; p += 6 * (N + 2);
    K.S.r1 = p; p += n + 2;
    K.S.v = p; p += n + 2;
    K.S.u = p;
    const double *src = Ar.band.dg[0];
    for (int64_t q = me; q < nband; q += S) sh[q] = src[q];
  } else {
    K.S.dg0 = Ar.band.dg[0];
    K.S.r1 = Ar.band.r1; K.S.v = Ar.band.v; K.S.u = Ar.band.u;
  }

  const int myslot = thread_slot(me, S);
  const int pslot = (myslot + S - 1) % S;  // slot of chase t-1 (t = myslot mod S)
  Task k;
  task_init(k, myslot, T, N, n);
  Rec recL, recR;
  recL.f = recR.f = nullptr;
  recL.cap = recR.cap = Ar.st.cap;
  recL.err = recR.err = Ar.status;
  int nl = 0, nr = 0;
  bind_rec(Ar, k, recL, recR);
  st[0][myslot] = enc(k);
  if (me == 0) {
    front[0] = 0; front[1] = INT_MAX; front[2] = INT_MAX;
    p1done = 0; ndone = 0;
  }
  bool fold_done = false;
  const long long max_steps = Ar.step_budget > 0 ? Ar.step_budget : 64LL * (n + 16) + 4096;
  long long step = 0;
  for (;; step++) {
    // Snapshot the shared counters between two barriers: during the step they
    // are incremented by threads that finish a chase.
    __syncthreads();
    const int p1d = p1done, nd = ndone;
    __syncthreads();
    if (!fold_done && p1d == p1) {
      const double u1 = *K.S.uptr(1);
      for (int j = me + 1; j <= n; j += S) K.S.r1[j] = Arith<FAST>::px(1.0, u1, K.S.r1[j], K.S.v[j]);
      __syncthreads();
      fold_done = true;
    }
    if (fold_done && nd == T) break;
    if (step >= max_steps) {
      if (me == 0) atomicOr(Ar.status, ERR_STEPS);
      break;
    }
    const int rd = step & 1, wr = rd ^ 1;
    const int f_rd = step % 3, f_wr = (step + 1) % 3, f_reset = (step + 2) % 3;
    if (me == 0) front[f_reset] = INT_MAX;
    const int fr = front[f_rd];
    if (!k.done) {
      const int t = k.t;
      bool ok = !(t >= p1 && !fold_done);
      int reach = INT_MAX;  // last position this chase may reach in this step
      if (ok) {
        const int lim = (t >= p1) ? p1 : 0;
        const int stop = fr > lim ? fr : lim;
        const int kt = kind_of(t, p1, p2);
        for (int u = t - 1; u >= stop; u--) {
          int2 w = st[rd][u == t - 1 ? pslot : u % S];
          if (w.x < u) { ok = false; break; }    // its slot still holds an older chase
          if (w.x > u || (w.y & 1)) continue;    // finished
          if (!(w.y & 2)) { ok = false; break; } // not started
          reach = (w.y >> 2) - lag(kind_of(u, p1, p2), kt, u == t - 1);
          break;
        }
      }
      // Keeps the op's band loads from being scheduled into the look-back
      // above (measured: about a quarter of the step time at n = 4096).
      asm volatile("" ::: "memory");
      for (int rep = 0; rep < kOpsPerStep && ok && k.pos <= reach; rep++) {
        K.run_op(k, recL, recR, nl, nr);
        k.started = true;
        if (k.done) {
          Ar.st.Ln[t] = nl;
          Ar.st.Rn[t] = nr;
          atomicAdd(&cnt[k.phase], (unsigned long long)nl);
          atomicAdd(&cnt[4 + k.phase], (unsigned long long)nr);
          if (t < p1) atomicAdd(&p1done, 1);
          atomicAdd(&ndone, 1);
          task_init(k, t + S, T, N, n);
          nl = nr = 0;
          bind_rec(Ar, k, recL, recR);
          break;
        }
      }
    }
    {
      const int mn = __reduce_min_sync(0xffffffffu, k.done ? INT_MAX : k.t);
      if ((me & 31) == 0 && mn != INT_MAX) atomicMin(&front[f_wr], mn);
    }
    st[wr][myslot] = enc(k);
  }
  __syncthreads();
  if (me == 0) {
    cnt[8] = step;
    for (int q = 0; q < 9; q++) atomicAdd(&Ar.counters[q], cnt[q]);
  }
  if (use_smem) {
    double *dst = Ar.band.dg[0];
    for (int64_t q = me; q < nband; q += S) dst[q] = sh[q];
  }
}

template <bool FAST>
__global__ void __launch_bounds__(kMaxThreads) k_chase(ChaseArgs Ar, int use_smem) {
  engine_cta<FAST>(Ar, use_smem);
}

// Many independent factorizations, one thread block each (the batched update
// of resident streams): block b runs the one-CTA engine on items[b]; an item
// whose band does not fit the launch's dynamic shared memory keeps it in
// global memory.
template <bool FAST>
__global__ void __launch_bounds__(kMaxThreads) k_chase_batch(const ChaseArgs *__restrict__ items,
                                                             size_t smem_bytes) {
  const ChaseArgs Ar = items[blockIdx.x];
  const int N = (Ar.m > Ar.n) ? Ar.n + 1 : Ar.n;
  const size_t need = sizeof(double) * (6 * (size_t)(N + 2) + 2 * (size_t)(Ar.n + 2) + (N + 2));
  engine_cta<FAST>(Ar, need <= smem_bytes ? 1 : 0);
}

// ----------------------------------------------------------------------------
// engine 2: a thread-block cluster
// ----------------------------------------------------------------------------
// The band stays in global memory (L2); chase t runs on CTA t % CS, logical
// slot (t / CS) % S.  Steps are separated by the cluster barrier, split into
// its arrive (release) and wait (acquire) halves:
//
//   wait      every band write and status word of the previous step is
//             visible cluster-wide;
//   loads     the status word of chase t-1 and the counters (shared memory)
//             are read first, then the planned op's band loads are issued at
//             once (speculatively: a lane whose chase may not run discards
//             them), so that the look-back overlaps their latency;
//   look-back may the chase run (lags behind the nearest earlier unfinished
//             chase, as in the one-CTA engine);
//   op        the rotation and its pairs, their stores, the chase's next
//             state;
//   publish   status words into this CTA's table and the next CTA's mirror
//             (chase t-1 always lives on the CTA before chase t's), each
//             warp's counters (chases done, phase-1 chases done, lowest
//             unfinished chase) into every CTA's inbox;
//   arrive    (release: waits for the band stores to be performed);
//   deferred  the rotation record, a finished chase's bookkeeping and the
//             next task, the plan (cell offsets) of the next op: nothing any
//             CTA reads before the next barrier.  (Measured at n = 4096: 146
//             ms per column against 158 with this work before the arrive.)
//
// Status words and inbox slots alternate with the step's parity: a slot
// written in step s is read in step s+1 and rewritten in step s+2 or later,
// after every reader of step s+1 has arrived.  So every CTA reads the same
// totals in a step and leaves the loop in the same step.  Totals are at least
// one step old, which is conservative.
__device__ __forceinline__ void cluster_arrive() {
  __syncwarp();
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  __syncwarp();
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
constexpr int kMaxWarps = kMaxThreads / 32;
// The cluster totals (chases done, phase-1 chases done, lowest unfinished
// chase) are exchanged every kTotalsEvery steps; between exchanges the last
// values stand, which only delays the fold and the exit by a few steps and
// makes the look-back scan a few finished chases more.
constexpr int kTotalsEvery = 8;

template <bool FAST>
__device__ __forceinline__ void engine_cluster(const ChaseArgs &Ar) {
  extern __shared__ double bslice[];     // this CTA's slice of the band (DsmStore)
  __shared__ int2 st[2][kMaxThreads];    // this CTA's chase status words
  __shared__ int2 pred[2][kMaxThreads];  // mirror of the previous CTA's status words
  __shared__ int4 inbox[2][kMaxCluster * kMaxWarps];  // every warp's counters (CTA-major): done, p1 done, min unfinished
  __shared__ unsigned long long cnt[9];

  cg::cluster_group cl = cg::this_cluster();
  constexpr int CS = kMaxCluster;  // the launch's cluster size; chase t runs on CTA t % CS
  const int cta = (int)cl.block_rank();
  const int m = Ar.m, n = Ar.n, N = (m > n) ? n + 1 : n;
  const int S = blockDim.x, me = threadIdx.x, lane = me & 31, wid = me >> 5;  // S: a power of two
  const int NW = S / 32;
  const int T = Ar.st.T;
  const int p1 = N - 1, p2 = n > 2 ? n - 2 : 0;
  const int next = (cta + 1) % CS;

  if (me < 9) cnt[me] = 0;
  __syncthreads();
  if (cta == 0 && me == 0) run_spike<FAST>(Ar, &cnt[0]);
  cl.sync();  // spike done (global u)

  using Ch = Chaser<DsmStore, FAST>;
  Ch K;
  K.zero = &g_zero_sink[0];
  static_assert(kMaxCluster == 16, "the slice layout takes index i to CTA i % 16, slot i / 16");
  const int B = dsm_slice(N);
  __shared__ uint32_t rbase[kMaxCluster];
  if (me < CS) {
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(bslice)), "r"(me));
    rbase[me] = r;
  }
  __syncthreads();
  K.S.loc = bslice; K.S.rb = rbase;
  K.S.B = B;
  K.N = N; K.n = n; K.m = m; K.err = Ar.status;
  // this CTA's slice of the nine arrays: indices cta * B .. cta * B + B - 1
  const double *gsrc[9] = {Ar.band.dg[0], Ar.band.dg[1], Ar.band.dg[2], Ar.band.dg[3], Ar.band.dg[4],
                           Ar.band.dg[5], Ar.band.r1, Ar.band.v, Ar.band.u};
  const int glen[9] = {N + 2, N + 2, N + 2, N + 2, N + 2, N + 2, n + 2, n + 2, N + 2};
  for (int arr = 0; arr < 9; arr++)
    for (int q = me; q < B; q += S) {
      const int idx = q * CS + cta;
      bslice[arr * B + q] = idx < glen[arr] ? __ldcg(gsrc[arr] + idx) : 0.0;
    }
  K.Ux = Ar.Ux; K.Vx = Ar.Vx; K.rx = Ar.rx;

  int2 *pred_next = cl.map_shared_rank(&pred[0][0], next);
  const int stride = CS * S;
  const int myslot = thread_slot(me, S);
  // this thread's chases are t = cta + CS * j with j = myslot (mod S); chase
  // t-1 sits on the previous CTA in slot j (or j-1 when cta = 0), which is
  // where that CTA pushes its status word in this CTA's mirror
  const int pslot = cta > 0 ? myslot : (myslot + S - 1) % S;
  Task k;
  task_init(k, cta + CS * myslot, T, N, n);
  Rec recL, recR;
  recL.f = recR.f = nullptr;
  recL.cap = recR.cap = Ar.st.cap;
  recL.err = recR.err = Ar.status;
  int nl = 0, nr = 0;
  bind_rec(Ar, k, recL, recR);
  st[0][myslot] = enc(k);
  pred_next[myslot] = enc(k);  // slot 0 of the next CTA's mirror
  int ndone = 0, np1 = 0;      // this thread's finished chases (all, phase 1)
  {
    const int mn = __reduce_min_sync(0xffffffffu, k.done ? INT_MAX : k.t);
    if (lane < CS) {
      int4 *ib = cl.map_shared_rank(&inbox[1][cta * NW + wid], lane);
      *ib = make_int4(0, 0, mn, 0);
    }
  }
  typename Ch::Plan P;
  K.make_plan(k, P);
  bool fold_done = false;
  int sd = 0, sp1 = 0, fr = 0;  // cluster totals, read every kTotalsEvery steps
  const long long max_steps = Ar.step_budget > 0 ? Ar.step_budget : 64LL * (n + 16) + 4096;
  long long step = 0;
  cluster_arrive();
  for (;; step++) {
    cluster_wait();  // every write of the previous step is visible cluster-wide
    const int rd = step & 1, wr = rd ^ 1;
    const bool totals = (step & (kTotalsEvery - 1)) == 0;
    const int2 wpred = pred[rd][pslot];  // chase t-1 (local mirror of the previous CTA)
    int4 iv[kMaxCluster * kMaxWarps / 32];
    if (totals) {
      // cluster totals at the end of the previous step (inbox slot wr)
#pragma unroll
      for (int q = 0; q < kMaxCluster * kMaxWarps / 32; q++) {
        const int e = lane + 32 * q;
        iv[q] = e < CS * NW ? inbox[wr][e] : make_int4(0, 0, INT_MAX, 0);
      }
    }
    double f, g, x[4], y[4];
    K.load_plan(P, f, g, x, y);
    if (totals) {
      int a0 = 0, a1 = 0, a2 = INT_MAX;
#pragma unroll
      for (int q = 0; q < kMaxCluster * kMaxWarps / 32; q++) {
        a0 += iv[q].x; a1 += iv[q].y; a2 = iv[q].z < a2 ? iv[q].z : a2;
      }
      sd = __reduce_add_sync(0xffffffffu, a0);
      sp1 = __reduce_add_sync(0xffffffffu, a1);
      fr = __reduce_min_sync(0xffffffffu, a2);
      if (fr == INT_MAX) fr = T;
      if (!fold_done && sp1 == p1) {
        // fold: row 1 += u(1) v^T, each CTA over the columns of its slice
        const double u1 = DsmStore::load(K.S.uptr(1));
        for (int q = me; q < B; q += S) {
          const int j = q * CS + cta;
          if (j >= 1 && j <= n) bslice[6 * B + q] = Arith<FAST>::px(1.0, u1, bslice[6 * B + q], bslice[7 * B + q]);
        }
        cl.sync();
        fold_done = true;
        K.load_plan(P, f, g, x, y);  // row 1 has changed
      }
      if (fold_done && sd == T) break;
    }
    if (step >= max_steps) {
      if (me == 0) atomicOr(Ar.status, ERR_STEPS);
      break;
    }
    bool run = false;
    const int t = k.t;
    if (!k.done) {
      bool ok = !(t >= p1 && !fold_done);
      int reach = INT_MAX;  // last position this chase may reach in this step
      if (ok) {
        const int lim = (t >= p1) ? p1 : 0;
        const int stop = fr > lim ? fr : lim;
        const int kt = kind_of(t, p1, p2);
        for (int u = t - 1; u >= stop; u--) {
          int2 w;
          if (u == t - 1) {
            w = wpred;
          } else {
            const int2 *su = cl.map_shared_rank(&st[0][0], u & (CS - 1));
            w = su[rd * kMaxThreads + ((u / CS) & (S - 1))];
          }
          if (w.x < u) { ok = false; break; }
          if (w.x > u || (w.y & 1)) continue;
          if (!(w.y & 2)) { ok = false; break; }
          reach = (w.y >> 2) - lag(kind_of(u, p1, p2), kt, u == t - 1);
          break;
        }
      }
      run = ok && k.pos <= reach;
    }
    // the op: one FP64 instruction sequence for the warp's interior ops, the
    // general form (ops touching row 1) apart
    bool rot = false, pend = false;
    double c = 0.0, sn = 0.0, b = 0.0;
    if (__any_sync(0xffffffffu, run && P.kind == Ch::kUniform)) {
      rot = K.exec_uniform(P, run && P.kind == Ch::kUniform, f, g, x, y, c, sn, b);
      pend = rot;
    }
    if (run && P.kind == Ch::kGeneric) rot = K.exec(P.rows, P.a, P.lo, P.w, P.src, P.withv, recL, recR, b);
    bool fin = false;
    if (run) {
      if (rot) { if (P.rows) nl++; else nr++; }
      K.advance(k, rot, b);
      k.started = true;
      if (k.done) {
        fin = true;
        ndone++;
        if (t < p1) np1++;
      }
    }
    // publish
    const int2 sw = enc(k);  // a finished chase reads as finished
    st[wr][myslot] = sw;
    pred_next[wr * kMaxThreads + myslot] = sw;  // push to the next CTA's mirror
    if (((step + 1) & (kTotalsEvery - 1)) == 0) {  // read in the next step
      const int wd = __reduce_add_sync(0xffffffffu, ndone);
      const int wp = __reduce_add_sync(0xffffffffu, np1);
      // lowest unfinished chase of the warp (a finished chase's slot moves on
      // to chase t + stride)
      const int wm = __reduce_min_sync(0xffffffffu, !k.done ? k.t : (fin && t + stride < T ? t + stride : INT_MAX));
      if (lane < CS) {
        int4 *ib = cl.map_shared_rank(&inbox[rd][cta * NW + wid], lane);
        *ib = make_int4(wd, wp, wm, 0);
      }
    }
    cluster_arrive();
    // deferred
    if (pend) (P.rows ? recL : recR).push(c, sn, P.a);
    if (fin) {
      Ar.st.Ln[t] = nl;
      Ar.st.Rn[t] = nr;
      atomicAdd(&cnt[k.phase], (unsigned long long)nl);
      atomicAdd(&cnt[4 + k.phase], (unsigned long long)nr);
      task_init(k, t + stride, T, N, n);  // the slot moves on: chase t reads as finished
      nl = nr = 0;
      bind_rec(Ar, k, recL, recR);
    }
    K.make_plan(k, P);
  }
  if (me == 0) {
    if (cta == 0) cnt[8] = step;
  }
  cl.sync();  // every CTA has left the loop; the slices and phase counters are final
  {
    double *gdst[9] = {Ar.band.dg[0], Ar.band.dg[1], Ar.band.dg[2], Ar.band.dg[3], Ar.band.dg[4],
                       Ar.band.dg[5], Ar.band.r1, Ar.band.v, Ar.band.u};
    for (int arr = 0; arr < 9; arr++)
      for (int q = me; q < B; q += S) {
        const int idx = q * CS + cta;
        if (idx < glen[arr]) gdst[arr][idx] = bslice[arr * B + q];
      }
  }
  if (me == 0) {
    for (int q = 0; q < 9; q++)
      if (cnt[q]) atomicAdd(&Ar.counters[q], cnt[q]);
  }
}

template <bool FAST>
__global__ void __launch_bounds__(kMaxThreads) k_chase_cluster(ChaseArgs Ar) {
  engine_cluster<FAST>(Ar);
}

// Many independent factorizations, one 16-CTA cluster each (the large items
// of a batched update): cluster c runs the cluster engine on items[c].
template <bool FAST>
__global__ void __launch_bounds__(kMaxThreads) k_chase_cluster_batch(const ChaseArgs *__restrict__ items) {
  const ChaseArgs Ar = items[blockIdx.x / kMaxCluster];
  engine_cluster<FAST>(Ar);
}

// Static shared memory of the cluster engine (status words, mirrors, inbox)
// with some margin, and its dynamic shared memory: the band slice of each CTA.
constexpr size_t kClusterStaticSmem = 16384;
size_t cluster_slice_bytes(int n, int m) {
  const int N = (m > n) ? n + 1 : n;
  return (size_t)9 * sizeof(double) * dsm_slice(N);
}

// Threads per CTA of the cluster engine: a slot for each of the ~n/3 chases in
// flight, a power of two (64..kMaxThreads) so that slot arithmetic is shifts.
int cluster_threads(int n) {
  const int need = (n / 3 + 16) / kMaxCluster;
  int t = 64;
  while (t < need && t < kMaxThreads) t *= 2;
  return t;
}

template <bool FAST>
cudaError_t launch_engine(const ChaseArgs &a, cudaStream_t s) {
  const int n = a.n, m = a.m;
  const int N = (m > n) ? n + 1 : n;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // by size: one CTA up to the measured crossover (n = 512: 17.2 vs 20.0 ms
  // per mixed column, 26.2 vs 28.0 FP64; n = 1024: 42.9 vs 40.9, 69.4 vs 56.9)
  const int cluster_from = FAST ? 896 : 640;
  // the cluster engine holds the band in its CTAs' shared memory (about
  // 9 (n + 2) / 16 doubles each: n < 48000)
  const bool fits = cluster_slice_bytes(n, m) + kClusterStaticSmem <= (size_t)optin;
  if (fits && a.engine != 1 && (a.engine == 2 || n >= cluster_from)) {
    // cluster engine
    const int CS = kMaxCluster;
    const int threads = cluster_threads(n);
    cudaError_t e = cudaFuncSetAttribute(k_chase_cluster<FAST>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    const size_t dyn = cluster_slice_bytes(n, m);
    e = cudaFuncSetAttribute(k_chase_cluster<FAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_chase_cluster<FAST>, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  int threads = ((n / 3 + 16 + 31) / 32) * 32;
  if (threads < 32) threads = 32;
  if (threads > kMaxThreads) threads = kMaxThreads;
  const size_t smem = sizeof(double) * (6 * (size_t)(N + 2) + 2 * (size_t)(n + 2) + (N + 2));
  const size_t static_smem = sizeof(int2) * 2 * kMaxThreads + 64 + 9 * 8;
  const int use_smem = (smem + static_smem + 1024 <= (size_t)optin) ? 1 : 0;
  const size_t dyn = use_smem ? smem : 0;
  if (use_smem) {
    cudaError_t e = cudaFuncSetAttribute(k_chase<FAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  k_chase<FAST><<<1, threads, dyn, s>>>(a, use_smem);
  return cudaGetLastError();
}

}  // namespace

// The items one thread-block cluster each; the block size suits the largest n.
cudaError_t launch_chase_cluster_batch(const ChaseArgs *d_items, int count, int max_n, int fast,
                                       cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int CS = kMaxCluster;
  const int threads = cluster_threads(max_n);
  const size_t dyn = cluster_slice_bytes(max_n, max_n + 1);  // N <= max_n + 1
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS * count);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e;
  if (fast) {
    e = cudaFuncSetAttribute(k_chase_cluster_batch<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_chase_cluster_batch<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k_chase_cluster_batch<true>, d_items);
  } else {
    e = cudaFuncSetAttribute(k_chase_cluster_batch<false>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_chase_cluster_batch<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k_chase_cluster_batch<false>, d_items);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_chase_batch(const ChaseArgs *d_items, int count, int max_n, int max_band_doubles,
                               int fast, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int threads = ((max_n / 3 + 16 + 31) / 32) * 32;
  if (threads < 32) threads = 32;
  if (threads > kMaxThreads) threads = kMaxThreads;
  const size_t static_smem = sizeof(int2) * 2 * kMaxThreads + 256;
  size_t dyn = sizeof(double) * (size_t)max_band_doubles;
  if (dyn + static_smem > (size_t)optin) dyn = (size_t)optin - static_smem;
  cudaError_t e;
  if (fast) {
    e = cudaFuncSetAttribute(k_chase_batch<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    k_chase_batch<true><<<count, threads, dyn, s>>>(d_items, dyn);
  } else {
    e = cudaFuncSetAttribute(k_chase_batch<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    k_chase_batch<false><<<count, threads, dyn, s>>>(d_items, dyn);
  }
  return cudaGetLastError();
}

bool chase_cluster_fits(int m, int n) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return cluster_slice_bytes(n, m) + kClusterStaticSmem <= (size_t)optin;
}

// Failure injection (BDU_INJECT_STEP_BUDGET) sets the step budget of a
// column whose caller set none.
cudaError_t launch_chase(const ChaseArgs &a0, cudaStream_t s) {
  ChaseArgs a = a0;
  const Injection inj = injection();
  if (a.step_budget == 0 && inj.site == BDU_INJECT_STEP_BUDGET) a.step_budget = inj.value;
  return a.fast ? launch_engine<true>(a, s) : launch_engine<false>(a, s);
}

}  // namespace bdu

