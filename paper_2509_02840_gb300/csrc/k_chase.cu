// K2: rotation generation and bulge chasing for one rank-1 column
// (Sec. 3.4, Algorithm 2), in FP64.
//
// The reduction of the core M = Bd + u v^T is a sequence of "chases": each
// starts with one rotation and pushes the bulge it creates down the band.
// Chases are generated in a fixed order (the schedule below) and every chase
// moves monotonically down the band, so chase t may run concurrently with
// chase t-1 as long as it stays a few positions behind it.  The engine
// assigns one chase per thread and advances all runnable chases by one
// rotation per synchronous step; a chase runs only when the nearest earlier
// unfinished chase is at least D positions ahead (D = 3 between phase-1
// chases, 4 otherwise).  This keeps every band cell's read/write order
// identical to the sequential algorithm, so the result is bit-identical to a
// one-rotation-at-a-time execution.
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
// Arithmetic: every multiply, add, divide and square root is a separately
// rounded IEEE operation (__dmul_rn, __dadd_rn, __ddiv_rn, __dsqrt_rn), never
// a fused multiply-add, so each value is fully determined by its inputs.
#include <climits>
#include <cstdio>

#include "bdu_internal.cuh"

namespace bdu {
namespace {

constexpr int kMaxThreads = 1024;

enum Kind : int { P1 = 0, P2 = 1, P3B = 2, P3C = 3 };
// states
enum : int { S_L0 = 0, S_R1 = 1, S_L1 = 2, S_A = 3, S_B = 4, S_C = 5, S_CL = 6, S_CR = 7, S_P2 = 8 };

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }

// Rotation generator (Eqs. giv, giv1, zero handling of Sec. 3.4):
// [c s; -s c][f; g] = [r; 0].  Returns false when g == 0 (no rotation).
// r = sign(f) hypot(f, g), evaluated with power-of-two safe scaling.
__device__ __forceinline__ bool rotg(double f, double g, double &c, double &s, double &r) {
  if (g == 0.0) return false;
  if (f == 0.0) {
    c = 0.0; s = 1.0; r = g;
    return true;
  }
  double af = fabs(f), ag = fabs(g);
  double amax = af > ag ? af : ag;
  double sigma = 1.0;
  if (amax > 0x1p500) sigma = 0x1p-600;
  else if (amax < 0x1p-500) sigma = 0x1p600;
  double fs = mul(f, sigma), gs = mul(g, sigma);
  double h = __dsqrt_rn(add(mul(fs, fs), mul(gs, gs)));
  double rs = copysign(h, f);
  c = __ddiv_rn(fs, rs);
  s = __ddiv_rn(gs, rs);
  r = __ddiv_rn(rs, sigma);
  return true;
}

struct Core {
  double *dg[6];
  double *r1, *u, *v;
  int N, n;
  int *err;
  double *Ux, *Vx;
  int rx, m;

  __device__ __forceinline__ bool inband(int i, int j) const {
    if (i < 1 || i > N || j < 1 || j > n) return false;
    if (i == 1) return true;
    int o = j - i;
    return o >= -2 && o <= 3;
  }
  __device__ __forceinline__ double get(int i, int j) const {
    if (!inband(i, j)) return 0.0;
    return (i == 1) ? r1[j] : dg[j - i + 2][i];
  }
  __device__ __forceinline__ void put(int i, int j, double x) {
    if (!inband(i, j)) {
      if (x != 0.0) atomicOr(err, ERR_BAND);
      return;
    }
    if (i == 1) r1[j] = x;
    else dg[j - i + 2][i] = x;
  }
};

struct Rec {
  double *c, *s;
  int32_t *a;
  int cnt, cap;
  int *err;
  __device__ __forceinline__ void push(double cc, double ss, int aa) {
    if (cnt < cap) {
      c[cnt] = cc; s[cnt] = ss; a[cnt] = aa;
    } else {
      atomicOr(err, ERR_CAP);
    }
    cnt++;
  }
};

// Left rotation on rows (a, a+1) over columns [jlo, jhi]; the eliminated entry
// is (a+1, ec) and the pivot (a, ec).  ec == 0: the eliminated entry is u(a+1)
// and the pivot u(a) (start of a phase-1 chase).
__device__ __forceinline__ void rows_op(Core &K, Rec &rec, int a, double c, double s, double r,
                                        int jlo, int jhi, int ec) {
  if (jlo < 1) jlo = 1;
  if (jhi > K.n) jhi = K.n;
  for (int j = jlo; j <= jhi; j++) {
    double x = K.get(a, j), y = K.get(a + 1, j);
    K.put(a, j, add(mul(c, x), mul(s, y)));
    K.put(a + 1, j, add(mul(-s, x), mul(c, y)));
  }
  if (ec > 0) {
    K.put(a, ec, r);
    K.put(a + 1, ec, 0.0);
  } else {
    K.u[a] = r;
    K.u[a + 1] = 0.0;
  }
  for (int t = 0; t < K.rx; t++) {
    double *U = K.Ux + (size_t)t * K.m - 1;
    double x = U[a], y = U[a + 1];
    U[a] = add(mul(c, x), mul(s, y));
    U[a + 1] = add(mul(-s, x), mul(c, y));
  }
  rec.push(c, s, a);
}

// Right rotation on columns (a, a+1) over rows [ilo, ihi] (and row 1 when
// with_row1); the eliminated entry is (er, a+1) and the pivot (er, a).
__device__ __forceinline__ void cols_op(Core &K, Rec &rec, int a, double c, double s, double r,
                                        int ilo, int ihi, int er, bool with_row1, bool rot_v) {
  if (ilo < 1) ilo = 1;
  if (ihi > K.N) ihi = K.N;
  if (with_row1 && ilo > 1) {
    double x = K.get(1, a), y = K.get(1, a + 1);
    K.put(1, a, add(mul(c, x), mul(s, y)));
    K.put(1, a + 1, add(mul(-s, x), mul(c, y)));
  }
  for (int i = ilo; i <= ihi; i++) {
    double x = K.get(i, a), y = K.get(i, a + 1);
    K.put(i, a, add(mul(c, x), mul(s, y)));
    K.put(i, a + 1, add(mul(-s, x), mul(c, y)));
  }
  K.put(er, a, r);
  K.put(er, a + 1, 0.0);
  if (rot_v) {
    double x = K.v[a], y = K.v[a + 1];
    K.v[a] = add(mul(c, x), mul(s, y));
    K.v[a + 1] = add(mul(-s, x), mul(c, y));
  }
  for (int t = 0; t < K.rx; t++) {
    double *V = K.Vx + (size_t)t * K.n - 1;
    double x = V[a], y = V[a + 1];
    V[a] = add(mul(c, x), mul(s, y));
    V[a + 1] = add(mul(-s, x), mul(c, y));
  }
  rec.push(c, s, a);
}

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

__device__ __forceinline__ void chase_start(Core &K, Task &k, int kk) {
  k.ii = kk;
  if (kk + 2 <= K.N && K.get(kk + 2, kk) != 0.0) {
    k.st = S_CL;
    k.pos = kk + 1;
  } else {
    k.done = true;
  }
}

// Runs one op of task k.  Left rotations go to recL, right ones to recR.
__device__ void run_op(Core &K, Task &k, Rec &recL, Rec &recR, int &nl, int &nr) {
  const int n = K.n, N = K.N;
  double c, s, r;
  switch (k.st) {
    case S_L0: {  // P1 start: left (j-1, j) zeroing u(j)
      int a = k.p - 1;
      if (!rotg(K.u[a], K.u[a + 1], c, s, r)) { k.done = true; return; }
      rows_op(K, recL, a, c, s, r, a, a + 2, 0); nl++;
      int i = k.p - 1;
      k.ii = i; k.st = S_R1;
      if (!(i + 2 <= n && K.get(i, i + 2) != 0.0)) { k.done = true; return; }
      k.pos = i + 1;
      return;
    }
    case S_R1: {  // P1: right (i+1, i+2) zeroing M(i, i+2)
      int i = k.ii, a = i + 1;
      if (!rotg(K.get(i, i + 1), K.get(i, i + 2), c, s, r)) { atomicOr(K.err, ERR_SCHEDULE); k.done = true; return; }
      cols_op(K, recR, a, c, s, r, a - 1, a + 2, i, false, true); nr++;
      if (i + 3 <= N && K.get(i + 3, i + 1) != 0.0) { k.st = S_L1; k.pos = i + 2; return; }
      i += 2; k.ii = i;
      if (!(i + 2 <= n && K.get(i, i + 2) != 0.0)) { k.done = true; return; }
      k.pos = i + 1;
      return;
    }
    case S_L1: {  // P1: left (i+2, i+3) zeroing M(i+3, i+1)
      int i = k.ii, a = i + 2;
      if (!rotg(K.get(i + 2, i + 1), K.get(i + 3, i + 1), c, s, r)) { atomicOr(K.err, ERR_SCHEDULE); k.done = true; return; }
      rows_op(K, recL, a, c, s, r, a - 1, a + 2, i + 1); nl++;
      i += 2; k.ii = i; k.st = S_R1;
      if (!(i + 2 <= n && K.get(i, i + 2) != 0.0)) { k.done = true; return; }
      k.pos = i + 1;
      return;
    }
    case S_P2: {  // P2: right (j-1, j) zeroing M(1, j)
      int j = k.p, a = j - 1;
      if (rotg(K.get(1, j - 1), K.get(1, j), c, s, r)) {
        cols_op(K, recR, a, c, s, r, a - 1, a + 2, 1, true, false); nr++;
      }
      chase_start(K, k, j - 1);
      return;
    }
    case S_A: {  // P3b (a): left (i, i+1) zeroing M(i+1, i)
      int i = k.p;
      k.st = S_B;
      if (i + 1 <= N && rotg(K.get(i, i), K.get(i + 1, i), c, s, r)) {
        rows_op(K, recL, i, c, s, r, i, i + 3, i); nl++;
      }
      if (i + 3 <= n) { k.pos = i + 2; return; }
      k.done = true;
      return;
    }
    case S_B: {  // P3b (b): right (i+2, i+3) zeroing M(i, i+3)
      int i = k.p;
      if (!rotg(K.get(i, i + 2), K.get(i, i + 3), c, s, r)) { k.done = true; return; }
      cols_op(K, recR, i + 2, c, s, r, i, i + 4, i, false, false); nr++;
      chase_start(K, k, i + 2);
      return;
    }
    case S_C: {  // P3c (c): right (i+1, i+2) zeroing M(i, i+2)
      int i = k.p;
      if (i + 2 > n) { k.done = true; return; }
      if (!rotg(K.get(i, i + 1), K.get(i, i + 2), c, s, r)) { k.done = true; return; }
      cols_op(K, recR, i + 1, c, s, r, i, i + 3, i, false, false); nr++;
      chase_start(K, k, i + 1);
      return;
    }
    case S_CL: {  // chase_lower: left (k+1, k+2) zeroing M(k+2, k)
      int kk = k.ii, a = kk + 1;
      if (!rotg(K.get(kk + 1, kk), K.get(kk + 2, kk), c, s, r)) { atomicOr(K.err, ERR_SCHEDULE); k.done = true; return; }
      rows_op(K, recL, a, c, s, r, a - 1, a + 3, kk); nl++;
      if (kk + 4 <= n && K.get(kk + 1, kk + 4) != 0.0) { k.st = S_CR; k.pos = kk + 3; return; }
      chase_start(K, k, kk + 3);
      return;
    }
    case S_CR: {  // chase_lower: right (k+3, k+4) zeroing M(k+1, k+4)
      int kk = k.ii, a = kk + 3;
      if (!rotg(K.get(kk + 1, kk + 3), K.get(kk + 1, kk + 4), c, s, r)) { atomicOr(K.err, ERR_SCHEDULE); k.done = true; return; }
      cols_op(K, recR, a, c, s, r, a - 2, a + 2, kk + 1, false, false); nr++;
      chase_start(K, k, kk + 3);
      return;
    }
  }
}

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

// status word of a slot: x = task id held, y = pos << 2 | started << 1 | done
__device__ __forceinline__ int2 enc(const Task &k) {
  int pos = k.done ? 0 : (k.pos > (INT_MAX >> 3) ? (INT_MAX >> 3) : k.pos);
  return make_int2(k.t, (pos << 2) | (k.started ? 2 : 0) | (k.done ? 1 : 0));
}

__global__ void __launch_bounds__(kMaxThreads) k_chase(ChaseArgs A, int use_smem) {
  extern __shared__ double sh[];
  __shared__ int2 st[2][kMaxThreads];
  __shared__ int front[3];
  __shared__ int p1done, ndone;
  __shared__ unsigned long long cnt[9];

  const int m = A.m, n = A.n, N = (m > n) ? n + 1 : n;
  const int S = blockDim.x, me = threadIdx.x;
  const int T = A.st.T, cap = A.st.cap;
  const int p1 = N - 1, p2 = n > 2 ? n - 2 : 0;

  if (me < 9) cnt[me] = 0;

  // ---- spike (m > n): one sequential chain on u in global memory ----------
  if (me == 0) {
    int ns = 0;
    double *u = A.band.u;
    for (int j = m; j >= n + 2; j--) {
      double c, s, r;
      if (!rotg(u[j - 1], u[j], c, s, r)) continue;
      u[j - 1] = r;
      u[j] = 0.0;
      for (int t = 0; t < A.rx; t++) {
        double *U = A.Ux + (size_t)t * m - 1;
        double x = U[j - 1], y = U[j];
        U[j - 1] = add(mul(c, x), mul(s, y));
        U[j] = add(mul(-s, x), mul(c, y));
      }
      A.st.Sc[ns] = c; A.st.Ss[ns] = s; A.st.Sa[ns] = j - 1;
      ns++;
    }
    A.st.Sn[0] = ns;
    cnt[0] = ns;
  }
  __syncthreads();

  // ---- working copy of the band: shared memory when it fits ---------------
  Core K;
  K.N = N; K.n = n; K.m = m; K.err = A.status;
  K.Ux = A.Ux; K.Vx = A.Vx; K.rx = A.rx;
  if (use_smem) {
    double *p = sh;
    for (int o = 0; o < 6; o++) { K.dg[o] = p; p += N + 2; }
    K.r1 = p; p += n + 2;
    K.v = p; p += n + 2;
    K.u = p;
    const int64_t cnt_band = 6 * (int64_t)(N + 2) + 2 * (int64_t)(n + 2) + (N + 2);
    const double *src = A.band.dg[0];
    for (int64_t q = me; q < cnt_band; q += S) sh[q] = src[q];
  } else {
    for (int o = 0; o < 6; o++) K.dg[o] = A.band.dg[o];
    K.r1 = A.band.r1; K.v = A.band.v; K.u = A.band.u;
  }

  // ---- engine ---------------------------------------------------------------
  Task k;
  task_init(k, me, T, N, n);
  Rec recL, recR;
  recL.cap = recR.cap = cap;
  recL.err = recR.err = A.status;
  int nl = 0, nr = 0;
  auto bind = [&]() {
    if (k.t < T) {
      recL.c = A.st.Lc + (size_t)k.t * cap; recL.s = A.st.Ls + (size_t)k.t * cap; recL.a = A.st.La + (size_t)k.t * cap;
      recR.c = A.st.Rc + (size_t)k.t * cap; recR.s = A.st.Rs + (size_t)k.t * cap; recR.a = A.st.Ra + (size_t)k.t * cap;
      recL.cnt = recR.cnt = 0;
      nl = nr = 0;
    }
  };
  bind();
  st[0][me] = enc(k);
  if (me == 0) {
    front[0] = 0; front[1] = INT_MAX; front[2] = INT_MAX;
    p1done = 0; ndone = 0;
  }
  bool fold_done = false;
  const long long max_steps = 64LL * (n + 16) + 4096;
  long long step = 0;
  for (;; step++) {
    // Snapshot the shared counters between two barriers: during the step they
    // are incremented by threads that finish a chase.
    __syncthreads();
    const int p1d = p1done, nd = ndone;
    __syncthreads();
    if (!fold_done && p1d == p1) {
      // fold: row 1 += u(1) v^T
      double u1 = K.u[1];
      for (int j = me + 1; j <= n; j += S) K.r1[j] = add(K.r1[j], mul(u1, K.v[j]));
      __syncthreads();
      fold_done = true;
    }
    if (fold_done && nd == T) break;
    if (step >= max_steps) {
      if (me == 0) atomicOr(A.status, ERR_STEPS);
      break;
    }
    const int rd = step & 1, wr = rd ^ 1;
    const int f_rd = step % 3, f_wr = (step + 1) % 3, f_reset = (step + 2) % 3;
    if (me == 0) front[f_reset] = INT_MAX;
    const int fr = front[f_rd];
    if (!k.done) {
      const int t = k.t;
      bool ok = true;
      if (t >= p1 && !fold_done) ok = false;
      if (ok) {
        const int lim = (t >= p1) ? p1 : 0;
        const int stop = fr > lim ? fr : lim;
        const int kt = kind_of(t, p1, p2);
        for (int u = t - 1; u >= stop; u--) {
          int2 w = st[rd][u % S];
          if (w.x < u) { ok = false; break; }   // its slot still holds an older chase
          if (w.x > u || (w.y & 1)) continue;   // finished
          if (!(w.y & 2)) { ok = false; break; } // not started
          ok = (w.y >> 2) >= k.pos + lag(kind_of(u, p1, p2), kt, u == t - 1);
          break;
        }
      }
      if (ok) {
        run_op(K, k, recL, recR, nl, nr);
        k.started = true;
        if (k.done) {
          A.st.Ln[t] = nl;
          A.st.Rn[t] = nr;
          atomicAdd(&cnt[k.phase], (unsigned long long)nl);
          atomicAdd(&cnt[4 + k.phase], (unsigned long long)nr);
          if (t < p1) atomicAdd(&p1done, 1);
          atomicAdd(&ndone, 1);
          task_init(k, t + S, T, N, n);
          bind();
        }
      }
    }
    if (!k.done) atomicMin(&front[f_wr], k.t);
    st[wr][me] = enc(k);
  }
  __syncthreads();
  if (me == 0) {
    cnt[8] = step;
    for (int q = 0; q < 9; q++) atomicAdd(&A.counters[q], cnt[q]);
  }
  if (use_smem) {
    const int64_t cnt_band = 6 * (int64_t)(N + 2) + 2 * (int64_t)(n + 2) + (N + 2);
    double *dst = A.band.dg[0];
    for (int64_t q = me; q < cnt_band; q += S) dst[q] = sh[q];
  }
}

}  // namespace

cudaError_t launch_chase(const ChaseArgs &a, cudaStream_t s) {
  const int n = a.n, m = a.m;
  const int N = (m > n) ? n + 1 : n;
  int threads = ((n / 3 + 16 + 31) / 32) * 32;
  if (threads < 32) threads = 32;
  if (threads > kMaxThreads) threads = kMaxThreads;
  const size_t smem = sizeof(double) * (6 * (size_t)(N + 2) + 2 * (size_t)(n + 2) + (N + 2));
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t static_smem = sizeof(int2) * 2 * kMaxThreads + 64 + 9 * 8;
  int use_smem = (smem + static_smem + 1024 <= (size_t)optin) ? 1 : 0;
  size_t dyn = use_smem ? smem : 0;
  if (use_smem) {
    cudaError_t e = cudaFuncSetAttribute(k_chase, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  k_chase<<<1, threads, dyn, s>>>(a, use_smem);
  return cudaGetLastError();
}

}  // namespace bdu
