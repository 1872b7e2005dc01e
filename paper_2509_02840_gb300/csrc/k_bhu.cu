// BHU, the bidiagonal Householder update (Sec. 3.3, Algorithm 1, Theorem 1),
// FP64, on the GPU.
//
// The m x n matrix A = B + U V^T (B upper bidiagonal, m >= n; U, V the rk <= 8
// projected columns of a rank-rk update, absorbed in one sweep) is
// bidiagonalized by Householder reflectors applied alternately from the left
// and the right, without forming A.  After j left and j right reflectors
//
//   Q_j = H_1 ... H_j = I - Y_j S_j Y_j^T,   P_j = I - W_j R'_j W_j^T,
//
// where Y_j, W_j hold the normalized reflector vectors (Eq. YW: y_k with zeros
// above row k, w_{k+1} with zeros in rows 1..k) and S_j = 2 T_j^{-1},
// R'_j = 2 R_j^{-1} are the inverses of the triangular matrices of Eq. TR
// (Eq. QP).  Keeping the inverses turns every solve with T or R into a
// product; they grow by one column per reflector:
//
//   S_{j+1} = [S_j, -2 S_j (Y_j^T y); 0, 2]     (Q_j H = I - [Y y] S_{j+1} [Y y]^T).
//
// Step j needs one column and one row of the transformed matrix (the products
// a_k = A_{k-1,k-1} e_k and a*_{k+1} of Algorithm 1); both come from the
// factored form Q^T (B + U V^T) P that Theorem 1 expands:
//
//   column j:  z = P_{j-1} e_j,  x = B z + U (V^T z),  a = Q_{j-1}^T x,
//   row j:     q = Q_j e_j,      r = B^T q + V (U^T q), a* = P_{j-1}^T r,
//
// each O((m + n) j) work in products with Y, W, S, R'.  The reflector of a
// (rows j..m) gives alpha_j and y_j, the reflector of a* (columns j+1..n)
// beta_j and w_{j+1}.  The readings are those of the oracle: row j (not j+1)
// defines the right reflector (Sec. 2.1), a left reflector for column n when
// m > n, and the last diagonal and superdiagonal entries read off without a
// reflector when m = n.
//
// One cooperative launch runs the whole loop; the blocks meet at a grid
// barrier (bounded waits) between the phases of a step, 16 at most per step.
// Column products: a column to one warp, or to a group of up to 16 warps of a
// block when there are few columns, lanes over rows in order, a fixed shuffle
// tree.  Row products: tiles of 512 rows x 64 columns, partial sums per
// column chunk, added in chunk order by the last block of each row group to
// finish, which also sums the group's share of the dot product or norm the next
// phase needs.  The new column of S (R') and the next product with it are one
// pass over the triangle with two right-hand sides:
//
//   Q_j e_j = e_j - Y_j S_j Y_j^T e_j,  S_j Y_j^T e_j = (S yr + eta S(:, j), 2 eta)
//
// with yr, eta the entries of row j of Y.  Every result is deterministic: no
// atomics on values, fixed summation orders.  Entries the structure makes zero
// (above y_j, in W's rows 1..j, below the diagonal of S, R') are skipped, and
// everything written inside the launch is read through L2 (ld.global.cg), since
// L1 is not coherent across SMs.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bdu_internal.cuh"

namespace bdu {
namespace {

constexpr int kCols = 64;  // columns per partial-sum chunk of a row product

// Structure of a stored matrix M (column-major): which entries are zero.
enum Shape : int {
  kFull = 0,
  kY = 1,   // M(r, c) = 0 for r < c   (reflector vectors y_c)
  kW = 2,   // M(r, c) = 0 for r <= c  (reflector vectors w_{c+1})
  kUT = 3,  // M(r, c) = 0 for r > c   (upper triangular S, R')
};

__device__ __forceinline__ int col_lo(int shape, int c, int r0) {
  const int lo = shape == kY ? c : (shape == kW ? c + 1 : 0);
  return lo > r0 ? lo : r0;
}
__device__ __forceinline__ int col_hi(int shape, int c, int R) {
  return (shape == kUT && c + 1 < R) ? c + 1 : R;
}

// The row tiles [ra, rb) x column chunk [ca, cb) that hold only structural zeros.
__device__ __forceinline__ bool tile_zero(int shape, int ra, int rb, int ca, int cb) {
  if (shape == kY) return rb <= ca;       // every r < c
  if (shape == kW) return rb <= ca + 1;   // every r <= c
  if (shape == kUT) return ra >= cb;      // every r > c
  return false;
}

// Deterministic block sum of v (every thread of the block calls it; the
// result is returned to every thread).
__device__ __forceinline__ double block_sum(double v, double *sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < nw; k++) s += sh[k];
  __syncthreads();
  return s;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

constexpr int kT = 512;           // threads of a block = rows of a row group
constexpr int kMaxRank = BDU_BHU_MAX_RANK;  // columns of U, V one sweep absorbs
constexpr int kBarSpin = 1 << 22;  // bound on the wait of one grid barrier

struct BhuArgs {
  int m, n, steps, nl, nr;
  int64_t ldl, ldr, ldp;
  const double *d, *e;
  const double *u, *v;  // U (m x rk, leading dimension ldu), V (n x rk, ldv)
  int rk;
  int64_t ldu, ldv, tps;  // tps: stride of the group partials of the rk dot products
  double *alpha, *beta, *Y, *W, *SL, *SR;
  double *z, *x, *a, *q, *ra, *as, *g, *hv, *p1, *gw, *hw, *sv, *part, *part2, *tp;
  unsigned *cnt, *bar;  // counters per row group (zero, left zero); the barrier's count and generation (zero)
  int *status;
  double rho;  // the symmetric variant's weight (k_tri_persist)
  int spin;   // bound on one barrier wait (polls)
  int stall;  // failure injection: block 0 leaves at once, so the others' first wait runs out
};

// Grid barrier (the blocks of a cooperative launch are co-resident): the last
// block to arrive resets the count and releases the next generation.  A wait
// that runs out sets ERR_BHU; every block stops at its next barrier once the
// bit is set, so the kernel ends in bounded time.  Returns false to stop.
__device__ bool grid_barrier(const BhuArgs &A, unsigned &gen) {
  __shared__ int s_stop;
  __syncthreads();
  if (threadIdx.x == 0) {
    int stop = 0;
    __threadfence();
    const unsigned arrived = atomicAdd(&A.bar[0], 1u);
    if (arrived == gridDim.x - 1) {
      A.bar[0] = 0;
      st_release_u32(&A.bar[1], gen + 1);
    } else {
      int it = 0;
      while (ld_acquire_u32(&A.bar[1]) == gen) {
        if (++it > A.spin) {
          atomicOr(A.status, ERR_BHU);
          stop = 1;
          break;
        }
        if ((it & 255) == 0 && (*(volatile int *)A.status & ERR_BHU)) {
          stop = 1;
          break;
        }
      }
    }
    // (the acquire load above orders this block's later reads after every
    // block's writes, which each fenced before arriving)
    if (*(volatile int *)A.status & ERR_BHU) stop = 1;
    s_stop = stop;
  }
  __syncthreads();
  gen++;
  return !s_stop;
}

__device__ __forceinline__ int groups_of(int rows) { return rows > 0 ? (rows + kT - 1) / kT : 0; }

// Sum of the row groups' partials, in group order (every thread, every block:
// the same value everywhere).
__device__ __forceinline__ double tp_sum(const double *tp, int groups) {
  double s = 0.0;
  int k = 0;
  for (; k + 7 < groups; k += 8) {  // eight loads in flight, added in order
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; q++) v[q] = __ldcg(tp + k + q);
#pragma unroll
    for (int q = 0; q < 8; q++) s += v[q];
  }
  for (; k < groups; k++) s += __ldcg(tp + k);
  return s;
}

// out[c] = sum_{r in [lo(c), hi(c))} M(r, c) x[r] for c < C.  A column goes to
// a group of wpc warps of one block (wpc = the grid's warps over C, a power of
// two up to 16: long columns get many warps when there are few of them); the
// lanes of the group take its rows in order, eight loads in flight each, and
// the group's sums are added in warp order (fixed shuffle tree inside a warp):
// the same result on every run (the split depends only on C and the grid).
__device__ void colprod(const double *__restrict__ M, int64_t ld, int r0, int R, int C, int shape,
                        const double *__restrict__ x, double *__restrict__ out) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  const int total = gridDim.x * nwb;
  int wpc = 1;
  while (wpc < nwb && wpc * 2 * C <= total) wpc *= 2;
  const int gpb = nwb / wpc;                            // column groups per block
  const int grp = warp / wpc, wi = warp - grp * wpc;    // this warp's group and rank in it
  const int groups = gridDim.x * gpb;
  const int stride = 32 * wpc;
  for (int base = 0; base < C; base += groups) {        // the same trip count in every block
    const int c = base + blockIdx.x * gpb + grp;
    double s = 0.0;
    if (c < C) {
      const int lo = col_lo(shape, c, r0), hi = col_hi(shape, c, R);
      const double *col = M + (size_t)c * ld;
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      int r = lo + wi * 32 + lane;
      for (; r + 7 * stride < hi; r += 8 * stride) {
        double cv[8], xv[8];
#pragma unroll
        for (int k = 0; k < 8; k++) {
          cv[k] = __ldcg(col + r + stride * k);
          xv[k] = __ldcg(x + r + stride * k);
        }
#pragma unroll
        for (int k = 0; k < 8; k++) acc[k & 3] = fma(cv[k], xv[k], acc[k & 3]);
      }
      for (; r < hi; r += stride) acc[0] = fma(__ldcg(col + r), __ldcg(x + r), acc[0]);
      s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (wpc == 1) {
      if (c < C && lane == 0) out[c] = s;
    } else {
      __syncthreads();
      if (lane == 0) red[warp] = s;
      __syncthreads();
      if (c < C && wi == 0 && lane == 0) {
        double t = 0.0;
        for (int k = 0; k < wpc; k++) t += red[grp * wpc + k];
        out[c] = t;
      }
    }
  }
}

// Row products over rows [r0, R), columns [0, C): s0(r) = sum_c M(r, c) t0[c ts0]
// (and s1(r) with t1 when NV = 2).  Tiles of kT rows x kCols columns go to the
// blocks; each writes its partial sums, and the last block of a row group to
// finish adds them in chunk order and calls epi(r, s0, s1, c), which stores
// the row's results and its shares c[0..np) of np sums; those are added over
// the group into tp_out[k tps + group] (when tp_out is set).
template <int NV, class Epi>
__device__ void rowprod(const BhuArgs &A, const double *__restrict__ M, int64_t ld, int r0, int R, int C, int shape,
                        const double *t0, int64_t ts0, const double *t1, int64_t ts1, Epi epi, double *tp_out,
                        int np = 1) {
  __shared__ double tc[2][kCols];
  __shared__ int s_last;
  __shared__ double red[32];
  const int groups = groups_of(R - r0), chunks = C > 0 ? (C + kCols - 1) / kCols : 0;
  for (int tile = blockIdx.x; tile < groups * chunks; tile += gridDim.x) {
    const int gi = tile / chunks, ch = tile - gi * chunks;
    const int ra = r0 + gi * kT, rb = min(ra + kT, R), ca = ch * kCols, cb = min(ca + kCols, C);
    const int r = ra + threadIdx.x;
    __syncthreads();
    if (!tile_zero(shape, ra, rb, ca, cb)) {
      for (int c = ca + threadIdx.x; c < cb; c += blockDim.x) {
        tc[0][c - ca] = __ldcg(t0 + (size_t)c * ts0);
        if (NV == 2) tc[1][c - ca] = __ldcg(t1 + (size_t)c * ts1);
      }
      __syncthreads();
      if (r < rb) {
        // eight independent loads in flight per thread, four accumulators
        const double *row = M + r;
        double sa[4] = {0.0, 0.0, 0.0, 0.0}, qa[4] = {0.0, 0.0, 0.0, 0.0};
        int c = ca;
        for (; c + 7 < cb; c += 8) {
          double mv[8];
#pragma unroll
          for (int k = 0; k < 8; k++) mv[k] = __ldcg(row + (size_t)(c + k) * ld);
#pragma unroll
          for (int k = 0; k < 8; k++) {
            sa[k & 3] = fma(mv[k], tc[0][c + k - ca], sa[k & 3]);
            if (NV == 2) qa[k & 3] = fma(mv[k], tc[1][c + k - ca], qa[k & 3]);
          }
        }
        for (; c < cb; c++) {
          const double m0 = __ldcg(row + (size_t)c * ld);
          sa[0] = fma(m0, tc[0][c - ca], sa[0]);
          if (NV == 2) qa[0] = fma(m0, tc[1][c - ca], qa[0]);
        }
        A.part[(size_t)ch * A.ldp + r] = (sa[0] + sa[1]) + (sa[2] + sa[3]);
        if (NV == 2) A.part2[(size_t)ch * A.ldp + r] = (qa[0] + qa[1]) + (qa[2] + qa[3]);
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned prev = atomicAdd(&A.cnt[gi], 1u);
      s_last = prev == (unsigned)chunks - 1;
      if (s_last) A.cnt[gi] = 0;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      double contrib[kMaxRank];
#pragma unroll
      for (int k = 0; k < kMaxRank; k++) contrib[k] = 0.0;
      if (r < rb) {
        // the chunks that hold more than structural zeros form one range
        // [k0, k1); eight partial loads in flight, added in chunk order
        int k0 = 0, k1 = chunks;
        while (k0 < k1 && tile_zero(shape, ra, rb, k0 * kCols, min(k0 * kCols + kCols, C))) k0++;
        while (k1 > k0 && tile_zero(shape, ra, rb, (k1 - 1) * kCols, min((k1 - 1) * kCols + kCols, C))) k1--;
        double a0 = 0.0, a1 = 0.0;
        int k = k0;
        for (; k + 7 < k1; k += 8) {
          double v0[8], v1[8];
#pragma unroll
          for (int q = 0; q < 8; q++) {
            v0[q] = __ldcg(A.part + (size_t)(k + q) * A.ldp + r);
            if (NV == 2) v1[q] = __ldcg(A.part2 + (size_t)(k + q) * A.ldp + r);
          }
#pragma unroll
          for (int q = 0; q < 8; q++) {
            a0 += v0[q];
            if (NV == 2) a1 += v1[q];
          }
        }
        for (; k < k1; k++) {
          a0 += __ldcg(A.part + (size_t)k * A.ldp + r);
          if (NV == 2) a1 += __ldcg(A.part2 + (size_t)k * A.ldp + r);
        }
        epi(r, a0, a1, contrib);
      }
      if (tp_out) {
        for (int k = 0; k < np; k++) {
          const double sum = block_sum(contrib[k], red);
          if (threadIdx.x == 0) tp_out[k * A.tps + gi] = sum;
        }
      }
    }
  }
}

// Group partials of sum w(r) over rows [r0, R) without a product (the first
// column or row of a step, when no reflector of that side exists yet).
template <class F>
__device__ void group_partials(int r0, int R, F w, double *tp_out) {
  __shared__ double red[32];
  for (int gi = blockIdx.x; gi < groups_of(R - r0); gi += gridDim.x) {
    const int r = r0 + gi * kT + threadIdx.x;
    const double sum = block_sum(r < R ? w(r) : 0.0, red);
    if (threadIdx.x == 0) tp_out[gi] = sum;
  }
}

// The whole of Algorithm 1 in one cooperative launch: per step j the phases
// below, each ended by a grid barrier.
__global__ void __launch_bounds__(kT, 1) k_bhu_persist(BhuArgs A) {
  unsigned gen = 0;
  if (A.stall && blockIdx.x == 0) return;
  const int m = A.m, n = A.n;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthreads = gridDim.x * blockDim.x;
  for (int j = 0; j < A.steps; j++) {
    const int cR = min(j, A.nr), cL = min(j, A.nl);
    // z = P_{j-1} e_j = e_j - W p1, p1 = R' W^T e_j (from the previous step); partials of v^T z
    if (cR > 0) {
      rowprod<1>(A, A.W, n, 0, n, cR, kW, A.p1, 1, nullptr, 0, [&](int r, double s, double, double *c) {
        const double zr = (r == j ? 1.0 : 0.0) - s;
        A.z[r] = zr;
        for (int k = 0; k < A.rk; k++) c[k] = A.v[r + k * A.ldv] * zr;
      }, A.tp, A.rk);
    } else {
      for (int r = gtid; r < n; r += gthreads) A.z[r] = r == j ? 1.0 : 0.0;
    }
    if (!grid_barrier(A, gen)) return;
    // x = B z + U (V^T z)
    {
      double w[kMaxRank];
      for (int k = 0; k < A.rk; k++) w[k] = cR > 0 ? tp_sum(A.tp + k * A.tps, groups_of(n)) : A.v[j + k * A.ldv];
      for (int r = gtid; r < m; r += gthreads) {
        double s = 0.0;
        if (r < n) s = A.d[r] * __ldcg(A.z + r);
        if (r + 1 < n) s = fma(A.e[r], __ldcg(A.z + r + 1), s);
        for (int k = 0; k < A.rk; k++) s = fma(A.u[r + k * A.ldu], w[k], s);
        A.x[r] = s;
      }
    }
    if (!grid_barrier(A, gen)) return;
    // a = Q_{j-1}^T x = x - Y S^T Y^T x (rows j..m); partials of a^2 there
    const double *acol = A.x;
    if (cL > 0) {
      colprod(A.Y, m, 0, m, cL, kY, A.x, A.g);
      if (!grid_barrier(A, gen)) return;
      colprod(A.SL, A.ldl, 0, cL, cL, kUT, A.g, A.hv);
      if (!grid_barrier(A, gen)) return;
      rowprod<1>(A, A.Y, m, j, m, cL, kY, A.hv, 1, nullptr, 0, [&](int r, double s, double, double *c) {
        const double ar = __ldcg(A.x + r) - s;
        A.a[r] = ar;
        c[0] = ar * ar;
      }, A.tp);
      acol = A.a;
    } else {
      group_partials(j, m, [&](int r) { const double xr = __ldcg(A.x + r); return xr * xr; }, A.tp);
    }
    if (!grid_barrier(A, gen)) return;
    // the left reflector of a(j..m): y_j, alpha_j, S(j, j) = 2 (Eq. house)
    const bool lmake = j < A.nl;
    double *yj = A.Y + (size_t)j * m;
    {
      const double a0 = __ldcg(acol + j);
      if (lmake) {
        const double sigma = sqrt(tp_sum(A.tp, groups_of(m - j)));
        const double sg = copysign(1.0, a0);
        const double inv = sigma > 0.0 ? 1.0 / sqrt(2.0 * sigma * (sigma + fabs(a0))) : 0.0;
        for (int r = j + gtid; r < m; r += gthreads) {
          const double y = (r == j ? fma(sg, sigma, a0) : __ldcg(acol + r)) * inv;
          yj[r] = y;
          if (r == 0) A.p1[0] = 2.0 * y;  // j = 0: S_0 Y_0^T e_0
        }
        if (gtid == 0) {
          A.alpha[j] = sigma > 0.0 ? -sg * sigma : 0.0;
          A.SL[j + (size_t)j * A.ldl] = 2.0;
        }
      } else if (gtid == 0) {
        A.alpha[j] = a0;
      }
    }
    if (!grid_barrier(A, gen)) return;
    const bool right = j <= n - 2;
    if (lmake && j > 0) {
      // s = Y_{j-1}^T y_j; then S(:, j) = -2 S s and p1 = S_j Y_j^T e_j =
      // (S yr + eta S(:, j), 2 eta), yr = Y(j, 0..j-1), eta = Y(j, j)
      colprod(A.Y, m, 0, m, j, kY, yj, A.sv);
      if (!grid_barrier(A, gen)) return;
      const double eta = __ldcg(yj + j);
      rowprod<2>(A, A.SL, A.ldl, 0, j, j, kUT, A.sv, 1, A.Y + j, m, [&](int r, double ss, double sy, double *) {
        const double col = -2.0 * ss;
        A.SL[r + (size_t)j * A.ldl] = col;
        A.p1[r] = fma(eta, col, sy);
      }, nullptr);
      if (gtid == 0) A.p1[j] = 2.0 * eta;
      if (!grid_barrier(A, gen)) return;
    }
    if (!right) continue;
    // q = Q_j e_j = e_j - Y p1; partials of U^T q
    const int cL1 = min(j + 1, A.nl);
    rowprod<1>(A, A.Y, m, 0, m, cL1, kY, A.p1, 1, nullptr, 0, [&](int r, double s, double, double *c) {
      const double qr = (r == j ? 1.0 : 0.0) - s;
      A.q[r] = qr;
      for (int k = 0; k < A.rk; k++) c[k] = A.u[r + k * A.ldu] * qr;
    }, A.tp, A.rk);
    if (!grid_barrier(A, gen)) return;
    // r = B^T q + V (U^T q)
    {
      double w[kMaxRank];
      for (int k = 0; k < A.rk; k++) w[k] = tp_sum(A.tp + k * A.tps, groups_of(m));
      for (int c = gtid; c < n; c += gthreads) {
        double s = A.d[c] * __ldcg(A.q + c);
        if (c > 0) s = fma(A.e[c - 1], __ldcg(A.q + c - 1), s);
        for (int k = 0; k < A.rk; k++) s = fma(A.v[c + k * A.ldv], w[k], s);
        A.ra[c] = s;
      }
    }
    if (!grid_barrier(A, gen)) return;
    // a* = P_{j-1}^T r = r - W R'^T W^T r (columns j+1..n); partials of a*^2 there
    const double *arow = A.ra;
    if (cR > 0) {
      colprod(A.W, n, 0, n, cR, kW, A.ra, A.gw);
      if (!grid_barrier(A, gen)) return;
      colprod(A.SR, A.ldr, 0, cR, cR, kUT, A.gw, A.hw);
      if (!grid_barrier(A, gen)) return;
      rowprod<1>(A, A.W, n, j + 1, n, cR, kW, A.hw, 1, nullptr, 0, [&](int r, double s, double, double *c) {
        const double ar = __ldcg(A.ra + r) - s;
        A.as[r] = ar;
        c[0] = ar * ar;
      }, A.tp);
      arow = A.as;
    } else {
      group_partials(j + 1, n, [&](int r) { const double xr = __ldcg(A.ra + r); return xr * xr; }, A.tp);
    }
    if (!grid_barrier(A, gen)) return;
    // the right reflector of a*(j+1..n): w_{j+1}, beta_j, R'(j, j) = 2
    const bool rmake = j < A.nr;
    double *wj = A.W + (size_t)j * n;
    {
      const double a0 = __ldcg(arow + j + 1);
      if (rmake) {
        const double sigma = sqrt(tp_sum(A.tp, groups_of(n - j - 1)));
        const double sg = copysign(1.0, a0);
        const double inv = sigma > 0.0 ? 1.0 / sqrt(2.0 * sigma * (sigma + fabs(a0))) : 0.0;
        for (int c = j + 1 + gtid; c < n; c += gthreads) {
          const double w = (c == j + 1 ? fma(sg, sigma, a0) : __ldcg(arow + c)) * inv;
          wj[c] = w;
          if (j == 0 && c == 1) A.p1[0] = 2.0 * w;  // the next step's R'_0 W_0^T e_1
        }
        if (gtid == 0) {
          A.beta[j] = sigma > 0.0 ? -sg * sigma : 0.0;
          A.SR[j + (size_t)j * A.ldr] = 2.0;
        }
      } else if (gtid == 0) {
        A.beta[j] = a0;
      }
    }
    if (!grid_barrier(A, gen)) return;
    if (j + 1 >= A.steps) continue;
    // the next step's p1 = R'_j W_j^T e_{j+1}
    if (rmake && j > 0) {
      colprod(A.W, n, 0, n, j, kW, wj, A.sv);  // s' = W_{j-1}^T w
      if (!grid_barrier(A, gen)) return;
      const double om = __ldcg(wj + j + 1);
      rowprod<2>(A, A.SR, A.ldr, 0, j, j, kUT, A.sv, 1, A.W + j + 1, n, [&](int r, double ss, double sw, double *) {
        const double col = -2.0 * ss;
        A.SR[r + (size_t)j * A.ldr] = col;
        A.p1[r] = fma(om, col, sw);
      }, nullptr);
      if (gtid == 0) A.p1[j] = 2.0 * om;
      if (!grid_barrier(A, gen)) return;
    } else if (!rmake) {
      const int c2 = A.nr;  // every right reflector made: p1 = R' W^T e_{j+1}
      if (c2 > 0) {
        rowprod<1>(A, A.SR, A.ldr, 0, c2, c2, kUT, A.W + j + 1, n, nullptr, 0, [&](int r, double s, double, double *) {
          A.p1[r] = s;
        }, nullptr);
        if (!grid_barrier(A, gen)) return;
      }
    }
  }
}

// d, e of the band at rest (r1[1], r1[2], dg[2][2..n], dg[3][2..n-1]) and back.
__global__ void k_band_get(BandPtrs b, int n, double *d, double *e) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    d[i] = i == 0 ? b.r1[1] : b.dg[2][i + 1];
    if (i + 1 < n) e[i] = i == 0 ? b.r1[2] : b.dg[3][i + 1];
  }
}
__global__ void k_band_put(BandPtrs b, int n, const double *d, const double *e) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i == 0) b.r1[1] = d[0]; else b.dg[2][i + 1] = d[i];
    if (i + 1 < n) {
      if (i == 0) b.r1[2] = e[0]; else b.dg[3][i + 1] = e[i];
    }
  }
}

// The symmetric variant (Sec. 6, future directions): the Householder
// tridiagonalization of T + rho u u^T (T symmetric tridiagonal, diagonal d,
// off-diagonal e; u = Q^T c).  Step j is the left half of a BHU step with the
// reflector applied on both sides: column j of Q_{j-1}^T (T + rho u u^T) Q_{j-1}
// from z = Q_{j-1} e_j, x = T z + u (rho u^T z), a = Q_{j-1}^T x, with
// Q_{j-1} = I - W R' W^T (w_j with zeros in rows 0..j, as the right reflectors
// of BHU); alpha_j = a(j), and the reflector of a(j+1..n) gives beta_j and w_j.
// Eight phases a step.
__global__ void __launch_bounds__(kT, 1) k_tri_persist(BhuArgs A) {
  unsigned gen = 0;
  if (A.stall && blockIdx.x == 0) return;
  const int n = A.n;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthreads = gridDim.x * blockDim.x;
  for (int j = 0; j < A.steps; j++) {
    const int cY = min(j, A.nr);
    // z = Q_{j-1} e_j = e_j - W p1 (p1 = R' W^T e_j from the previous step); partials of u^T z
    if (cY > 0) {
      rowprod<1>(A, A.W, n, 0, n, cY, kW, A.p1, 1, nullptr, 0, [&](int r, double s, double, double *c) {
        const double zr = (r == j ? 1.0 : 0.0) - s;
        A.z[r] = zr;
        c[0] = A.u[r] * zr;
      }, A.tp);
    } else {
      for (int r = gtid; r < n; r += gthreads) A.z[r] = r == j ? 1.0 : 0.0;
    }
    if (!grid_barrier(A, gen)) return;
    // x = T z + u (rho u^T z)
    {
      const double w = A.rho * (cY > 0 ? tp_sum(A.tp, groups_of(n)) : A.u[j]);
      for (int r = gtid; r < n; r += gthreads) {
        double s = A.d[r] * __ldcg(A.z + r);
        if (r + 1 < n) s = fma(A.e[r], __ldcg(A.z + r + 1), s);
        if (r > 0) s = fma(A.e[r - 1], __ldcg(A.z + r - 1), s);
        A.x[r] = fma(A.u[r], w, s);
      }
    }
    if (!grid_barrier(A, gen)) return;
    // a = Q_{j-1}^T x (rows j..n); partials of a^2 over rows j+1..n
    const double *acol = A.x;
    if (cY > 0) {
      colprod(A.W, n, 0, n, cY, kW, A.x, A.g);
      if (!grid_barrier(A, gen)) return;
      colprod(A.SR, A.ldr, 0, cY, cY, kUT, A.g, A.hv);
      if (!grid_barrier(A, gen)) return;
      rowprod<1>(A, A.W, n, j, n, cY, kW, A.hv, 1, nullptr, 0, [&](int r, double s, double, double *c) {
        const double ar = __ldcg(A.x + r) - s;
        A.a[r] = ar;
        c[0] = r > j ? ar * ar : 0.0;
      }, A.tp);
      acol = A.a;
    } else {
      group_partials(j, n, [&](int r) { const double xr = __ldcg(A.x + r); return r > j ? xr * xr : 0.0; }, A.tp);
    }
    if (!grid_barrier(A, gen)) return;
    // alpha_j = a(j); the reflector of a(j+1..n): w_j, beta_j, R'(j, j) = 2
    const bool make = j < A.nr;
    double *wj = A.W + (size_t)j * n;
    if (gtid == 0) A.alpha[j] = __ldcg(acol + j);
    if (make) {
      const double a0 = __ldcg(acol + j + 1);
      const double sigma = sqrt(tp_sum(A.tp, groups_of(n - j)));
      const double sg = copysign(1.0, a0);
      const double inv = sigma > 0.0 ? 1.0 / sqrt(2.0 * sigma * (sigma + fabs(a0))) : 0.0;
      for (int r = j + 1 + gtid; r < n; r += gthreads) {
        const double w = (r == j + 1 ? fma(sg, sigma, a0) : __ldcg(acol + r)) * inv;
        wj[r] = w;
        if (j == 0 && r == 1) A.p1[0] = 2.0 * w;  // the next step's R'_0 W_0^T e_1
      }
      if (gtid == 0) {
        A.beta[j] = sigma > 0.0 ? -sg * sigma : 0.0;
        A.SR[j + (size_t)j * A.ldr] = 2.0;
      }
    } else if (j == n - 2 && gtid == 0) {
      A.beta[j] = __ldcg(acol + j + 1);
    }
    if (!grid_barrier(A, gen)) return;
    if (j + 1 >= A.steps) continue;
    // the next step's p1 = R'_j W_j^T e_{j+1}
    if (make && j > 0) {
      colprod(A.W, n, 0, n, j, kW, wj, A.sv);
      if (!grid_barrier(A, gen)) return;
      const double om = __ldcg(wj + j + 1);
      rowprod<2>(A, A.SR, A.ldr, 0, j, j, kUT, A.sv, 1, A.W + j + 1, n, [&](int r, double ss, double sw, double *) {
        const double col = -2.0 * ss;
        A.SR[r + (size_t)j * A.ldr] = col;
        A.p1[r] = fma(om, col, sw);
      }, nullptr);
      if (gtid == 0) A.p1[j] = 2.0 * om;
      if (!grid_barrier(A, gen)) return;
    } else if (!make && A.nr > 0) {
      const int c2 = A.nr;
      rowprod<1>(A, A.SR, A.ldr, 0, c2, c2, kUT, A.W + j + 1, n, nullptr, 0, [&](int r, double s, double, double *) {
        A.p1[r] = s;
      }, nullptr);
      if (!grid_barrier(A, gen)) return;
    }
  }
}

int grid_for(int64_t count, int threads) {
  int64_t g = (count + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > 1184 ? 1184 : g));
}

}  // namespace

BhuSizes bhu_sizes(int64_t m, int64_t n, int64_t steps) {
  BhuSizes z{};
  const int64_t nl = m > n ? n : n - 1, nr = n > 2 ? n - 2 : 0;
  z.kl = steps < nl ? steps : nl;
  z.kr = steps < nr ? steps : nr;
  const int64_t big = m > n ? m : n;
  const int64_t chunks = (big + kCols - 1) / kCols + 1;
  const int64_t groups = (big + kT - 1) / kT + 1;
  // twelve vectors, two partial-sum planes, the group partials of kMaxRank sums
  z.ws_doubles = 12 * big + 2 * chunks * big + kMaxRank * groups + 8;
  z.ws_counters = groups + 4;  // per row group, then the barrier's count and generation
  return z;
}

cudaError_t launch_bhu(int m, int n, int steps, int rk, const double *d, const double *e, const double *u,
                       int64_t ldu, const double *v, int64_t ldv, double *alpha, double *beta, double *Y, double *W,
                       double *SL, double *SR, double *ws, unsigned *cnt, int *status, cudaStream_t s,
                       int64_t *launches) {
  if (rk < 1 || rk > kMaxRank) return cudaErrorInvalidValue;
  const BhuSizes z = bhu_sizes(m, n, steps);
  const int big = m > n ? m : n;
  const int64_t chunks = (big + kCols - 1) / kCols + 1;
  const int64_t groups = (big + kT - 1) / kT + 1;
  BhuArgs A{};
  A.m = m; A.n = n; A.steps = steps;
  A.nl = m > n ? n : n - 1;
  A.nr = n > 2 ? n - 2 : 0;
  A.ldl = z.kl > 0 ? z.kl : 1;
  A.ldr = z.kr > 0 ? z.kr : 1;
  A.ldp = big;
  A.d = d; A.e = e; A.u = u; A.v = v;
  A.rk = rk; A.ldu = ldu; A.ldv = ldv; A.tps = groups;
  A.alpha = alpha; A.beta = beta; A.Y = Y; A.W = W; A.SL = SL; A.SR = SR;
  double *p = ws;
  double **vecs[12] = {&A.z, &A.x, &A.a, &A.q, &A.ra, &A.as, &A.g, &A.hv, &A.p1, &A.gw, &A.hw, &A.sv};
  for (double **vp : vecs) { *vp = p; p += big; }
  A.part = p; p += chunks * big;
  A.part2 = p; p += chunks * big;
  A.tp = p;
  A.cnt = cnt;
  A.bar = cnt + groups;
  A.status = status;
  const Injection inj = injection();
  A.stall = inj.site == BDU_INJECT_BHU_STALL ? 1 : 0;
  A.spin = A.stall ? (int)(inj.value < kBarSpin ? inj.value : kBarSpin) : kBarSpin;
  cudaError_t err = cudaSuccess;
  if (z.kl > 0) err = cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)m * z.kl, s);
  if (err == cudaSuccess && z.kr > 0) err = cudaMemsetAsync(W, 0, sizeof(double) * (size_t)n * z.kr, s);
  if (err == cudaSuccess && z.kl > 0) err = cudaMemsetAsync(SL, 0, sizeof(double) * (size_t)z.kl * z.kl, s);
  if (err == cudaSuccess && z.kr > 0) err = cudaMemsetAsync(SR, 0, sizeof(double) * (size_t)z.kr * z.kr, s);
  if (err == cudaSuccess) err = cudaMemsetAsync(A.bar, 0, 2 * sizeof(unsigned), s);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0, per = 0;
  err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bhu_persist, kT, 0);
  if (err != cudaSuccess) return err;
  if (per < 1) return cudaErrorLaunchOutOfResources;
  const int blocks = sms * (per > 2 ? 2 : per);
  void *args[] = {&A};
  err = cudaLaunchCooperativeKernel((const void *)k_bhu_persist, dim3(blocks), dim3(kT), args, 0, s);
  if (launches) *launches += 1;
  return err;
}

cudaError_t launch_tri(int n, int steps, const double *a, const double *b, double rho, const double *u,
                       double *alpha, double *beta, double *Y, double *S, double *ws, unsigned *cnt, int *status,
                       cudaStream_t s) {
  const BhuSizes z = bhu_sizes(n, n, steps);
  const int64_t chunks = (n + kCols - 1) / kCols + 1;
  const int64_t groups = (n + kT - 1) / kT + 1;
  BhuArgs A{};
  A.m = n; A.n = n; A.steps = steps;
  A.nl = 0;
  A.nr = n > 2 ? n - 2 : 0;  // reflectors of a complete run
  const int64_t k = z.kr;     // reflectors of this run
  A.ldl = 1;
  A.ldr = k > 0 ? k : 1;
  A.ldp = n;
  A.d = a; A.e = b; A.u = u; A.v = u; A.rho = rho;
  A.rk = 1; A.ldu = n; A.ldv = n; A.tps = groups;
  A.alpha = alpha; A.beta = beta; A.W = Y; A.SR = S;
  double *p = ws;
  double **vecs[12] = {&A.z, &A.x, &A.a, &A.q, &A.ra, &A.as, &A.g, &A.hv, &A.p1, &A.gw, &A.hw, &A.sv};
  for (double **vp : vecs) { *vp = p; p += n; }
  A.part = p; p += chunks * n;
  A.part2 = p; p += chunks * n;
  A.tp = p;
  A.cnt = cnt;
  A.bar = cnt + groups;
  A.status = status;
  const Injection inj = injection();
  A.stall = inj.site == BDU_INJECT_BHU_STALL ? 1 : 0;
  A.spin = A.stall ? (int)(inj.value < kBarSpin ? inj.value : kBarSpin) : kBarSpin;
  cudaError_t err = cudaSuccess;
  if (k > 0) err = cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)n * k, s);
  if (err == cudaSuccess && k > 0) err = cudaMemsetAsync(S, 0, sizeof(double) * (size_t)k * k, s);
  if (err == cudaSuccess) err = cudaMemsetAsync(A.bar, 0, 2 * sizeof(unsigned), s);
  if (err != cudaSuccess) return err;
  int dev = 0, sms = 0, per = 0;
  err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tri_persist, kT, 0);
  if (err != cudaSuccess) return err;
  if (per < 1) return cudaErrorLaunchOutOfResources;
  void *args[] = {&A};
  return cudaLaunchCooperativeKernel((const void *)k_tri_persist, dim3(sms), dim3(kT), args, 0, s);
}

cudaError_t launch_bhu_band_get(double *band, int m, int n, double *d, double *e, cudaStream_t s) {
  k_band_get<<<grid_for(n, 256), 256, 0, s>>>(band_ptrs(band, m, n), n, d, e);
  return cudaGetLastError();
}
cudaError_t launch_bhu_band_put(double *band, int m, int n, const double *d, const double *e, cudaStream_t s) {
  k_band_put<<<grid_for(n, 256), 256, 0, s>>>(band_ptrs(band, m, n), n, d, e);
  return cudaGetLastError();
}

}  // namespace bdu
