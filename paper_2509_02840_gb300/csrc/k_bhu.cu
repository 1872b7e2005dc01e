// BHU, the bidiagonal Householder update (Sec. 3.3, Algorithm 1, Theorem 1),
// FP64, on the GPU.
//
// The m x n matrix A = B + u v^T (B upper bidiagonal, m >= n) is
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
// factored form Q^T (B + u v^T) P that Theorem 1 expands:
//
//   column j:  z = P_{j-1} e_j,  x = B z + u (v^T z),  a = Q_{j-1}^T x,
//   row j:     q = Q_j e_j,      r = B^T q + v (u^T q), a* = P_{j-1}^T r,
//
// each O((m + n) j) work in products with Y, W, S, R'.  The reflector of a
// (rows j..m) gives alpha_j and y_j, the reflector of a* (columns j+1..n)
// beta_j and w_{j+1}.  The readings are those of the oracle: row j (not j+1)
// defines the right reflector (Sec. 2.1), a left reflector for column n when
// m > n, and the last diagonal and superdiagonal entries read off without a
// reflector when m = n.
//
// Kernels: column products (one warp per column, lanes over rows in order,
// a fixed shuffle tree), row products (tiles of 256 rows x 64 columns, partial
// sums per column chunk, added in chunk order by the last block of each row
// tile to finish), the reflector (one block) and small vector kernels.  Every
// result is deterministic: no atomics on values, fixed summation orders.
// Entries the structure makes zero (above y_j, in W's rows 1..j, below the
// diagonal of S, R') are skipped, never read.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bdu_internal.cuh"

namespace bdu {
namespace {

constexpr int kRows = 256;  // rows per tile of a row product (one thread per row)
constexpr int kCols = 64;   // columns per partial-sum chunk
constexpr int kHouseThreads = 1024;

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

// out[c] = scale * sum_{r in [lo(c), hi(c))} M(r, c) x[r], c < C.
__global__ void k_gemv_t(const double *__restrict__ M, int64_t ld, int r0, int R, int C, int shape,
                         const double *__restrict__ x, double scale, double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < C; c += warps) {
    const int lo = col_lo(shape, c, r0), hi = col_hi(shape, c, R);
    const double *col = M + (size_t)c * ld;
    double s0 = 0.0, s1 = 0.0;
    int r = lo + lane;
    for (; r + 32 < hi; r += 64) {
      s0 = fma(col[r], x[r], s0);
      s1 = fma(col[r + 32], x[r + 32], s1);
    }
    if (r < hi) s0 = fma(col[r], x[r], s0);
    double s = s0 + s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[c] = scale * s;
  }
}

// The row tiles [ra, rb) x column chunk [ca, cb) that hold only structural zeros.
__device__ __forceinline__ bool tile_zero(int shape, int ra, int rb, int ca, int cb) {
  if (shape == kY) return rb <= ca;       // every r < c
  if (shape == kW) return rb <= ca + 1;   // every r <= c
  if (shape == kUT) return ra >= cb;      // every r > c
  return false;
}

// out[r] = base(r) + scale * sum_{c < C} M(r, c) t[c * ts] for r in [r0, R),
// base(r) = (base ? base[r] : 0) + (r == unit ? 1 : 0).
// grid (row tiles, column chunks); part: chunks x ldp partial sums; cnt: one
// counter per row tile, zero on entry and left zero.
__global__ void __launch_bounds__(kRows) k_gemv_n(const double *__restrict__ M, int64_t ld, int r0, int R, int C,
                                                  int shape, const double *__restrict__ t, int64_t ts,
                                                  const double *__restrict__ base, int unit, double scale,
                                                  double *__restrict__ out, double *part, int64_t ldp,
                                                  unsigned *cnt) {
  const int tile = blockIdx.x, chunk = blockIdx.y, chunks = gridDim.y;
  const int ra = r0 + tile * kRows, rb = min(ra + kRows, R);
  const int ca = chunk * kCols, cb = min(ca + kCols, C);
  const int r = ra + threadIdx.x;
  __shared__ double tc[kCols];
  __shared__ bool last;
  if (!tile_zero(shape, ra, rb, ca, cb)) {
    for (int c = ca + threadIdx.x; c < cb; c += blockDim.x) tc[c - ca] = t[(size_t)c * ts];
    __syncthreads();
    if (r < rb) {
      const double *row = M + r;
      double s0 = 0.0, s1 = 0.0;
      int c = ca;
      for (; c + 1 < cb; c += 2) {
        s0 = fma(row[(size_t)c * ld], tc[c - ca], s0);
        s1 = fma(row[(size_t)(c + 1) * ld], tc[c + 1 - ca], s1);
      }
      if (c < cb) s0 = fma(row[(size_t)c * ld], tc[c - ca], s0);
      part[(size_t)chunk * ldp + r] = s0 + s1;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&cnt[tile], 1u);
    last = prev == (unsigned)chunks - 1;
    if (last) cnt[tile] = 0;
  }
  __syncthreads();
  if (!last || r >= rb) return;
  __threadfence();
  double s = 0.0;
  for (int k = 0; k < chunks; k++) {
    const int ka = k * kCols, kb = min(ka + kCols, C);
    if (tile_zero(shape, ra, rb, ka, kb)) continue;
    s += __ldcg(part + (size_t)k * ldp + r);
  }
  double b = base ? base[r] : 0.0;
  if (r == unit) b += 1.0;
  out[r] = fma(scale, s, b);
}

// Deterministic block sum of v over the block (blockDim.x a multiple of 32).
__device__ __forceinline__ double block_sum(double v, double *sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < nw; k++) s += sh[k];
  return s;
}

// out[0] = sum_{r < len} a[r] b[r] (one block).
__global__ void k_dot(const double *__restrict__ a, const double *__restrict__ b, int len, double *out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int r = threadIdx.x; r < len; r += blockDim.x) s = fma(a[r], b[r], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] = s;
}

// x = B z + u * dot: x[r] = d[r] z[r] + e[r] z[r+1] + u[r] dot (r < m; B is m x n).
__global__ void k_bmv(const double *__restrict__ d, const double *__restrict__ e, int m, int n,
                      const double *__restrict__ z, const double *__restrict__ u, const double *dot,
                      double *__restrict__ x) {
  const double w = dot[0];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    double s = 0.0;
    if (r < n) s = d[r] * z[r];
    if (r + 1 < n) s = fma(e[r], z[r + 1], s);
    x[r] = fma(u[r], w, s);
  }
}

// y = B^T q + v * dot: y[c] = d[c] q[c] + e[c-1] q[c-1] + v[c] dot (c < n).
__global__ void k_bmvt(const double *__restrict__ d, const double *__restrict__ e, int n,
                       const double *__restrict__ q, const double *__restrict__ v, const double *dot,
                       double *__restrict__ y) {
  const double w = dot[0];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    double s = d[c] * q[c];
    if (c > 0) s = fma(e[c - 1], q[c - 1], s);
    y[c] = fma(v[c], w, s);
  }
}

__global__ void k_unit(double *z, int n, int j) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) z[r] = r == j ? 1.0 : 0.0;
}

// The reflector of a[lo..R) (Sec. 2.1, Eq. house, normalized): with make,
// y[lo..R) = (a + sign(a_lo) ||a|| e_lo) / ||.||, *alpha = -sign(a_lo) ||a||,
// *sdiag = 2 (the new diagonal entry of S or R'); a = 0 gives y = 0,
// alpha = 0.  Without make, *alpha = a[lo] (an entry read off without a
// reflector).
__global__ void __launch_bounds__(kHouseThreads) k_house(const double *__restrict__ a, int lo, int R, int make,
                                                         double *__restrict__ y, double *alpha, double *sdiag) {
  __shared__ double sh[32];
  if (!make) {
    if (threadIdx.x == 0) alpha[0] = a[lo];
    return;
  }
  double s = 0.0;
  for (int r = lo + threadIdx.x; r < R; r += blockDim.x) s = fma(a[r], a[r], s);
  const double ss = block_sum(s, sh);
  const double sigma = sqrt(ss);
  const double a0 = a[lo];
  const double sg = copysign(1.0, a0);
  // ||a + sg sigma e_lo||^2 = 2 sigma (sigma + |a0|)
  const double inv = sigma > 0.0 ? 1.0 / sqrt(2.0 * sigma * (sigma + fabs(a0))) : 0.0;
  for (int r = lo + threadIdx.x; r < R; r += blockDim.x) {
    const double v = r == lo ? fma(sg, sigma, a0) : a[r];
    y[r] = v * inv;
  }
  if (threadIdx.x == 0) {
    alpha[0] = sigma > 0.0 ? -sg * sigma : 0.0;
    sdiag[0] = 2.0;
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

int grid_for(int64_t count, int threads) {
  int64_t g = (count + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > 1184 ? 1184 : g));
}

struct Gemv {
  double *part;
  int64_t ldp;
  unsigned *cnt;
  cudaStream_t s;
  int64_t *launches;
  cudaError_t err = cudaSuccess;
  void t(const double *M, int64_t ld, int r0, int R, int C, int shape, const double *x, double scale, double *out) {
    if (err != cudaSuccess || C <= 0) return;
    const int threads = 256, blocks = grid_for((int64_t)C * 32, threads);
    k_gemv_t<<<blocks, threads, 0, s>>>(M, ld, r0, R, C, shape, x, scale, out);
    err = cudaGetLastError();
    (*launches)++;
  }
  void n(const double *M, int64_t ld, int r0, int R, int C, int shape, const double *tv, int64_t ts,
         const double *base, int unit, double scale, double *out) {
    if (err != cudaSuccess || R <= r0) return;
    if (C <= 0) {  // out = base(r) only
      return;
    }
    dim3 grid((R - r0 + kRows - 1) / kRows, (C + kCols - 1) / kCols);
    k_gemv_n<<<grid, kRows, 0, s>>>(M, ld, r0, R, C, shape, tv, ts, base, unit, scale, out, part, ldp, cnt);
    err = cudaGetLastError();
    (*launches)++;
  }
};

}  // namespace

BhuSizes bhu_sizes(int64_t m, int64_t n, int64_t steps) {
  BhuSizes z{};
  const int64_t nl = m > n ? n : n - 1, nr = n > 2 ? n - 2 : 0;
  z.kl = steps < nl ? steps : nl;
  z.kr = steps < nr ? steps : nr;
  const int64_t big = m > n ? m : n;
  const int64_t chunks = (big + kCols - 1) / kCols + 1;
  const int64_t tiles = (big + kRows - 1) / kRows + 1;
  // vectors: z, x, a, q, ra, astar (big each), g, h, p1, gw, hw, sv (big each), dot (2), d, e (big each)
  z.ws_doubles = 14 * big + 8 + chunks * big;
  z.ws_counters = tiles;
  return z;
}

cudaError_t launch_bhu(int m, int n, int steps, const double *d, const double *e, const double *u, const double *v,
                       double *alpha, double *beta, double *Y, double *W, double *SL, double *SR, double *ws,
                       unsigned *cnt, cudaStream_t s, int64_t *launches) {
  const BhuSizes z = bhu_sizes(m, n, steps);
  const int nl = m > n ? n : n - 1, nr = n > 2 ? n - 2 : 0;
  const int kl = (int)z.kl, kr = (int)z.kr;
  const int big = m > n ? m : n;
  const int64_t ldl = kl > 0 ? kl : 1, ldr = kr > 0 ? kr : 1;
  double *p = ws;
  double *zv = p; p += big;
  double *x = p; p += big;
  double *av = p; p += big;
  double *q = p; p += big;
  double *ra = p; p += big;
  double *as = p; p += big;
  double *g = p; p += big;
  double *hv = p; p += big;
  double *p1 = p; p += big;
  double *gw = p; p += big;
  double *hw = p; p += big;
  double *sv = p; p += big;
  p += 2 * big;  // (d, e copies live with the caller)
  double *dot = p; p += 8;
  double *part = p;
  int64_t dummy = 0;
  Gemv G{part, big, cnt, s, launches ? launches : &dummy};
  cudaError_t err = cudaSuccess;
  auto chk = [&]() { if (err == cudaSuccess) err = cudaGetLastError(); if (err == cudaSuccess) err = G.err; };
  if (kl > 0) err = cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)m * kl, s);
  if (err == cudaSuccess && kr > 0) err = cudaMemsetAsync(W, 0, sizeof(double) * (size_t)n * kr, s);
  if (err == cudaSuccess && kl > 0) err = cudaMemsetAsync(SL, 0, sizeof(double) * (size_t)kl * kl, s);
  if (err == cudaSuccess && kr > 0) err = cudaMemsetAsync(SR, 0, sizeof(double) * (size_t)kr * kr, s);
  const int vb = grid_for(big, 256);
  for (int j = 0; j < steps && err == cudaSuccess; j++) {
    // ---- column j of Q_{j-1}^T A P_{j-1}
    const int cR = j < nr ? j : nr;  // right reflectors so far
    if (cR > 0) {
      G.n(SR, ldr, 0, cR, cR, kUT, W + j, n, nullptr, -1, 1.0, p1);   // p1 = R' W^T e_j
      G.n(W, n, 0, n, cR, kW, p1, 1, nullptr, j, -1.0, zv);          // z = e_j - W p1
    } else {
      k_unit<<<vb, 256, 0, s>>>(zv, n, j);
      (*G.launches)++;
    }
    k_dot<<<1, 1024, 0, s>>>(v, zv, n, dot);
    k_bmv<<<vb, 256, 0, s>>>(d, e, m, n, zv, u, dot, x);
    *G.launches += 2;
    chk();
    const double *acol = x;
    const int cL = j < nl ? j : nl;  // left reflectors so far
    if (cL > 0) {
      G.t(Y, m, 0, m, cL, kY, x, 1.0, g);                            // g = Y^T x
      G.t(SL, ldl, 0, cL, cL, kUT, g, 1.0, hv);                      // h = S^T g
      G.n(Y, m, j, m, cL, kY, hv, 1, x, -1, -1.0, av);               // a = x - Y h (rows j..m)
      acol = av;
    }
    const bool lmake = j < nl;
    k_house<<<1, kHouseThreads, 0, s>>>(acol, j, m, lmake ? 1 : 0, lmake ? Y + (size_t)j * m : nullptr, alpha + j,
                                        lmake ? SL + j + (size_t)j * ldl : nullptr);
    (*G.launches)++;
    chk();
    if (lmake && j > 0) {
      G.t(Y, m, 0, m, j, kY, Y + (size_t)j * m, 1.0, sv);           // s = Y^T y_j
      G.n(SL, ldl, 0, j, j, kUT, sv, 1, nullptr, -1, -2.0, SL + (size_t)j * ldl);  // S(:, j) = -2 S s
    }
    if (j > n - 2) continue;
    // ---- row j of Q_j^T A P_{j-1}
    const int cL1 = (j + 1) < nl ? (j + 1) : nl;
    G.n(SL, ldl, 0, cL1, cL1, kUT, Y + j, m, nullptr, -1, 1.0, p1);   // p1 = S Y^T e_j
    G.n(Y, m, 0, m, cL1, kY, p1, 1, nullptr, j, -1.0, q);            // q = e_j - Y p1
    k_dot<<<1, 1024, 0, s>>>(u, q, m, dot + 1);
    k_bmvt<<<vb, 256, 0, s>>>(d, e, n, q, v, dot + 1, ra);
    *G.launches += 2;
    chk();
    const double *arow = ra;
    if (cR > 0) {
      G.t(W, n, 0, n, cR, kW, ra, 1.0, gw);                          // gw = W^T r
      G.t(SR, ldr, 0, cR, cR, kUT, gw, 1.0, hw);                     // hw = R'^T gw
      G.n(W, n, j + 1, n, cR, kW, hw, 1, ra, -1, -1.0, as);          // a* = r - W hw (columns j+1..n)
      arow = as;
    }
    const bool rmake = j < nr;
    k_house<<<1, kHouseThreads, 0, s>>>(arow, j + 1, n, rmake ? 1 : 0, rmake ? W + (size_t)j * n : nullptr, beta + j,
                                        rmake ? SR + j + (size_t)j * ldr : nullptr);
    (*G.launches)++;
    chk();
    if (rmake && j > 0) {
      G.t(W, n, 0, n, j, kW, W + (size_t)j * n, 1.0, sv);           // s = W^T w
      G.n(SR, ldr, 0, j, j, kUT, sv, 1, nullptr, -1, -2.0, SR + (size_t)j * ldr);  // R'(:, j) = -2 R' s
    }
    chk();
  }
  return err;
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
