// D = A B for FP32 operands on the tensor cores: the contractions of the
// mixed form's re-orthogonalization (Sec. 4.2; the Newton-Schulz step
// X <- X - X (X^T X - I) / 2).
//
// Operands are K-contiguous: A(m, k) at A[m * a_sr + k], B(k, n) at
// B[n * b_sr + k] (row strides multiples of 4 floats, bases 16-byte aligned),
// so that every 16-byte group of four consecutive k of one row is one row of
// a tensor-core core matrix.  One thread block per 128 x 128 tile of D walks
// K in chunks of 32: cp.async copies each chunk's groups straight from global
// memory into a shared-memory stage laid out as the MMA's K-major operand
// without swizzling (core matrices of 8 rows x 16 bytes; for each step of 8 in
// K, two 4-wide chunks of 16 cores), four stages deep, so that the copies run
// three chunks ahead.  One thread issues tcgen05.mma kind::tf32 (M = N = 128)
// on a chunk into one of two tensor-memory accumulators; tcgen05.commit
// arrives on the chunk's mbarrier when its MMAs are done, and the threads then
// add that accumulator (tcgen05.ld) into FP32 registers while the next
// chunk's MMAs run.
//
// Precision.  The tensor cores read an FP32 operand as TF32 (its top 10
// mantissa bits).  passes = 3 is 3xTF32: with x_hi the FP32 value as read and
// x_lo = x - x_hi (exact; formed in shared memory for each chunk),
// D = A_hi B_hi + (A_hi B_lo + A_lo B_hi), the correction terms in a second
// accumulator -- about FP32 accuracy.  passes = 1 is plain TF32, for products
// that are corrections of relative size far below FP32's.  The tensor cores'
// FP32 accumulation truncates toward zero, so a long sum kept in tensor
// memory drifts when one term dominates it (the nearly orthogonal factors'
// X^T X: 3.6e-5 off after a step at k = 8192, 5e-7 at 1024); each chunk of 32
// therefore starts a fresh accumulator, and the chunks' sums are added in
// registers with rounding to nearest.
//
// Output: D(m, n) = alpha * sum + beta * D(m, n) (beta 0 or 1; one fused
// multiply-add), at D[m * d_sm + n * d_sn].  For a symmetric product (A = B,
// M = N) only the tiles on and above the diagonal are computed, and each
// one above it is written twice, as itself and as its mirror image.
//
// Every wait is bounded; one that runs out sets ERR_GEMM, the block stops
// issuing, waits (bounded) for what it has issued, frees its tensor memory
// and returns.
#include <algorithm>

#include "async_copy.cuh"
#include "bdu_internal.cuh"
#include "tcgen05.cuh"

namespace bdu {
namespace {

using namespace tc;

constexpr int kT = 128;      // rows and columns of a D tile: the MMA's M and N, the TMEM lanes
constexpr int kTK = 32;      // K per chunk: one accumulator's sum
constexpr int kStages = 4;   // shared-memory stages of copied chunks
constexpr int kThreads = 256;
constexpr uint32_t kPart = kT * kTK * 4;  // bytes of one operand's chunk
constexpr uint32_t kStageBytes = 2 * kPart;

// Byte offset of element (r, k) of a 128 x kTK operand chunk in the K-major,
// no-swizzle layout: k-step k / 8 is a block of two 4-wide K chunks of 16
// core matrices of 8 rows x 16 bytes (LBO = 2048, SBO = 128).
__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return (uint32_t)((k >> 3) * 4096 + ((k >> 2) & 1) * 2048 + (r >> 3) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// 16-byte global -> shared copy; of the 16 bytes, `bytes` are read and the
// rest zero-filled
__device__ __forceinline__ void cp16(uint32_t dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

struct Operand {
  const float *p;
  int64_t sr;  // row stride (floats); k is contiguous
  int rows;
};

// Copies rows [r0, r0 + 128) x k [k0, k0 + kTK) of op into the stage at dst
// (zeros outside).  The eight threads of a quarter warp take eight
// consecutive rows at the same four k (one core matrix).
__device__ __forceinline__ void copy_chunk(const Operand &op, int r0, int k0, int K, uint32_t dst) {
  for (int it = threadIdx.x; it < kT * (kTK / 4); it += kThreads) {
    const int ln = it & 31, w = it >> 5;
    const int r = (ln & 7) + 8 * (w >> 1), kq = ((ln >> 3) + 4 * (w & 1)) * 4;
    const int gr = r0 + r, gk = k0 + kq;
    const int valid = (gr < op.rows && gk < K) ? min(4, K - gk) : 0;
    const float *src = valid ? op.p + (int64_t)gr * op.sr + gk : op.p;
    cp16(dst + core_off(r, kq), src, (uint32_t)valid * 4u);
  }
}

// lo = x - x_hi for a stage (both operands), x_hi = x with its low 13
// mantissa bits cleared (what the tensor cores read)
__device__ __forceinline__ void form_lo(const unsigned char *stage, unsigned char *lo) {
  for (int i = threadIdx.x; i < (int)(kStageBytes / 16); i += kThreads) {
    const uint4 v = reinterpret_cast<const uint4 *>(stage)[i];
    const uint32_t x[4] = {v.x, v.y, v.z, v.w};
    uint32_t y[4];
#pragma unroll
    for (int u = 0; u < 4; u++) y[u] = __float_as_uint(__uint_as_float(x[u]) - __uint_as_float(x[u] & 0xFFFFE000u));
    reinterpret_cast<uint4 *>(lo)[i] = make_uint4(y[0], y[1], y[2], y[3]);
  }
}

template <int P>
__host__ __device__ constexpr uint32_t buf_cols() { return P == 3 ? 2 * kT : kT; }
template <int P>
__host__ __device__ constexpr int smem_bytes() { return kStages * kStageBytes + (P == 3 ? 2 * kStageBytes : 0); }

template <int P>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(Operand A, Operand B, int K, float *__restrict__ D, int64_t d_sm, int64_t d_sn, float alpha,
              int beta, int sym, int *status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar_done[2];
  __shared__ uint32_t tbase;
  __shared__ int failed;
  constexpr uint32_t kBuf = buf_cols<P>();
  constexpr uint32_t kCols = 2 * kBuf;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int mt = blockIdx.x, nt = blockIdx.y;
  if (sym) {
    // block b of the upper triangle of the T x T tile grid, row by row
    const int T = (A.rows + kT - 1) / kT;
    int b = blockIdx.x;
    mt = 0;
    while (b >= T - mt) { b -= T - mt; mt++; }
    nt = mt + b;
  }
  const int m0 = mt * kT, n0 = nt * kT;
  if (warp == 0) {
    tmem_alloc(&tbase, kCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    async::mbar_init(&bar_done[0], 1);
    async::mbar_init(&bar_done[1], 1);
    async::mbar_init_fence();
    failed = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tm = tbase;
  const uint32_t s0 = su32(smem);
  unsigned char *lobuf = smem + kStages * kStageBytes;
  // this thread's part of the tile: TMEM lane quarter warp % 4 (its row), the
  // half warp / 4 of the columns
  const int q = warp & 3, half = warp >> 2;
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;
  constexpr int kHalf = kT / 2;
  float acc[kHalf];
#pragma unroll
  for (int u = 0; u < kHalf; u++) acc[u] = 0.0f;
  // adds accumulator b (one chunk's sums) into acc
  auto drain = [&](int b) {
#pragma unroll
    for (int cc = 0; cc < kHalf; cc += 16) {
      uint32_t v[16], w[16];
      tmem_ld16(tm + lane_off + b * kBuf + half * kHalf + cc, v);
      if (P == 3) tmem_ld16(tm + lane_off + b * kBuf + kT + half * kHalf + cc, w);
      tc_wait_ld();
#pragma unroll
      for (int u = 0; u < 16; u++)
        acc[cc + u] += P == 3 ? __uint_as_float(v[u]) + __uint_as_float(w[u]) : __uint_as_float(v[u]);
    }
  };
  const int nchunks = (K + kTK - 1) / kTK;
  // copies run kStages - 1 chunks ahead (an empty group keeps the count even)
#pragma unroll
  for (int c = 0; c < kStages - 1; c++) {
    if (c < nchunks) {
      copy_chunk(A, m0, c * kTK, K, s0 + c * kStageBytes);
      copy_chunk(B, n0, c * kTK, K, s0 + c * kStageBytes + kPart);
    }
    cp_commit();
  }
  int issued = 0;  // chunks whose MMAs were issued (thread 0)
  for (int c = 0; c < nchunks; c++) {
    const int st = c % kStages, b = c & 1;
    cp_wait<kStages - 2>();  // chunk c has landed (this thread's copies)
    fence_async_smem();
    __syncthreads();
    if (P == 3) {
      form_lo(smem + st * kStageBytes, lobuf + b * kStageBytes);
      fence_async_smem();
      __syncthreads();
    }
    if (failed) break;
    // chunk c into accumulator b (drained in the previous iteration)
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = s0 + st * kStageBytes, b0 = a0 + kPart;
      const uint32_t al0 = su32(lobuf) + b * kStageBytes, bl0 = al0 + kPart;
      const uint32_t idesc = idesc_tf32(kT, kT);
      const uint32_t dst = tm + b * kBuf;
#pragma unroll
      for (int s = 0; s < kTK / 8; s++) {
        const uint32_t ac = s > 0 ? 1u : 0u;
        const uint64_t ah = smem_desc(a0 + s * 4096, 2048, 128), bh = smem_desc(b0 + s * 4096, 2048, 128);
        mma_tf32_ss(dst, ah, bh, idesc, ac);
        if (P == 3) {
          const uint64_t al = smem_desc(al0 + s * 4096, 2048, 128), bl = smem_desc(bl0 + s * 4096, 2048, 128);
          mma_tf32_ss(dst + kT, ah, bl, idesc, ac);
          mma_tf32_ss(dst + kT, al, bh, idesc, 1u);
        }
      }
      mma_commit(&bar_done[b]);
      issued = c + 1;
    }
    // chunk c - 1 done: drain its accumulator, refill its stage
    if (c >= 1) {
      if (!async::mbar_wait(&bar_done[b ^ 1], (unsigned)((c - 1) >> 1) & 1)) atomicOr(&failed, 1);
      tc_fence_after();
      if (!failed) drain(b ^ 1);
      tc_fence_before();
    }
    const int cn = c + kStages - 1;
    if (cn < nchunks) {
      const uint32_t dn = s0 + (cn % kStages) * kStageBytes;
      copy_chunk(A, m0, cn * kTK, K, dn);
      copy_chunk(B, n0, cn * kTK, K, dn + kPart);
    }
    cp_commit();
  }
  cp_wait<0>();
  __shared__ int last;
  if (tid == 0) last = issued;
  __syncthreads();
  bool ok = !failed && last == nchunks;
  // the last chunk's sums
  if (last > 0) {
    const int c = last - 1;
    if (!async::mbar_wait(&bar_done[c & 1], (unsigned)(c >> 1) & 1)) ok = false;
    tc_fence_after();
    if (ok) drain(c & 1);
  }
  if (!ok) {
    if (tid == 0) atomicOr(status, ERR_GEMM);
  } else {
    const int m = m0 + 32 * q + lane;
    if (m < A.rows) {
#pragma unroll
      for (int u = 0; u < kHalf; u++) {
        const int n = n0 + half * kHalf + u;
        if (n < B.rows) {
          float *o = D + (int64_t)m * d_sm + (int64_t)n * d_sn;
          *o = beta ? fmaf(alpha, acc[u], *o) : alpha * acc[u];
          if (sym && nt > mt) {
            float *t = D + (int64_t)n * d_sm + (int64_t)m * d_sn;
            *t = beta ? fmaf(alpha, acc[u], *t) : alpha * acc[u];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, kCols);
}

template <int P>
cudaError_t run(const Operand &A, const Operand &B, int K, float *D, int64_t d_sm, int64_t d_sn, float alpha,
                int beta, int *status, cudaStream_t s) {
  constexpr int bytes = smem_bytes<P>();
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  const int T = (A.rows + kT - 1) / kT;
  const int sym = (A.p == B.p && A.sr == B.sr && A.rows == B.rows) ? 1 : 0;
  const dim3 grid = sym ? dim3(T * (T + 1) / 2, 1) : dim3(T, (B.rows + kT - 1) / kT);
  k_gemm_tc<P><<<grid, kThreads, bytes, s>>>(A, B, K, D, d_sm, d_sn, alpha, beta, sym, status);
  return cudaGetLastError();
}

// XT[i + r * ldt] = X[r + i * rows] (32 x 32 tiles through shared memory)
__global__ void k_transpose(const float *__restrict__ X, int64_t rows, int k, float *__restrict__ XT, int64_t ldt) {
  __shared__ float t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int i0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t r = r0 + threadIdx.x;
    const int i = i0 + y;
    t[y][threadIdx.x] = (r < rows && i < k) ? X[r + (int64_t)i * rows] : 0.0f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int i = i0 + threadIdx.x;
    const int64_t r = r0 + y;
    if (r < rows && i < k) XT[i + r * ldt] = t[threadIdx.x][y];
  }
}

// Y[r + i * ldy] = X[r + i * rows]
__global__ void k_pad_copy(const float *__restrict__ X, int64_t rows, int k, float *__restrict__ Y, int64_t ldy) {
  const int i = blockIdx.y;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
    Y[r + (int64_t)i * ldy] = X[r + (int64_t)i * rows];
}

bool aligned_operand(const float *p, int64_t sr) { return p && sr % 4 == 0 && ((uintptr_t)p % 16) == 0; }

}  // namespace

cudaError_t launch_gemm_tc(int passes, const float *A, int64_t a_sr, const float *B, int64_t b_sr, int M, int N,
                           int K, float *D, int64_t d_sm, int64_t d_sn, float alpha, int beta, int *status,
                           cudaStream_t s) {
  if ((passes != 1 && passes != 3) || !aligned_operand(A, a_sr) || !aligned_operand(B, b_sr) || !D || !status ||
      M < 1 || N < 1 || K < 1)
    return cudaErrorInvalidValue;
  const Operand oa{A, a_sr, M}, ob{B, b_sr, N};
  return passes == 3 ? run<3>(oa, ob, K, D, d_sm, d_sn, alpha, beta, status, s)
                     : run<1>(oa, ob, K, D, d_sm, d_sn, alpha, beta, status, s);
}

void reorth32_workspace(int64_t rows, int k, size_t *e_floats, size_t *w_floats) {
  const int64_t kp = (k + 3) / 4 * 4, rp = (rows + 3) / 4 * 4;
  *e_floats = (size_t)(kp * k);
  *w_floats = (size_t)std::max(rp * k, kp * rows);
}

cudaError_t launch_transpose32(const float *X, int64_t rows, int k, float *XT, int64_t ldt, cudaStream_t s) {
  const dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((k + 31) / 32)), block(32, 8);
  k_transpose<<<grid, block, 0, s>>>(X, rows, k, XT, ldt);
  return cudaGetLastError();
}

cudaError_t launch_pad_copy32(const float *X, int64_t rows, int k, float *Y, int64_t ldy, cudaStream_t s) {
  const unsigned bx = (unsigned)std::min<int64_t>((rows + 255) / 256, 64);
  k_pad_copy<<<dim3(bx, (unsigned)k), 256, 0, s>>>(X, rows, k, Y, ldy);
  return cudaGetLastError();
}

}  // namespace bdu
