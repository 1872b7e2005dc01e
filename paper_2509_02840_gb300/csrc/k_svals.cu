// Singular values of the upper bidiagonal Bd (d, e) on the device, by
// multisection with Sturm counts.
//
// The singular values of Bd are the nonnegative eigenvalues of the
// Golub-Kahan matrix T (order 2n, zero diagonal, off-diagonal
// b = d_1, e_1, d_2, e_2, ..., d_n), whose spectrum is {+-sigma_i}.  The
// number of eigenvalues of T below x is the number of negative pivots of
// the LDL^T factorization of T - x I: q_1 = -x, q_i = -x - b_{i-1}^2 / q_{i-1}
// (a zero pivot replaced by -pivmin), so for x > 0 the number of singular
// values below x is that count minus n.
//
// One warp per requested singular value; each iteration its 32 lanes count at
// 32 interior points of the current interval and the interval shrinks to the
// 1/33 that holds the value.  On GB300 a warp's FP64 instruction costs the same
// whatever its active lanes, so the 32 counts cost what one would.
#include "bdu_internal.cuh"

namespace bdu {
namespace {

__global__ void k_bidiag_svals(const double *__restrict__ b2, int n, double hi0, double pivmin, int k,
                               double *__restrict__ sv) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);  // the (j+1)-th largest value
  if (j >= k) return;  // whole warps exit together
  // #(sigma < x) >= n - j exactly when x lies above sigma_(j+1)
  const int target = n - j;
  double lo = 0.0, hi = hi0;
  for (int it = 0; it < 64; it++) {
    const double w = hi - lo;
    if (!(w > 2.2e-16 * hi)) break;  // uniform across the warp
    const double x = lo + w * (double)(lane + 1) / 33.0;
    int cnt = 0;
    double q = -x;
    cnt += q < 0.0;
    for (int i = 1; i < 2 * n; i++) {
      q = -x - b2[i - 1] / q;
      if (q == 0.0) q = -pivmin;
      cnt += q < 0.0;
    }
    // #(sigma < x) = cnt - n; the lanes with #(sigma < x) >= target lie above sigma_(j+1)
    const unsigned above = __ballot_sync(0xffffffffu, cnt - n >= target);
    const int first = above ? __ffs(above) - 1 : 32;
    const double nlo = first == 0 ? lo : lo + w * (double)first / 33.0;
    const double nhi = first == 32 ? hi : lo + w * (double)(first + 1) / 33.0;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) sv[j] = 0.5 * (lo + hi);
}

}  // namespace

// b2: the 2n-1 squared off-diagonal entries d_1^2, e_1^2, d_2^2, ..., d_n^2 of
// the Golub-Kahan matrix (device); sv: the k largest singular values,
// descending (device).  hi: an upper bound of sigma_max; pivmin: the smallest
// pivot magnitude used.
cudaError_t launch_bidiag_svals(const double *b2, int n, double hi, double pivmin, int k, double *sv,
                                cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  const int warps = 4;
  k_bidiag_svals<<<(k + warps - 1) / warps, 32 * warps, 0, s>>>(b2, n, hi, pivmin, k, sv);
  return cudaGetLastError();
}

}  // namespace bdu
