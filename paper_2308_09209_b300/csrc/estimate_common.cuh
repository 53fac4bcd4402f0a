// Device helpers shared by the colour-estimate kernels (the per-frame
// estimate and the batched pair labeller).
#pragma once

#include "stitch_internal.h"

namespace stitch {
namespace est {

// Inclusive prefix sum of 256 uint32 values by one warp (8 per lane).
__device__ __forceinline__ void warp_scan256(const uint32_t *__restrict__ in, uint32_t *out) {
  const int lane = threadIdx.x & 31;
  const uint4 a = *reinterpret_cast<const uint4 *>(in + 8 * lane);
  const uint4 b = *reinterpret_cast<const uint4 *>(in + 8 * lane + 4);
  uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
  for (int k = 1; k < 8; ++k) v[k] += v[k - 1];
  uint32_t run = v[7];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, run, o);
    if (lane >= o) run += t;
  }
  const uint32_t base = run - v[7];
#pragma unroll
  for (int k = 0; k < 8; ++k) out[8 * lane + k] = v[k] + base;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// M = A^-1 B for a symmetric 3x3 A by nine lanes of one warp (lane e = 3r + c
// holds entry (r, c)): cofactors, determinant by the first row, inverse =
// adjugate / det, then M = A^-1 B. Returns (in every lane) false if det is
// zero or not finite, or cond_1(A) = |A|_1 |A^-1|_1 exceeds kCondLimit (NaN
// counts as ill-conditioned). Lanes 9..31 take part in the shuffles only.
__device__ __forceinline__ bool warp_solve3(double a, double b, double &m) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int e = lane < 9 ? lane : 0;
  const int r = e / 3, c = e % 3;
  // cofactor of (r, c): rows r1 < r2 != r, columns c1 < c2 != c
  const int r1 = r == 0 ? 1 : 0, r2 = r == 2 ? 1 : 2;
  const int c1 = c == 0 ? 1 : 0, c2 = c == 2 ? 1 : 2;
  const double a11 = __shfl_sync(full, a, r1 * 3 + c1), a12 = __shfl_sync(full, a, r1 * 3 + c2);
  const double a21 = __shfl_sync(full, a, r2 * 3 + c1), a22 = __shfl_sync(full, a, r2 * 3 + c2);
  double cof = a11 * a22 - a12 * a21;
  if ((r + c) & 1) cof = -cof;
  // det by the first row: sum_c A(0,c) C(0,c)
  const double p = (lane < 3) ? a * cof : 0.0;
  double det = p + __shfl_sync(full, p, 1) + __shfl_sync(full, p, 2);
  det = __shfl_sync(full, det, 0);
  const bool ok_det = det != 0.0 && isfinite(det);
  const double inv_det = ok_det ? 1.0 / det : 0.0;
  // A^-1 = adj(A) / det, adj = cofactor matrix transposed
  const double ai = __shfl_sync(full, cof, c * 3 + r) * inv_det;
  // 1-norms: maximum absolute column sum
  double ca = fabs(a), ci = fabs(ai);
  ca += __shfl_sync(full, ca, (e + 3) % 9) + __shfl_sync(full, ca, (e + 6) % 9);
  ci += __shfl_sync(full, ci, (e + 3) % 9) + __shfl_sync(full, ci, (e + 6) % 9);
  const double nA = fmax(fmax(__shfl_sync(full, ca, 0), __shfl_sync(full, ca, 1)), __shfl_sync(full, ca, 2));
  const double nI = fmax(fmax(__shfl_sync(full, ci, 0), __shfl_sync(full, ci, 1)), __shfl_sync(full, ci, 2));
  // M(r, c) = sum_k A^-1(r, k) B(k, c)
  double mm = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) mm += __shfl_sync(full, ai, r * 3 + k) * __shfl_sync(full, b, k * 3 + c);
  m = mm;
  const double cond = nA * nI;
  return ok_det && cond <= kCondLimit;
}

// Chain the pair matrices to the reference camera (row-vector convention of
// Eq. 4): M_ref = I, M_k = M_pair(k) . M_(k+1) left of the reference and
// M_k = M_pair(k-1) . M_(k-1) right of it. Called by one whole warp; lane
// e < 9 computes entry e of each camera in turn.
__device__ __forceinline__ void warp_chain(const double (*M_pair)[9], double (*M_cam)[9], int n, int ref) {
  const int e = threadIdx.x & 31, r = e / 3, c = e % 3;
  if (e < 9) M_cam[ref][e] = (r == c) ? 1.0 : 0.0;
  __syncwarp();
  for (int k = ref - 1; k >= 0; --k) {
    if (e < 9)
      M_cam[k][e] = M_pair[k][r * 3 + 0] * M_cam[k + 1][0 * 3 + c] + M_pair[k][r * 3 + 1] * M_cam[k + 1][1 * 3 + c] +
                    M_pair[k][r * 3 + 2] * M_cam[k + 1][2 * 3 + c];
    __syncwarp();
  }
  for (int k = ref + 1; k < n; ++k) {
    if (e < 9)
      M_cam[k][e] = M_pair[k - 1][r * 3 + 0] * M_cam[k - 1][0 * 3 + c] +
                    M_pair[k - 1][r * 3 + 1] * M_cam[k - 1][1 * 3 + c] +
                    M_pair[k - 1][r * 3 + 2] * M_cam[k - 1][2 * 3 + c];
    __syncwarp();
  }
}

// (c, d) with c != d -> index into the value-weighted histograms
__device__ __forceinline__ int w_index(int c, int d) { return c * 2 + (d > c ? d - 1 : d); }

}  // namespace est
}  // namespace stitch
