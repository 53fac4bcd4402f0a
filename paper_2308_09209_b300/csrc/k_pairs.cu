// Plain colour estimate of many independent overlap pairs, one block per pair
// (the labeller and feature builder of the learned estimator).
//
// A pair is two small packed-RGB patches: side i (the camera to correct) and
// side j (its reference neighbour). For each pair the block computes, with
// the same integer rules as the per-frame path (paper section 2.1 steps 2-4,
// Eq. 1-3 with a window of one frame; section 2.2 knots):
//   * histograms G_i, G_j, the value-weighted histograms of side i and the
//     Gram sums A = I_i^T I_i;
//   * the specification L of G_i onto G_j, B = I_i^T L(I_i) and M = A^-1 B
//     (float64, adjugate; ill-conditioned -> identity and a flag);
//   * the balance knot span (m2 - m1) / 255 per channel of the pooled
//     histogram G_i + G_j (the lambda-quantile knots of section 2.2; the
//     linear segment of Eq. 5 has slope (d2 - d1) / (m2 - m1)).
// Outputs: features (bfloat16, 1536 per pair: 256 G_i / n_i then 256 G_j /
// n_j, channel-major), targets (float32, 12: M - I row-major, then the three spans), the
// float64 M and the flag.
#include <cuda_bf16.h>

#include "estimate_common.cuh"
#include "stitch_internal.h"

namespace stitch {

namespace {

using namespace est;

constexpr int kPT = 256;

__global__ void __launch_bounds__(kPT) k_pair_label(const PairParams P) {
  const int pair = blockIdx.x;
  const int npx = P.pw * P.ph;
  const uint8_t *__restrict__ pi = P.pairs + (size_t)pair * 2 * npx * 3;
  const uint8_t *__restrict__ pj = pi + (size_t)npx * 3;
  __shared__ __align__(16) uint32_t Hi[768];
  __shared__ __align__(16) uint32_t Hj[768];
  __shared__ __align__(16) uint32_t Hp[768];
  __shared__ __align__(16) uint32_t Wv[1536];
  __shared__ __align__(16) uint32_t cdf[9][256];   // i (3), j (3), pooled (3)
  __shared__ uint8_t L[3][256];
  __shared__ unsigned long long sA[6];
  __shared__ unsigned long long sB[9];
  __shared__ double sM[9];
  __shared__ int knot[3][2];
  __shared__ int ok_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int i = tid; i < 768; i += kPT) Hi[i] = Hj[i] = 0u;
  for (int i = tid; i < 1536; i += kPT) Wv[i] = 0u;
  if (tid < 6) sA[tid] = 0ull;
  __syncthreads();

  unsigned long long a[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
  for (int k = tid; k < npx; k += kPT) {
    const uint32_t r = pi[3 * k], g = pi[3 * k + 1], b = pi[3 * k + 2];
    atomicAdd(&Hi[r], 1u);
    atomicAdd(&Hi[256 + g], 1u);
    atomicAdd(&Hi[512 + b], 1u);
    atomicAdd(&Wv[0 * 256 + g], r);
    atomicAdd(&Wv[1 * 256 + b], r);
    atomicAdd(&Wv[2 * 256 + r], g);
    atomicAdd(&Wv[3 * 256 + b], g);
    atomicAdd(&Wv[4 * 256 + r], b);
    atomicAdd(&Wv[5 * 256 + g], b);
    a[0] += r * r; a[1] += r * g; a[2] += r * b; a[3] += g * g; a[4] += g * b; a[5] += b * b;
    const uint32_t rj = pj[3 * k], gj = pj[3 * k + 1], bj = pj[3 * k + 2];
    atomicAdd(&Hj[rj], 1u);
    atomicAdd(&Hj[256 + gj], 1u);
    atomicAdd(&Hj[512 + bj], 1u);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const unsigned long long s = warp_sum(a[k]);
    if (lane == 0 && s) atomicAdd(&sA[k], s);
  }
  __syncthreads();
  for (int i = tid; i < 768; i += kPT) Hp[i] = Hi[i] + Hj[i];
  __syncthreads();
  for (int q = warp; q < 9; q += kPT / 32) {
    const uint32_t *src = q < 3 ? Hi + 256 * q : (q < 6 ? Hj + 256 * (q - 3) : Hp + 256 * (q - 6));
    warp_scan256(src, cdf[q]);
  }
  __syncthreads();
  // specification of G_i onto G_j
  const unsigned long long ni = cdf[0][255], nj = cdf[3][255];
  for (int i = tid; i < 768; i += kPT) {
    const int c = i / 256, v = i % 256;
    int Lv = v;
    if (ni != 0ull && nj != 0ull) {
      const unsigned long long need = (unsigned long long)cdf[c][v] * nj;
      int lo = 0, hi = 255;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((unsigned long long)cdf[3 + c][mid] * ni >= need) hi = mid; else lo = mid + 1;
      }
      Lv = lo;
    }
    L[c][v] = (uint8_t)Lv;
  }
  // knots of the pooled histogram
  {
    const unsigned long long N = cdf[6][255];
    const unsigned long long lo = (unsigned long long)P.lambda_q * N;
    const unsigned long long hi = (unsigned long long)(1000000 - P.lambda_q) * N;
    for (int i = tid; i < 768; i += kPT) {
      const int c = i / 256, v = i % 256;
      const unsigned long long cur = 1000000ull * cdf[6 + c][v];
      const unsigned long long prev = v ? 1000000ull * cdf[6 + c][v - 1] : 0ull;
      if (cur >= lo && (v == 0 || prev < lo)) knot[c][0] = v;
      if (cur >= hi && (v == 0 || prev < hi)) knot[c][1] = v;
    }
  }
  __syncthreads();
  // B entries, one warp each
  for (int q = warp; q < 9; q += kPT / 32) {
    const int c = q / 3, d = q % 3;
    unsigned long long s = 0ull;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int v = 8 * lane + k;
      const unsigned long long Ld = L[d][v];
      s += (c == d) ? Ld * (unsigned long long)v * Hi[256 * d + v] : Ld * (unsigned long long)Wv[256 * w_index(c, d) + v];
    }
    s = warp_sum(s);
    if (lane == 0) sB[q] = s;
  }
  __syncthreads();
  if (warp == 0) {
    static const int sym[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
    const int e = lane < 9 ? lane : 0;
    double m = 0.0;
    const bool ok = warp_solve3((double)sA[sym[e]], (double)sB[e], m) && ni != 0ull && nj != 0ull;
    if (lane < 9) sM[lane] = ok ? m : ((lane % 4 == 0) ? 1.0 : 0.0);
    if (lane == 0) ok_flag = ok ? 0 : 1;
  }
  __syncthreads();
  // outputs
  // (H * 256) / n in float64, then float32, then bfloat16 (each rounding to nearest even)
  __nv_bfloat16 *f = P.feat + (size_t)pair * 1536;
  for (int i = tid; i < 768; i += kPT) {
    const double fi = ni ? ((double)Hi[i] * 256.0) / (double)ni : 0.0;
    const double fj = nj ? ((double)Hj[i] * 256.0) / (double)nj : 0.0;
    f[i] = __float2bfloat16_rn(__double2float_rn(fi));
    f[768 + i] = __float2bfloat16_rn(__double2float_rn(fj));
  }
  if (tid < 9) {
    P.targ[(size_t)pair * 12 + tid] = (float)(sM[tid] - ((tid % 4 == 0) ? 1.0 : 0.0));
    if (P.M) P.M[(size_t)pair * 9 + tid] = sM[tid];
  }
  if (tid >= 32 && tid < 35) {
    const int c = tid - 32;
    P.targ[(size_t)pair * 12 + 9 + c] = (float)(knot[c][1] - knot[c][0]) / 255.0f;
  }
  if (tid == 64 && P.flags) P.flags[pair] = ok_flag;
}

}  // namespace

cudaError_t launch_pair_label(const PairParams &p, cudaStream_t s) {
  if (p.n <= 0) return cudaSuccess;
  k_pair_label<<<p.n, kPT, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace stitch
