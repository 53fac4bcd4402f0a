// K2 -- colour estimate of frame T, one thread block (paper section 2.1 steps
// 3-5, Eq. 1-4; section 2.2, Eq. 5-7).
//
// Per adjacent pair (i = colour-source camera, j = its neighbour toward the
// reference camera):
//   * histogram specification of G_i onto G_j (step 3): L_c(v) is the
//     smallest level u with CDF_j,c(u) * n_i >= CDF_i,c(v) * n_j, exact in
//     64-bit integers (binary search per level);
//   * this frame's Eq. 3 terms A_T = I_i^T I_i and B_T = I_i^T L(I_i), B from
//     the value-weighted histograms of the stats pass, exact in 64-bit
//     integers, stored in a ring of the last STITCH_MAX_WINDOW frames;
//   * M = A^-1 B over the window's summed A and B (Eq. 2-3), float64 Gaussian
//     elimination with partial pivoting; a 1-norm condition number above 1e12
//     (or an empty overlap side) keeps the pair's previous M and raises the
//     singular condition.
// Then the pair matrices are chained to the reference camera (row-vector
// convention of Eq. 4), the lambda-quantile knots of the pooled histogram are
// found (exact integer test), averaged over the current and the last two
// frames (Eq. 6-7) and turned into the piecewise curve's parameters (Eq. 5).
// Finally the statistics slot of the previous frame is cleared for reuse and
// the frame index advances.
//
// Layout of the work: 1024 threads. Every 256-level prefix sum is done by one
// warp (8 levels per lane plus a shuffle scan), so all of a frame's scans run
// at once; the B sums are one warp each as well. Only the float64 solves (one
// thread per pair) and the short chain are serial.
#include "stitch_internal.h"

namespace stitch {

namespace {

constexpr int kT = 1024;
constexpr int kWarps = kT / 32;
constexpr int kScanTasksMax = kMaxPairs * 6 + 3;

struct EstSmem {
  uint32_t cdf[kScanTasksMax][256];   // task q: pair q/6, side (q%6)/3 (0 = i, 1 = j), channel q%3; last 3: pooled
  uint8_t L[kMaxPairs][3][256];
  double M_pair[kMaxPairs][9];
  double M_cam[kMaxCams][9];
  int knot[3][2];
  int sing;
};

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

// Gaussian elimination with partial pivoting on [A | B | I]. Returns false if
// a pivot vanishes or cond_1(A) > kCondLimit (NaN counts as ill-conditioned).
__device__ bool solve3(const double A[9], const double B[9], double M[9]) {
  double a[3][9];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) {
      a[r][c] = A[r * 3 + c];
      a[r][3 + c] = B[r * 3 + c];
      a[r][6 + c] = (r == c) ? 1.0 : 0.0;
    }
  }
  for (int k = 0; k < 3; ++k) {
    int piv = k;
    double best = fabs(a[k][k]);
    for (int r = k + 1; r < 3; ++r)
      if (fabs(a[r][k]) > best) { best = fabs(a[r][k]); piv = r; }
    if (!(best > 0.0)) return false;
    if (piv != k)
      for (int c = 0; c < 9; ++c) { const double t = a[k][c]; a[k][c] = a[piv][c]; a[piv][c] = t; }
    for (int r = k + 1; r < 3; ++r) {
      const double f = a[r][k] / a[k][k];
      for (int c = k; c < 9; ++c) a[r][c] -= f * a[k][c];
    }
  }
  for (int k = 2; k >= 0; --k) {
    for (int c = 3; c < 9; ++c) {
      double s = a[k][c];
      for (int j = k + 1; j < 3; ++j) s -= a[k][j] * a[j][c];
      a[k][c] = s / a[k][k];
    }
  }
  double nA = 0.0, nI = 0.0;
  for (int c = 0; c < 3; ++c) {
    double sa = 0.0, si = 0.0;
    for (int r = 0; r < 3; ++r) { sa += fabs(A[r * 3 + c]); si += fabs(a[r][6 + c]); }
    nA = fmax(nA, sa);
    nI = fmax(nI, si);
  }
  const double cond = nA * nI;
  if (!(cond <= kCondLimit)) return false;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) M[r * 3 + c] = a[r][3 + c];
  return true;
}

// (c, d) with c != d -> index into the value-weighted histograms
__device__ __forceinline__ int w_index(int c, int d) { return c * 2 + (d > c ? d - 1 : d); }

__global__ void __launch_bounds__(kT) k_estimate(const EstimateParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EstSmem &sm = *reinterpret_cast<EstSmem *>(smem_raw);
  ColorState *S = P.state;
  const int T = S->T;
  RawStats *raw = P.raw + (T % P.raw_slots);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ring = T % kMaxWindow;
  const int np = P.n_pairs;
  const int n_scan = np * 6 + 3;

  if (tid == 0) sm.sing = 0;
  if (tid < np * 9) sm.M_pair[tid / 9][tid % 9] = S->M_pair[tid / 9][tid % 9];

  // 1. All prefix sums at once, one warp per histogram.
  for (int q = warp; q < n_scan; q += kWarps) {
    const uint32_t *src;
    if (q < np * 6) {
      const int p = q / 6, side = (q % 6) / 3, c = q % 3;
      src = side == 0 ? raw->Hi[p][c] : raw->Hj[p][c];
    } else {
      src = raw->pooled[q - np * 6];
    }
    warp_scan256(src, sm.cdf[q]);
  }
  __syncthreads();

  // 2. Histogram specification of every pair and channel (binary search).
  for (int i = tid; i < np * 3 * 256; i += kT) {
    const int p = i / 768, c = (i / 256) % 3, v = i % 256;
    const uint32_t *ci = sm.cdf[p * 6 + c];
    const uint32_t *cj = sm.cdf[p * 6 + 3 + c];
    const unsigned long long ni = ci[255], nj = cj[255];
    int L = v;
    if (ni != 0ull && nj != 0ull) {
      const unsigned long long need = (unsigned long long)ci[v] * nj;
      int lo = 0, hi = 255;                  // smallest u with cdf_j[u] * ni >= need
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((unsigned long long)cj[mid] * ni >= need) hi = mid; else lo = mid + 1;
      }
      L = lo;
    }
    sm.L[p][c][v] = (uint8_t)L;
  }
  __syncthreads();

  // 3. This frame's B = sum_v L_d(v) W_cd(v) (c != d), sum_v L_d(v) v H_d(v) (c == d); one warp per entry.
  for (int q = warp; q < np * 9; q += kWarps) {
    const int p = q / 9, c = (q % 9) / 3, d = q % 3;
    unsigned long long s = 0ull;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int v = 8 * lane + k;
      const unsigned long long Ld = sm.L[p][d][v];
      s += (c == d) ? Ld * (unsigned long long)v * raw->Hi[p][d][v]
                    : Ld * (unsigned long long)raw->Wv[p][w_index(c, d)][v];
    }
    s = warp_sum(s);
    if (lane == 0) S->B_ring[ring][p][c * 3 + d] = s;
  }
  if (tid < np * 6) S->A_ring[ring][tid / 6][tid % 6] = raw->A[tid / 6][tid % 6];
  if (tid >= 512 && tid < 512 + np) {
    const int p = tid - 512;
    S->n_ring[ring][p][0] = (int)sm.cdf[p * 6][255];
    S->n_ring[ring][p][1] = (int)sm.cdf[p * 6 + 3][255];
  }
  __syncthreads();

  // 4. Windowed solve, one thread per pair.
  if (tid < np) {
    const int p = tid;
    const int nw = min(T + 1, P.window);
    unsigned long long As[6] = {0, 0, 0, 0, 0, 0}, Bs[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool empty = false;
    for (int i = 0; i < nw; ++i) {
      const int sl = (T - i) % kMaxWindow;
      for (int k = 0; k < 6; ++k) As[k] += S->A_ring[sl][p][k];
      for (int k = 0; k < 9; ++k) Bs[k] += S->B_ring[sl][p][k];
      if (S->n_ring[sl][p][0] == 0 || S->n_ring[sl][p][1] == 0) empty = true;
    }
    const double A[9] = {(double)As[0], (double)As[1], (double)As[2],
                         (double)As[1], (double)As[3], (double)As[4],
                         (double)As[2], (double)As[4], (double)As[5]};
    double B[9], M[9];
    for (int k = 0; k < 9; ++k) B[k] = (double)Bs[k];
    if (!empty && solve3(A, B, M)) {
      for (int k = 0; k < 9; ++k) sm.M_pair[p][k] = M[k];
    } else {
      atomicOr(&sm.sing, 1 << p);
    }
  }
  // 5. Knots of the pooled histogram (exact integer quantile test).
  {
    const uint32_t *cp0 = sm.cdf[np * 6];
    const unsigned long long N = cp0[255];
    const unsigned long long lo = (unsigned long long)P.lambda_q * N;
    const unsigned long long hi = (unsigned long long)(1000000 - P.lambda_q) * N;
    for (int i = tid; i < 3 * 256; i += kT) {
      const int c = i / 256, v = i % 256;
      const uint32_t *cp = sm.cdf[np * 6 + c];
      const unsigned long long cur = 1000000ull * cp[v];
      const unsigned long long prev = v ? 1000000ull * cp[v - 1] : 0ull;
      if (cur >= lo && (v == 0 || prev < lo)) sm.knot[c][0] = v;
      if (cur >= hi && (v == 0 || prev < hi)) sm.knot[c][1] = v;
    }
  }
  __syncthreads();

  // 6. Chain to the reference camera (warp 0, one lane per matrix entry) and
  //    the balance curve (warp 1, one lane per channel).
  if (warp == 0) {
    const int e = lane, r = e / 3, c = e % 3;
    const int n = P.n_cams, ref = P.ref;
    if (e < 9) sm.M_cam[ref][e] = (r == c) ? 1.0 : 0.0;
    __syncwarp();
    for (int k = ref - 1; k >= 0; --k) {
      if (e < 9)
        sm.M_cam[k][e] = sm.M_pair[k][r * 3 + 0] * sm.M_cam[k + 1][0 * 3 + c] +
                         sm.M_pair[k][r * 3 + 1] * sm.M_cam[k + 1][1 * 3 + c] +
                         sm.M_pair[k][r * 3 + 2] * sm.M_cam[k + 1][2 * 3 + c];
      __syncwarp();
    }
    for (int k = ref + 1; k < n; ++k) {
      if (e < 9)
        sm.M_cam[k][e] = sm.M_pair[k - 1][r * 3 + 0] * sm.M_cam[k - 1][0 * 3 + c] +
                         sm.M_pair[k - 1][r * 3 + 1] * sm.M_cam[k - 1][1 * 3 + c] +
                         sm.M_pair[k - 1][r * 3 + 2] * sm.M_cam[k - 1][2 * 3 + c];
      __syncwarp();
    }
    ColorOut &o = S->out[T % kColorSlots];
    for (int i = lane; i < n * 9; i += 32) {
      S->M_cam[i / 9][i % 9] = sm.M_cam[i / 9][i % 9];
      o.M[i / 9][i % 9] = (float)sm.M_cam[i / 9][i % 9];
    }
    for (int i = lane; i < np * 9; i += 32) S->M_pair[i / 9][i % 9] = sm.M_pair[i / 9][i % 9];
    if (lane == 0) {
      S->singular_last = sm.sing;
      if (sm.sing) S->cond_word |= 1;
    }
  } else if (warp == 1 && lane < 3) {
    const int c = lane;
    const int slot = T % kSmoothFrames;
    S->knots[slot][c][0] = sm.knot[c][0];
    S->knots[slot][c][1] = sm.knot[c][1];
    const int cnt = min(T + 1, kSmoothFrames);
    long long s1 = 0, s2 = 0;
    for (int i = cnt - 1; i >= 0; --i) {
      const int sl = (T - i) % kSmoothFrames;
      s1 += (sl == slot) ? sm.knot[c][0] : S->knots[sl][c][0];
      s2 += (sl == slot) ? sm.knot[c][1] : S->knots[sl][c][1];
    }
    const double m1 = (double)s1 / (double)cnt;
    const double m2 = (double)s2 / (double)cnt;
    S->knot_mean[c][0] = m1;
    S->knot_mean[c][1] = m2;
    const double lam = (double)P.lambda_q / 1e6;
    const double d1 = 255.0 * lam, d2 = 255.0 * (1.0 - lam);
    const bool ident = (m2 - m1) < 1.0;
    const double span = ident ? 1.0 : (m2 - m1);
    const double s = (d2 - d1) / span;
    const double g1 = s * m1 / d1;
    const double g2 = s * (255.0 - m2) / (255.0 - d2);
    Curve cv;
    cv.m1 = (float)m1;
    cv.m2 = (float)m2;
    cv.d1 = (float)d1;
    cv.d2 = (float)d2;
    cv.s = (float)s;
    cv.g1 = (float)g1;
    cv.g2 = (float)g2;
    cv.inv_m1 = m1 > 0.0 ? (float)(1.0 / m1) : 0.0f;
    cv.inv_bm = m2 < 255.0 ? (float)(1.0 / (255.0 - m2)) : 0.0f;
    cv.ident = ident ? 1.0f : 0.0f;
    S->out[T % kColorSlots].curve[c] = cv;
  } else if (warp >= 2) {
    // 7. Clear the slot of frame T - 1 (already consumed): the stats pass of
    //    frame T + raw_slots - 1 accumulates into it. Warps 2..31 only, so the
    //    index tid - 64 starts at 0.
    uint4 *z = reinterpret_cast<uint4 *>(P.raw + ((T + P.raw_slots - 1) % P.raw_slots));
    const int n16 = (int)(sizeof(RawStats) / 16);
    for (int i = tid - 64; i < n16; i += kT - 64) z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  __syncthreads();
  if (tid == 0) S->T = T + 1;
}

}  // namespace

// Once per device, outside any stream capture: the block uses ~53 KB of
// dynamic shared memory.
cudaError_t estimate_setup() {
  return cudaFuncSetAttribute(k_estimate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(EstSmem));
}

cudaError_t launch_estimate(const EstimateParams &p, cudaStream_t s) {
  static_assert(sizeof(RawStats) % 16 == 0, "raw statistics must be a whole number of 16-byte words");
  k_estimate<<<1, kT, sizeof(EstSmem), s>>>(p);
  return cudaGetLastError();
}

}  // namespace stitch
