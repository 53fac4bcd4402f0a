// K2 -- colour estimate of frame T, one thread block (paper section 2.1 steps
// 3-5, Eq. 1-4; section 2.2, Eq. 5-7).
//
// Per adjacent pair (i = colour-source camera, j = its neighbour toward the
// reference camera):
//   * histogram specification of G_i onto G_j (step 3): L_c(v) is the
//     smallest level u with CDF_j,c(u) * n_i >= CDF_i,c(v) * n_j, exact in
//     64-bit integers (one thread per level, binary search);
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
// Finally the other raw-statistics slot is cleared for the next frame and the
// frame index advances.
#include "stitch_internal.h"

namespace stitch {

namespace {

constexpr int kT = kEstimateThreads;  // one thread per histogram level
constexpr int kW = kT / 32;

__device__ __forceinline__ unsigned long long block_scan_u64(unsigned long long v, unsigned long long *s_wt) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) s_wt[wid] = v;
  __syncthreads();
  unsigned long long add = 0ull;
  for (int i = 0; i < wid; ++i) add += s_wt[i];
  __syncthreads();
  return v + add;
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

__device__ __forceinline__ void mat3_mul(const double *X, const double *Y, double *Z) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      Z[r * 3 + c] = X[r * 3 + 0] * Y[0 * 3 + c] + X[r * 3 + 1] * Y[1 * 3 + c] + X[r * 3 + 2] * Y[2 * 3 + c];
}

// (c, d) with c != d -> index into the value-weighted histograms
__device__ __forceinline__ int w_index(int c, int d) { return c * 2 + (d > c ? d - 1 : d); }

__global__ void __launch_bounds__(kT) k_estimate(const EstimateParams P) {
  ColorState *S = P.state;
  const int T = S->T;
  RawStats *raw = P.raw + (T & 1);
  const int v = threadIdx.x;
  const int lane = v & 31, wid = v >> 5;
  const int ring = T % kMaxWindow;

  __shared__ unsigned long long s_ci[3][256];
  __shared__ unsigned long long s_cj[3][256];
  __shared__ int s_L[3][256];
  __shared__ unsigned long long s_wt[kW];
  __shared__ unsigned long long s_red[9][kW];
  __shared__ int s_knot[3][2];
  __shared__ int s_sing;

  if (v == 0) s_sing = 0;

  for (int p = 0; p < P.n_pairs; ++p) {
    for (int c = 0; c < 3; ++c) {
      const unsigned long long ci = block_scan_u64(raw->Hi[p][c][v], s_wt);
      const unsigned long long cj = block_scan_u64(raw->Hj[p][c][v], s_wt);
      s_ci[c][v] = ci;
      s_cj[c][v] = cj;
    }
    __syncthreads();
    const unsigned long long ni = s_ci[0][255], nj = s_cj[0][255];
    for (int c = 0; c < 3; ++c) {
      int L = v;
      if (ni != 0ull && nj != 0ull) {
        const unsigned long long need = s_ci[c][v] * nj;
        int lo = 0, hi = 255;                 // smallest u with cdf_j[u] * ni >= need
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (s_cj[c][mid] * ni >= need) hi = mid; else lo = mid + 1;
        }
        L = lo;
      }
      s_L[c][v] = L;
    }
    __syncthreads();
    unsigned long long part[9];
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) {
        const unsigned long long Ld = (unsigned long long)s_L[d][v];
        part[c * 3 + d] = (c == d) ? Ld * (unsigned long long)v * raw->Hi[p][d][v]
                                   : Ld * (unsigned long long)raw->Wv[p][w_index(c, d)][v];
      }
    for (int k = 0; k < 9; ++k) {
      const unsigned long long s = warp_sum(part[k]);
      if (lane == 0) s_red[k][wid] = s;
    }
    __syncthreads();
    if (v < 9) {
      unsigned long long s = 0ull;
      for (int k = 0; k < kW; ++k) s += s_red[v][k];
      S->B_ring[ring][p][v] = s;
    }
    if (v >= 16 && v < 22) S->A_ring[ring][p][v - 16] = raw->A[p][v - 16];
    if (v == 32) {
      S->n_ring[ring][p][0] = (int)ni;
      S->n_ring[ring][p][1] = (int)nj;
    }
    __syncthreads();
  }

  // Windowed solve, one thread per pair.
  if (v < P.n_pairs) {
    const int p = v;
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
    const bool ok = !empty && solve3(A, B, M);
    if (ok) {
      for (int k = 0; k < 9; ++k) S->M_pair[p][k] = M[k];
    } else {
      atomicOr(&s_sing, 1 << p);
    }
  }
  __syncthreads();

  // Chain the pair matrices to the reference camera.
  if (v == 0) {
    const int n = P.n_cams, r = P.ref;
    for (int k = 0; k < 9; ++k) S->M_cam[r][k] = (k % 4 == 0) ? 1.0 : 0.0;
    for (int k = r - 1; k >= 0; --k) mat3_mul(S->M_pair[k], S->M_cam[k + 1], S->M_cam[k]);
    for (int k = r + 1; k < n; ++k) mat3_mul(S->M_pair[k - 1], S->M_cam[k - 1], S->M_cam[k]);
    ColorOut &o = S->out[T & 1];
    for (int k = 0; k < n; ++k)
      for (int e = 0; e < 9; ++e) o.M[k][e] = (float)S->M_cam[k][e];
    S->singular_last = s_sing;
    if (s_sing) S->cond_word |= 1;
  }

  // Balance knots from the pooled histogram (exact integer quantile test).
  for (int c = 0; c < 3; ++c) s_ci[c][v] = block_scan_u64(raw->pooled[c][v], s_wt);
  __syncthreads();
  {
    const unsigned long long N = s_ci[0][255];
    const unsigned long long lo = (unsigned long long)P.lambda_q * N;
    const unsigned long long hi = (unsigned long long)(1000000 - P.lambda_q) * N;
    for (int c = 0; c < 3; ++c) {
      const unsigned long long cur = 1000000ull * s_ci[c][v];
      const unsigned long long prev = v ? 1000000ull * s_ci[c][v - 1] : 0ull;
      if (cur >= lo && (v == 0 || prev < lo)) s_knot[c][0] = v;
      if (cur >= hi && (v == 0 || prev < hi)) s_knot[c][1] = v;
    }
  }
  __syncthreads();
  if (v < 3) {
    const int c = v;
    const int slot = T % kSmoothFrames;
    S->knots[slot][c][0] = s_knot[c][0];
    S->knots[slot][c][1] = s_knot[c][1];
    const int cnt = min(T + 1, kSmoothFrames);
    long long s1 = 0, s2 = 0;
    for (int i = cnt - 1; i >= 0; --i) {
      const int sl = (T - i) % kSmoothFrames;
      s1 += S->knots[sl][c][0];
      s2 += S->knots[sl][c][1];
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
    S->out[T & 1].curve[c] = cv;
  }

  // Clear the other raw slot: the stats pass of frame T + 1 accumulates into it.
  {
    uint32_t *z = reinterpret_cast<uint32_t *>(P.raw + ((T + 1) & 1));
    const int words = (int)(sizeof(RawStats) / 4);
    for (int i = v; i < words; i += kT) z[i] = 0u;
  }
  __syncthreads();
  if (v == 0) S->T = T + 1;
}

}  // namespace

cudaError_t launch_estimate(const EstimateParams &p, cudaStream_t s) {
  k_estimate<<<1, kEstimateThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace stitch
