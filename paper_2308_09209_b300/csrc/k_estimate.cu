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
#include "estimate_common.cuh"

namespace stitch {

namespace {

using namespace est;

constexpr int kT = 1024;

// One entry of the output table: the fused, clamped value x = n / 16 through
// the balance curve F (Eq. 5, as read for the oracle: linear between the
// knots, the gamma tails outside them, identity for a degenerate span or with
// the balance off), clamped to [0, 255] and rounded half to even.
__device__ __forceinline__ uint32_t lut_entry(const Curve &cv, bool off, int n) {
  const float x = fminf((float)n * (1.0f / 16.0f), 255.0f);
  float F = x;
  if (!off && cv.ident == 0.0f) {
    F = cv.d1 + cv.s * (x - cv.m1);
    if (cv.m1 > 0.0f && x < cv.m1) F = cv.d1 * powf(x * cv.inv_m1, cv.g1);
    if (cv.m2 < 255.0f && x > cv.m2) F = 255.0f - (255.0f - cv.d2) * powf((255.0f - x) * cv.inv_bm, cv.g2);
  }
  return (uint32_t)__float2int_rn(fminf(fmaxf(F, 0.0f), 255.0f));
}

// The three channel tables (kLutEntries bytes each), four entries per store.
__device__ void write_lut(const Curve *cv, bool off, uint8_t *lut) {
  uint32_t *L = reinterpret_cast<uint32_t *>(lut);
  for (int i = threadIdx.x; i < kLutBytes / 4; i += blockDim.x) {
    const int c = (4 * i) / kLutEntries, n = (4 * i) % kLutEntries;
    L[i] = lut_entry(cv[c], off, n) | (lut_entry(cv[c], off, n + 1) << 8) | (lut_entry(cv[c], off, n + 2) << 16) |
           (lut_entry(cv[c], off, n + 3) << 24);
  }
}
constexpr int kWarps = kT / 32;
constexpr int kScanTasksMax = kMaxPairs * 6 + 3;

struct EstSmem {
  uint32_t cdf[kScanTasksMax][256];   // task q: pair q/6, side (q%6)/3 (0 = i, 1 = j), channel q%3; last 3: pooled
  uint8_t L[kMaxPairs][3][256];
  double M_pair[kMaxPairs][9];
  double M_cam[kMaxCams][9];
  int knot[3][2];
  int sing;
  Curve curve[3];
};

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
  // Balance on the stitched image: the knots come from the pre-balance
  // histogram of frame T - 1's panorama (none for frame 0).
  const bool out_mode = (P.flags & STITCH_BALANCE_OUTPUT) && P.out_hist;
  const uint32_t *ohist = (out_mode && T > 0) ? P.out_hist + ((T - 1) & 1) * 768 : nullptr;

  // 1. All prefix sums at once, one warp per histogram.
  for (int q = warp; q < n_scan; q += kWarps) {
    const uint32_t *src;
    if (q < np * 6) {
      const int p = q / 6, side = (q % 6) / 3, c = q % 3;
      src = side == 0 ? raw->Hi[p][c] : raw->Hj[p][c];
    } else {
      src = ohist ? ohist + (q - np * 6) * 256 : raw->pooled[q - np * 6];
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
  if (tid >= kT / 2 && tid < kT / 2 + np) {
    const int p = tid - kT / 2;
    S->n_ring[ring][p][0] = (int)sm.cdf[p * 6][255];
    S->n_ring[ring][p][1] = (int)sm.cdf[p * 6 + 3][255];
  }
  __syncthreads();

  // 4. Windowed solve, one warp per pair (nine lanes hold the matrix entries).
  if (warp < np) {
    const int p = warp;
    const int e = lane < 9 ? lane : 0;
    const int r = e / 3, c = e % 3;
    static const int sym[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
    const int nw = min(T + 1, P.window);
    unsigned long long As = 0ull, Bs = 0ull;
    int empty = 0;
    for (int i = 0; i < nw; ++i) {
      const int sl = (T - i) % kMaxWindow;
      As += S->A_ring[sl][p][sym[e]];
      Bs += S->B_ring[sl][p][e];
      empty |= (S->n_ring[sl][p][0] == 0 || S->n_ring[sl][p][1] == 0);
    }
    (void)r;
    (void)c;
    double m = 0.0;
    const bool ok = warp_solve3((double)As, (double)Bs, m) && !empty;
    if (ok) {
      if (lane < 9) sm.M_pair[p][lane] = m;
    } else if (lane == 0) {
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
    const int n = P.n_cams;
    warp_chain(sm.M_pair, sm.M_cam, n, P.ref);
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
    // with the stitched image's histogram, frame 0 (no predecessor) and an
    // empty histogram leave the frame unbalanced
    const bool no_hist = out_mode && (!ohist || sm.cdf[np * 6][255] == 0u);
    if (!no_hist) {
      S->knots[slot][c][0] = sm.knot[c][0];
      S->knots[slot][c][1] = sm.knot[c][1];
    }
    const int cnt = no_hist ? 1 : min(out_mode ? T : T + 1, kSmoothFrames);
    long long s1 = 0, s2 = 0;
    for (int i = no_hist ? -1 : cnt - 1; i >= 0; --i) {   // unbalanced: both knot means 0, as the oracle's
      const int sl = (T - i) % kSmoothFrames;
      s1 += (sl == slot) ? sm.knot[c][0] : S->knots[sl][c][0];
      s2 += (sl == slot) ? sm.knot[c][1] : S->knots[sl][c][1];
    }
    // Float32 throughout: the fuse kernel reads float32 parameters, and the
    // knot means of integer sums are correctly rounded either way.
    const float m1 = (float)s1 / (float)cnt;
    const float m2 = (float)s2 / (float)cnt;
    S->knot_mean[c][0] = m1;
    S->knot_mean[c][1] = m2;
    const float lam = (float)((double)P.lambda_q / 1e6);
    const float d1 = (float)(255.0 * ((double)P.lambda_q / 1e6));
    const float d2 = (float)(255.0 * (1.0 - (double)P.lambda_q / 1e6));
    (void)lam;
    const bool ident = no_hist || (m2 - m1) < 1.0f;
    const float span = ident ? 1.0f : (m2 - m1);
    const float sl = (d2 - d1) / span;
    Curve cv;
    cv.m1 = m1;
    cv.m2 = m2;
    cv.d1 = d1;
    cv.d2 = d2;
    cv.s = sl;
    cv.g1 = sl * m1 / d1;
    cv.g2 = sl * (255.0f - m2) / (255.0f - d2);
    cv.inv_m1 = m1 > 0.0f ? 1.0f / m1 : 0.0f;
    cv.inv_bm = m2 < 255.0f ? 1.0f / (255.0f - m2) : 0.0f;
    cv.ident = ident ? 1.0f : 0.0f;
    S->out[T % kColorSlots].curve[c] = cv;
    sm.curve[c] = cv;
  } else if (warp >= 2) {
    // 7. Clear the slot of frame T - 1 (already consumed): the stats pass of
    //    frame T + raw_slots - 1 accumulates into it. Warps 2..31 only, so the
    //    index tid - 64 starts at 0.
    uint4 *z = reinterpret_cast<uint4 *>(P.raw + ((T + P.raw_slots - 1) % P.raw_slots));
    const int n16 = (int)(sizeof(RawStats) / 16);
    for (int i = tid - 64; i < n16; i += kT - 64) z[i] = make_uint4(0u, 0u, 0u, 0u);
    // the stitched image's histogram just consumed: frame T + 1's fuse
    // accumulates into this slot
    if (ohist)
      for (int i = tid - 64; i < 768 / 4; i += kT - 64) reinterpret_cast<uint4 *>(const_cast<uint32_t *>(ohist))[i] =
          make_uint4(0u, 0u, 0u, 0u);
  }
  __syncthreads();
  // 8. The output table of this frame's curve (read by the fuse kernels).
  if (P.lut) write_lut(sm.curve, (P.flags & STITCH_BALANCE_OFF) != 0, P.lut + (size_t)(T % kColorSlots) * kLutBytes);
  if (tid == 0) S->T = T + 1;
}

__global__ void __launch_bounds__(256) k_curve_lut(const ColorOut *slot, int flags, uint8_t *lut) {
  __shared__ Curve cv[3];
  if (threadIdx.x < 3) cv[threadIdx.x] = slot->curve[threadIdx.x];
  __syncthreads();
  write_lut(cv, (flags & STITCH_BALANCE_OFF) != 0, lut);
}

}  // namespace

// Once per device, outside any stream capture: the block uses ~53 KB of
// dynamic shared memory.
cudaError_t estimate_setup() {
  return cudaFuncSetAttribute(k_estimate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(EstSmem));
}

// The estimate is one block on the critical path of every frame: launch it at
// the device's highest priority so that it gets the next free SM ahead of the
// many blocks of the throughput kernels running beside it.
cudaError_t launch_estimate(const EstimateParams &p, cudaStream_t s) {
  static_assert(sizeof(RawStats) % 16 == 0, "raw statistics must be a whole number of 16-byte words");
  int least = 0, greatest = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1);
  cfg.blockDim = dim3(kT);
  cfg.dynamicSmemBytes = sizeof(EstSmem);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = greatest;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_estimate, p);
}

cudaError_t launch_curve_lut(const ColorOut *slot, int flags, uint8_t *lut, cudaStream_t s) {
  k_curve_lut<<<1, 256, 0, s>>>(slot, flags, lut);
  return cudaGetLastError();
}

}  // namespace stitch
