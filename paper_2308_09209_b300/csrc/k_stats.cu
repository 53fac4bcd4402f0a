// K1 -- integer colour statistics of one frame (paper section 2.1 steps 2-4,
// Eq. 1-3 terms; section 2.2 histogram for the balance knots).
//
// Each block takes a band of rows of one camera frame, in groups of 16
// consecutive pixels (48 bytes, three 16-byte loads when the row is 16-byte
// aligned):
//   * first every pixel: its three channel values go to the pooled
//     full-frame histogram (section 2.2: the lambda-quantile knots);
//   * then the block's part of each of the camera's pair rectangles, read
//     again (from cache): the pixels go to that side's overlap histogram
//     (section 2.1 step 2); on the colour-source side i also to the value-
//     weighted histograms W_cd[x_d] += x_c (c != d) and to the Gram sums
//     x_c x_d. With these, the estimate kernel forms B = I_i^T L(I_i) without
//     a second pass over the pixels once the specification L is known:
//     B_cd = sum_v L_d(v) W_cd(v), B_dd = sum_v L_d(v) v H_i,d(v).
// Walking each rectangle separately keeps a warp's lanes on one kind of
// update (only a rectangle's edge groups test their pixels one by one).
// Counts are accumulated in shared memory and flushed with one global atomic
// per non-zero bin. All arithmetic is integer, so results are bit-exact.
#include "stitch_internal.h"

namespace stitch {

namespace {

constexpr int kPoolWords = 3 * 256;
constexpr int kRoleWords = 3 * 256 + 6 * 256;   // H then W

__device__ __forceinline__ uint32_t byte_of(const uint32_t (&w)[12], int j) {
  return (w[j >> 2] >> ((j & 3) * 8)) & 0xffu;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// The group's 48 bytes as 12 little-endian words (bytes past the row's
// npx pixels are 0).
__device__ __forceinline__ void load_group(const uint8_t *__restrict__ p, int npx, bool vec, uint32_t (&wd)[12]) {
  if (vec && npx == 16) {
    const uint4 q0 = __ldg(reinterpret_cast<const uint4 *>(p));
    const uint4 q1 = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
    const uint4 q2 = __ldg(reinterpret_cast<const uint4 *>(p) + 2);
    wd[0] = q0.x; wd[1] = q0.y; wd[2] = q0.z; wd[3] = q0.w;
    wd[4] = q1.x; wd[5] = q1.y; wd[6] = q1.z; wd[7] = q1.w;
    wd[8] = q2.x; wd[9] = q2.y; wd[10] = q2.z; wd[11] = q2.w;
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) wd[k] = 0u;
#pragma unroll
    for (int j = 0; j < 48; ++j)
      if (j < 3 * npx) wd[j >> 2] |= (uint32_t)__ldg(p + j) << ((j & 3) * 8);
  }
}

// Calls f(y, g) for every row y in [ya, yb) and group g in [ga, gb), the
// block's threads taking (row, group) pairs with a fixed stride; one integer
// division per call when a row has at most blockDim groups.
template <typename F>
__device__ __forceinline__ void span_walk(int ya, int yb, int ga, int gb, F &&f) {
  const int ng = gb - ga, nt = blockDim.x;
  if (ya >= yb || ng <= 0) return;
  if (ng <= nt) {
    const int rpi = nt / ng;
    int rr = (int)threadIdx.x / ng;
    const int g = ga + (int)threadIdx.x - rr * ng;
    if (rr >= rpi) return;
    for (int y = ya + rr; y < yb; y += rpi) f(y, g);
  } else {
    for (int i = threadIdx.x; i < (yb - ya) * ng; i += nt) {
      const int rr = i / ng;
      f(ya + rr, ga + i - rr * ng);
    }
  }
}

__global__ void __launch_bounds__(kStatsThreads) k_stats(const StatsParams P) {
  const int cam = blockIdx.y;
  if (cam >= P.n_cams) return;
  const int h = P.h[cam];
  const int w = P.w[cam];
  const int r0 = blockIdx.x * P.rows_per_block;
  if (r0 >= h) return;
  const int r1 = min(h, r0 + P.rows_per_block);

  extern __shared__ uint32_t sm[];
  uint32_t *s_pool = sm;
  uint32_t *s_role = sm + kPoolWords;  // [2][kRoleWords]
  unsigned long long *s_A = reinterpret_cast<unsigned long long *>(sm + kPoolWords + 2 * kRoleWords);  // [2][6]

  for (int i = threadIdx.x; i < kPoolWords + 2 * kRoleWords; i += blockDim.x) sm[i] = 0u;
  if (threadIdx.x < 12) s_A[threadIdx.x] = 0ull;

  RoleDev R[2];
  bool act[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    act[q] = false;
    if (q < P.n_roles[cam]) {
      R[q] = P.roles[cam][q];
      act[q] = R[q].ry0 < r1 && R[q].ry1 > r0 && R[q].rx1 > R[q].rx0;
    } else {
      R[q] = RoleDev{0, 0, 0, 0, 0, 0};
    }
  }
  __syncthreads();

  const uint8_t *__restrict__ src = P.src[cam];
  const int pitch = P.pitch[cam];
  const int groups = (w + 15) >> 4;
  const bool vec = P.vec_ok[cam] != 0;

  // A camera is the colour-source side of at most one pair: role iq (or -1).
  const int iq = (act[0] && R[0].is_i) ? 0 : ((act[1] && R[1].is_i) ? 1 : -1);
  unsigned long long acc[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};

  // Pass 1, every pixel of rows [r0, r1): the pooled histogram.
  span_walk(r0, r1, 0, groups, [&](int y, int g) {
    const int x0 = g << 4;
    const int npx = min(16, w - x0);
    uint32_t wd[12];
    load_group(src + (size_t)y * pitch + 3 * x0, npx, vec, wd);
    if (npx == 16) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        atomicAdd(&s_pool[byte_of(wd, 3 * i)], 1u);
        atomicAdd(&s_pool[256 + byte_of(wd, 3 * i + 1)], 1u);
        atomicAdd(&s_pool[512 + byte_of(wd, 3 * i + 2)], 1u);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (i < npx) {
          atomicAdd(&s_pool[byte_of(wd, 3 * i)], 1u);
          atomicAdd(&s_pool[256 + byte_of(wd, 3 * i + 1)], 1u);
          atomicAdd(&s_pool[512 + byte_of(wd, 3 * i + 2)], 1u);
        }
      }
    }
  });

  // Pass 2, each rectangle's part of the block: overlap histograms, and on
  // side i the value-weighted histograms and the Gram sums.
#pragma unroll 1
  for (int q = 0; q < 2; ++q) {
    if (!act[q]) continue;
    const int ya = max(r0, R[q].ry0), yb = min(r1, R[q].ry1);
    const int rx0 = R[q].rx0, rx1 = R[q].rx1;
    uint32_t *Hs = s_role + q * kRoleWords;
    uint32_t *W = Hs + 768;
    const bool side_i = q == iq;
    span_walk(ya, yb, rx0 >> 4, (rx1 + 15) >> 4, [&](int y, int g) {
      const int x0 = g << 4;
      const int npx = min(16, w - x0);
      uint32_t wd[12];
      load_group(src + (size_t)y * pitch + 3 * x0, npx, vec, wd);
      const int i0 = max(0, rx0 - x0), i1 = min(npx, rx1 - x0);
      uint32_t a0 = 0u, a1 = 0u, a2 = 0u, a3 = 0u, a4 = 0u, a5 = 0u;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (i >= i0 && i < i1) {
          const uint32_t r = byte_of(wd, 3 * i);
          const uint32_t gg = byte_of(wd, 3 * i + 1);
          const uint32_t b = byte_of(wd, 3 * i + 2);
          atomicAdd(&Hs[r], 1u);
          atomicAdd(&Hs[256 + gg], 1u);
          atomicAdd(&Hs[512 + b], 1u);
          if (side_i) {
            atomicAdd(&W[0 * 256 + gg], r);   // (c,d) = (0,1): indexed by x_1, adds x_0
            atomicAdd(&W[1 * 256 + b], r);    // (0,2)
            atomicAdd(&W[2 * 256 + r], gg);   // (1,0)
            atomicAdd(&W[3 * 256 + b], gg);   // (1,2)
            atomicAdd(&W[4 * 256 + r], b);    // (2,0)
            atomicAdd(&W[5 * 256 + gg], b);   // (2,1)
            a0 += r * r;
            a1 += r * gg;
            a2 += r * b;
            a3 += gg * gg;
            a4 += gg * b;
            a5 += b * b;
          }
        }
      }
      // 16 pixels x 255^2 fits in 32 bits; the running total needs 64.
      acc[0] += a0; acc[1] += a1; acc[2] += a2; acc[3] += a3; acc[4] += a4; acc[5] += a5;
    });
  }
  // Gram sums: warp reduction, then one shared 64-bit add per warp.
  if (iq >= 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const unsigned long long sum = warp_sum_u64(acc[k]);
      if ((threadIdx.x & 31) == 0 && sum) atomicAdd(&s_A[iq * 6 + k], sum);
    }
  }
  __syncthreads();

  RawStats *raw = P.raw;
  for (int i = threadIdx.x; i < kPoolWords; i += blockDim.x) {
    const uint32_t c = s_pool[i];
    if (c) atomicAdd(&raw->pooled[0][0] + i, c);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (!act[q]) continue;
    const uint32_t *Hs = s_role + q * kRoleWords;
    uint32_t *dstH = R[q].is_i ? &raw->Hi[R[q].pair][0][0] : &raw->Hj[R[q].pair][0][0];
    for (int i = threadIdx.x; i < 768; i += blockDim.x) {
      const uint32_t c = Hs[i];
      if (c) atomicAdd(dstH + i, c);
    }
    if (R[q].is_i) {
      uint32_t *dstW = &raw->Wv[R[q].pair][0][0];
      for (int i = threadIdx.x; i < 1536; i += blockDim.x) {
        const uint32_t c = Hs[768 + i];
        if (c) atomicAdd(dstW + i, c);
      }
      if (threadIdx.x < 6) {
        const unsigned long long s = s_A[q * 6 + threadIdx.x];
        if (s) atomicAdd(&raw->A[R[q].pair][threadIdx.x], s);
      }
    }
  }
}

}  // namespace

size_t stats_smem_bytes() { return (size_t)(kPoolWords + 2 * kRoleWords) * 4 + (size_t)2 * 6 * 8; }

cudaError_t launch_stats(const StatsParams &p, int grid_x, cudaStream_t s) {
  const size_t smem = stats_smem_bytes();   // ~22 KB, below the default limit
  dim3 grid(grid_x, p.n_cams);
  k_stats<<<grid, kStatsThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace stitch
