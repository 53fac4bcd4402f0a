// K1 -- integer colour statistics of one frame (paper section 2.1 steps 2-4,
// Eq. 1-3 terms; section 2.2 histogram for the balance knots).
//
// One streaming pass over every camera frame. Each thread takes groups of 16
// consecutive pixels (48 bytes, three 16-byte loads when the row is 16-byte
// aligned) and, per pixel:
//   * adds the three channel values to the pooled full-frame histogram
//     (section 2.2: the lambda-quantile knots);
//   * inside a pair's source rectangle, adds to that side's overlap histogram
//     (section 2.1 step 2); on the colour-source side i it also adds to the
//     value-weighted histograms W_cd[x_d] += x_c (c != d) and to the Gram sums
//     x_c x_d. With these, the estimate kernel forms B = I_i^T L(I_i) without
//     a second pass over the pixels once the specification L is known:
//     B_cd = sum_v L_d(v) W_cd(v), B_dd = sum_v L_d(v) v H_i,d(v).
// Runs of equal consecutive values within a thread's 16 pixels are merged
// into one shared-memory atomic; counts are flushed with one global atomic
// per non-zero bin. All arithmetic is integer, so results are bit-exact.
#include "stitch_internal.h"

namespace stitch {

namespace {

constexpr int kPoolWords = 3 * 256;
constexpr int kRoleWords = 3 * 256 + 6 * 256;   // H then W

__device__ __forceinline__ uint32_t byte_of(const uint32_t (&w)[12], int j) {
  return (w[j >> 2] >> ((j & 3) * 8)) & 0xffu;
}

// Add the 16 values of one channel (bytes 3 i + c of the group) to a
// histogram, merging runs of equal consecutive values into one atomic each.
template <int kC>
__device__ __forceinline__ void hist_runs(const uint32_t (&wd)[12], int i0, int i1, uint32_t *h) {
  uint32_t run_v = 0xffffffffu, run_n = 0u;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    if (i >= i0 && i < i1) {
      const uint32_t v = byte_of(wd, 3 * i + kC);
      if (v != run_v) {
        if (run_n) atomicAdd(&h[run_v], run_n);
        run_v = v;
        run_n = 0u;
      }
      ++run_n;
    }
  }
  if (run_n) atomicAdd(&h[run_v], run_n);
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

  // Rows are walked by a fixed thread -> (row, group) assignment: no division
  // inside the loop when a row has at most blockDim groups.
  const int nt = blockDim.x;
  const bool rowwise = groups <= nt;
  const int rpi = rowwise ? nt / groups : 1;
  int rr = rowwise ? (int)threadIdx.x / groups : 0;
  int g = rowwise ? (int)threadIdx.x - rr * groups : 0;
  int idx = threadIdx.x;
  const bool idle = rowwise && (int)threadIdx.x >= rpi * groups;
  while (!idle) {
    if (!rowwise) {
      if (idx >= (r1 - r0) * groups) break;
      rr = idx / groups;
      g = idx - rr * groups;
    } else if (r0 + rr >= r1) {
      break;
    }
    const int y = r0 + rr;
    const int x0 = g << 4;
    const int npx = min(16, w - x0);
    const uint8_t *p = src + (size_t)y * pitch + 3 * x0;
    uint32_t wd[12];
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
    // Pooled full-frame histogram.
    hist_runs<0>(wd, 0, npx, s_pool);
    hist_runs<1>(wd, 0, npx, s_pool + 256);
    hist_runs<2>(wd, 0, npx, s_pool + 512);
    // Overlap rectangles: the group's pixel range [i0, i1) inside each.
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!act[q] || y < R[q].ry0 || y >= R[q].ry1) continue;
      const int i0 = max(0, R[q].rx0 - x0), i1 = min(npx, R[q].rx1 - x0);
      if (i0 >= i1) continue;
      uint32_t *Hs = s_role + q * kRoleWords;
      hist_runs<0>(wd, i0, i1, Hs);
      hist_runs<1>(wd, i0, i1, Hs + 256);
      hist_runs<2>(wd, i0, i1, Hs + 512);
      if (R[q].is_i) {
        uint32_t *W = Hs + 768;
        uint32_t a0 = 0u, a1 = 0u, a2 = 0u, a3 = 0u, a4 = 0u, a5 = 0u;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (i >= i0 && i < i1) {
            const uint32_t r = byte_of(wd, 3 * i);
            const uint32_t gg = byte_of(wd, 3 * i + 1);
            const uint32_t b = byte_of(wd, 3 * i + 2);
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
        // 16 pixels x 255^2 fits in 32 bits; the block total needs 64.
        atomicAdd(&s_A[q * 6 + 0], (unsigned long long)a0);
        atomicAdd(&s_A[q * 6 + 1], (unsigned long long)a1);
        atomicAdd(&s_A[q * 6 + 2], (unsigned long long)a2);
        atomicAdd(&s_A[q * 6 + 3], (unsigned long long)a3);
        atomicAdd(&s_A[q * 6 + 4], (unsigned long long)a4);
        atomicAdd(&s_A[q * 6 + 5], (unsigned long long)a5);
      }
    }
    if (rowwise) rr += rpi; else idx += nt;
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
