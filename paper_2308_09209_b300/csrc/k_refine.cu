// Homography refinement from the blend-band flows (paper section 3.1, Eq.
// 13-14, with the supplied flow fields in place of SURF matches): the exact
// medians of each band's flow components and of their forward differences.
//
// Eight statistics per pair (problems): the x and y components of flow_ij,
// the x-differences of its x component and the y-differences of its y
// component (float32 subtractions of neighbouring samples), then the same four
// of flow_ji. Each median is the ((n - 1) // 2)-th smallest finite value,
// found by radix selection on an order-preserving 32-bit key of the float:
// four passes over the data, each building a 256-bin histogram of the next 8
// key bits among the values that match the key bits chosen so far (shared
// atomics, one global add per non-zero bin), then one block per problem picks
// the bin that holds the wanted rank. Integer counts only, so the result is
// the exact element whatever the launch order.
#include "stitch_internal.h"

namespace stitch {

namespace {

constexpr int kRefineThreads = 256;

// Ascending keys for ascending floats (-0 sorts just below +0).
__device__ __forceinline__ uint32_t order_key(float v) {
  const uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Number of values of statistic `kind` (0: x, 1: y, 2: x-difference of x,
// 3: y-difference of y) in a bw x bh band.
__device__ __forceinline__ int n_values(int kind, int bw, int bh) {
  if (kind == 2) return bw > 1 ? (bw - 1) * bh : 0;
  if (kind == 3) return bh > 1 ? bw * (bh - 1) : 0;
  return bw * bh;
}

// Value e of statistic `kind`; false when it is not finite.
__device__ __forceinline__ bool stat_value(const float2 *__restrict__ f, int kind, int bw, int e, float &v) {
  if (kind == 0) {
    v = __ldg(&f[e].x);
  } else if (kind == 1) {
    v = __ldg(&f[e].y);
  } else if (kind == 2) {
    const int y = e / (bw - 1), x = e - y * (bw - 1);
    const int i = y * bw + x;
    v = __fsub_rn(__ldg(&f[i + 1].x), __ldg(&f[i].x));
  } else {
    v = __fsub_rn(__ldg(&f[e + bw].y), __ldg(&f[e].y));
  }
  return isfinite(v);
}

__global__ void __launch_bounds__(kRefineThreads) k_refine_hist(const RefineParams P, int shift) {
  const int prob = blockIdx.y;
  const int pair = prob >> 3, q = prob & 7, kind = q & 3;
  const float2 *f = q < 4 ? P.fij[pair] : P.fji[pair];
  const int bw = P.bw[pair], bh = P.bh[pair];
  const int n = n_values(kind, bw, bh);
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0u;
  __syncthreads();
  const uint32_t mask = P.state[prob].mask, prefix = P.state[prob].prefix;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    float v;
    if (!stat_value(f, kind, bw, e, v)) continue;
    const uint32_t key = order_key(v);
    if ((key & mask) != prefix) continue;
    atomicAdd(&h[(key >> shift) & 255u], 1u);
  }
  __syncthreads();
  const uint32_t c = h[threadIdx.x];
  if (c) atomicAdd(P.hist + (size_t)prob * 256 + threadIdx.x, c);
}

// One block per problem: the bin holding the wanted rank; the histogram is
// cleared for the next pass. The first pass also counts the finite values and
// sets the rank (n - 1) / 2.
__global__ void __launch_bounds__(kRefineThreads) k_refine_pick(const RefineParams P, int shift) {
  const int prob = blockIdx.x;
  __shared__ uint32_t h[256];
  uint32_t *g = P.hist + (size_t)prob * 256;
  h[threadIdx.x] = g[threadIdx.x];
  g[threadIdx.x] = 0u;
  __syncthreads();
  if (threadIdx.x != 0) return;
  RefineState S = P.state[prob];
  if (shift == 24) {
    uint32_t n = 0u;
    for (int b = 0; b < 256; ++b) n += h[b];
    S.n = n;
    S.k = n ? (n - 1u) / 2u : 0u;
  }
  if (S.n > 0u && !S.bad) {
    uint32_t below = 0u;
    int b = 0;
    while (b < 256 && S.k >= below + h[b]) below += h[b++];
    if (b == 256) {
      S.bad = 1u;                     // the counts changed between passes (flows modified meanwhile)
    } else {
      S.k -= below;
      S.prefix |= (uint32_t)b << shift;
      S.mask |= 0xFFu << shift;
    }
  }
  P.state[prob] = S;
}

}  // namespace

cudaError_t launch_refine_pass(const RefineParams &p, int shift, cudaStream_t s) {
  if (p.n_pairs <= 0) return cudaSuccess;
  int most = 0;
  for (int i = 0; i < p.n_pairs; ++i) most = std::max(most, p.bw[i] * p.bh[i]);
  const int bx = std::max(1, std::min(64, (most + kRefineThreads - 1) / kRefineThreads));
  k_refine_hist<<<dim3(bx, 8 * p.n_pairs), kRefineThreads, 0, s>>>(p, shift);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_refine_pick<<<8 * p.n_pairs, kRefineThreads, 0, s>>>(p, shift);
  return cudaGetLastError();
}

}  // namespace stitch
