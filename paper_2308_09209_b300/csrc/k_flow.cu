// Optical flow between the pre-warped images of every pair over its blend
// band (paper section 3.2: the flow that drives the local warping of Eq.
// 17-18). The paper takes it from a library routine; this is a
// coarse-to-fine block matcher on integer luminance:
//
// k_flow_luma:  Y = round-half-even(clamp((R + 2G + B) / 4, 0, 255)) of both
//               cameras' float32 pre-warped band images (uint8).
// k_flow_down:  the next pyramid level, (a + b + c + d + 2) >> 2 over 2 x 2
//               blocks, the last row / column repeated for odd sizes.
// k_flow_match: per pixel of a level and direction, the displacement d with
//               the smallest sum of |Y_a(q + d + o) - Y_b(q + o)| over the
//               7 x 7 window o (coordinates clamped into the level), over
//               [-R, R]^2 at the coarsest level and 2 d_up + [-1, 1]^2 below;
//               candidates are visited in the tie-break order (|d - start|^2,
//               then d_y, then d_x) and only a strictly smaller cost replaces
//               the best, so ties resolve the same way in any schedule.
// k_flow_final: per axis the parabola through the costs of d - 1, d, d + 1,
//               off = (c- - c+) / (2 (c- - 2 c0 + c+)) in float32 (0 unless
//               the denominator is positive, clamped to [-0.5, 0.5]); the
//               flow is float(d) + off.
//
// One thread per pixel; blockIdx.y is (pair, camera) or (pair, direction):
// direction 0 moves the left camera onto the right one (flow_ij), 1 the
// right onto the left (flow_ji). All costs are integers, so the chosen
// displacements follow from the luminance images alone.
#include "stitch_internal.h"

namespace stitch {

namespace {

constexpr int kFlowThreads = 256;
constexpr int kWin = 3;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

__device__ __forceinline__ int window_cost(const uint8_t *__restrict__ A, const uint8_t *__restrict__ B, int w, int h,
                                           int x, int y, int dx, int dy) {
  int c = 0;
#pragma unroll
  for (int oy = -kWin; oy <= kWin; ++oy) {
    const uint8_t *ra = A + (size_t)clampi(y + dy + oy, 0, h - 1) * w;
    const uint8_t *rb = B + (size_t)clampi(y + oy, 0, h - 1) * w;
#pragma unroll
    for (int ox = -kWin; ox <= kWin; ++ox) {
      const int a = __ldg(ra + clampi(x + dx + ox, 0, w - 1));
      const int b = __ldg(rb + clampi(x + ox, 0, w - 1));
      c += abs(a - b);
    }
  }
  return c;
}

__global__ void __launch_bounds__(kFlowThreads) k_flow_luma(const FlowParams P) {
  const int pair = blockIdx.y >> 1, side = blockIdx.y & 1;
  const int w = P.lev[0].w[pair], h = P.lev[0].h[pair];
  const int n = w * h;
  const float4 *src = P.pw + P.pw_off[pair][side];
  uint8_t *Y = P.Y + P.lev[0].y_off[pair][side];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 v = __ldg(src + i);
    const float s = __fmul_rn(__fadd_rn(__fadd_rn(v.x, __fmul_rn(2.0f, v.y)), v.z), 0.25f);
    Y[i] = (uint8_t)__float2int_rn(fminf(fmaxf(s, 0.0f), 255.0f));
  }
}

__global__ void __launch_bounds__(kFlowThreads) k_flow_down(const FlowParams P, int lev) {
  const int pair = blockIdx.y >> 1, side = blockIdx.y & 1;
  const int wi = P.lev[lev - 1].w[pair], hi = P.lev[lev - 1].h[pair];
  const int w = P.lev[lev].w[pair], h = P.lev[lev].h[pair];
  const uint8_t *in = P.Y + P.lev[lev - 1].y_off[pair][side];
  uint8_t *out = P.Y + P.lev[lev].y_off[pair][side];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < w * h; i += gridDim.x * blockDim.x) {
    const int y = i / w, x = i - y * w;
    const int x0 = 2 * x, y0 = 2 * y, x1 = min(2 * x + 1, wi - 1), y1 = min(2 * y + 1, hi - 1);
    const int s = in[y0 * wi + x0] + in[y1 * wi + x0] + in[y0 * wi + x1] + in[y1 * wi + x1];
    out[i] = (uint8_t)((s + 2) >> 2);
  }
}

__global__ void __launch_bounds__(kFlowThreads) k_flow_match(const FlowParams P, int lev) {
  const int pair = blockIdx.y >> 1, dir = blockIdx.y & 1;
  const int w = P.lev[lev].w[pair], h = P.lev[lev].h[pair];
  const uint8_t *A = P.Y + P.lev[lev].y_off[pair][dir];        // the image that moves
  const uint8_t *B = P.Y + P.lev[lev].y_off[pair][dir ^ 1];    // the target
  int16_t *dxo = P.dx + P.lev[lev].d_off[pair][dir];
  int16_t *dyo = P.dy + P.lev[lev].d_off[pair][dir];
  const bool top = lev == kFlowLevels - 1;
  const int n_cand = top ? P.n_cand_top : 9;
  const int8_t *cand = top ? P.cand_top : P.cand_fine;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < w * h; i += gridDim.x * blockDim.x) {
    const int y = i / w, x = i - y * w;
    int sx = 0, sy = 0;
    if (!top) {
      const int wu = P.lev[lev + 1].w[pair];
      const size_t j = P.lev[lev + 1].d_off[pair][dir] + (size_t)(y >> 1) * wu + (x >> 1);
      sx = 2 * P.dx[j];
      sy = 2 * P.dy[j];
    }
    int best = INT_MAX, bx = sx, by = sy;
    for (int c = 0; c < n_cand; ++c) {
      const int dx = sx + cand[2 * c], dy = sy + cand[2 * c + 1];
      const int cost = window_cost(A, B, w, h, x, y, dx, dy);
      if (cost < best) {
        best = cost;
        bx = dx;
        by = dy;
      }
    }
    dxo[i] = (int16_t)bx;
    dyo[i] = (int16_t)by;
  }
}

__device__ __forceinline__ float subpixel(int cm, int c0, int cp) {
  const float num = (float)(cm - cp);
  const float den = __fmul_rn(2.0f, (float)(cm - 2 * c0 + cp));
  const float off = den > 0.0f ? __fdiv_rn(num, den) : 0.0f;
  return fminf(fmaxf(off, -0.5f), 0.5f);
}

__global__ void __launch_bounds__(kFlowThreads) k_flow_final(const FlowParams P) {
  const int pair = blockIdx.y >> 1, dir = blockIdx.y & 1;
  const int w = P.lev[0].w[pair], h = P.lev[0].h[pair];
  const uint8_t *A = P.Y + P.lev[0].y_off[pair][dir];
  const uint8_t *B = P.Y + P.lev[0].y_off[pair][dir ^ 1];
  const int16_t *dxi = P.dx + P.lev[0].d_off[pair][dir];
  const int16_t *dyi = P.dy + P.lev[0].d_off[pair][dir];
  float2 *out = dir == 0 ? P.out_ij[pair] : P.out_ji[pair];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < w * h; i += gridDim.x * blockDim.x) {
    const int y = i / w, x = i - y * w;
    const int dx = dxi[i], dy = dyi[i];
    const int c0 = window_cost(A, B, w, h, x, y, dx, dy);
    const float ox = subpixel(window_cost(A, B, w, h, x, y, dx - 1, dy), c0, window_cost(A, B, w, h, x, y, dx + 1, dy));
    const float oy = subpixel(window_cost(A, B, w, h, x, y, dx, dy - 1), c0, window_cost(A, B, w, h, x, y, dx, dy + 1));
    out[i] = make_float2(__fadd_rn((float)dx, ox), __fadd_rn((float)dy, oy));
  }
}

dim3 flow_grid(const FlowParams &p, int lev) {
  int most = 0;
  for (int i = 0; i < p.n_pairs; ++i) most = std::max(most, p.lev[lev].w[i] * p.lev[lev].h[i]);
  return dim3(std::max(1, std::min(1024, (most + kFlowThreads - 1) / kFlowThreads)), 2 * p.n_pairs);
}

}  // namespace

cudaError_t launch_flow(const FlowParams &p, cudaStream_t s) {
  if (p.n_pairs <= 0) return cudaSuccess;
  k_flow_luma<<<flow_grid(p, 0), kFlowThreads, 0, s>>>(p);
  for (int lev = 1; lev < kFlowLevels; ++lev) k_flow_down<<<flow_grid(p, lev), kFlowThreads, 0, s>>>(p, lev);
  for (int lev = kFlowLevels - 1; lev >= 0; --lev) k_flow_match<<<flow_grid(p, lev), kFlowThreads, 0, s>>>(p, lev);
  k_flow_final<<<flow_grid(p, 0), kFlowThreads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace stitch
