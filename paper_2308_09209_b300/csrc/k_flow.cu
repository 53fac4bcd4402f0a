// Optical flow between the pre-warped images of every pair over its blend
// band (paper section 3.2: the flow that drives the local warping of Eq.
// 17-18). The paper takes it from a library routine; this is a
// coarse-to-fine block matcher on integer luminance:
//
// luminance:    Y = round-half-even(clamp((R + 2G + B) / 4, 0, 255)) of both
//               cameras' float32 pre-warped band samples (uint8), written by
//               the band pre-warp itself (k_prewarp_band, kFlagPwLuma).
// k_flow_down:  the next pyramid level, (a + b + c + d + 2) >> 2 over 2 x 2
//               blocks, the last row / column repeated for odd sizes.
// k_flow_match: per pixel of a level and direction, the displacement d with
//               the smallest sum of |Y_a(q + d + o) - Y_b(q + o)| over the
//               7 x 7 window o (coordinates clamped into the level), over
//               [-R, R]^2 at the coarsest level and 2 d_up + [-1, 1]^2 below;
//               candidates are visited in the tie-break order (|d - start|^2,
//               then d_y, then d_x) and only a strictly smaller cost replaces
//               the best, so ties resolve the same way in any schedule.
// sub-pixel:   at the full level, per axis the parabola through the costs
//               of d - 1, d, d + 1, off = (c- - c+) / (2 (c- - 2 c0 + c+)) in
//               float32 (0 unless the denominator is positive, clamped to
//               [-0.5, 0.5]); the flow is float(d) + off.
//
// The matcher stages both images of a 64 x 16 pixel tile in shared memory and
// gives each thread a 2 x 2 block of pixels: the four share their parent at
// the level above, so they test the same candidates, and the eight window
// rows of the block serve both of its pixel rows (row differences four bytes
// at a time, summed per pixel column with byte-masked dot products). At the
// full level the matcher (k_flow_match_final) ends with the sub-pixel step,
// reusing the costs of the candidates among d's four neighbours.
// blockIdx.y is (pair, camera) or (pair, direction):
// direction 0 moves the left camera onto the right one (flow_ij), 1 the
// right onto the left (flow_ji). All costs are integers, so the chosen
// displacements follow from the luminance images alone.
#include "stitch_internal.h"

namespace stitch {

namespace {

constexpr int kFlowThreads = 256;
constexpr int kWin = 3;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

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

// Shared-memory tiles of the matcher: a 64 x 16 block of pixels, the target
// image over the block plus the window's reach, and the moving image over
// the block plus the window and the largest displacement the level can
// test. Both are loaded with the same clamped coordinates as the plain
// definition, so a tile read equals the clamped image read it replaces.
constexpr int kReach0 = 4 * kFlowMaxRadius + 2 + 1 + 1;   // |d| at the finest level, plus the sub-pixel neighbours
constexpr int kHaloA = kWin + kReach0;
// 2 x 2 pixels per thread. Rows are padded to whole 32-bit words with room
// for the third word an 8-byte read at any offset takes (the bytes beyond a
// row's data are never used).
constexpr int kMX = 64, kMY = 16;
constexpr int kMAW = kMX + 2 * kHaloA, kMAH = kMY + 2 * kHaloA;
constexpr int kMBW = kMX + 2 * kWin, kMBH = kMY + 2 * kWin;
constexpr int kMAWP = (kMAW + 8) & ~3, kMBWP = (kMBW + 8) & ~3;

struct MatchTile2 {
  __align__(16) uint8_t a[kMAH][kMAWP];
  __align__(16) uint8_t b[kMBH][kMBWP];
};

// Rows [0, rows) x columns [0, cols) of a tile from the image, origin (x0, y0)
// in image coordinates, clamped into the image: thread i takes column i % cols
// of rows i / cols, i / cols + rows per pass, ... (one division per call).
template <int kPitch>
__device__ __forceinline__ void load_rect(uint8_t (*t)[kPitch], const uint8_t *__restrict__ img, int w, int h, int x0,
                                          int y0, int cols, int rows) {
  const int nt = blockDim.x;
  if (cols <= nt) {
    const int rpp = nt / cols;
    const int r = (int)threadIdx.x / cols;
    const int c = (int)threadIdx.x - r * cols;
    if (r >= rpp) return;
    const int x = clampi(x0 + c, 0, w - 1);
    for (int rr = r; rr < rows; rr += rpp) t[rr][c] = __ldg(img + (size_t)clampi(y0 + rr, 0, h - 1) * w + x);
  } else {
    for (int i = threadIdx.x; i < cols * rows; i += nt) {
      const int rr = i / cols, c = i - rr * cols;
      t[rr][c] = __ldg(img + (size_t)clampi(y0 + rr, 0, h - 1) * w + clampi(x0 + c, 0, w - 1));
    }
  }
}

// The eight bytes [o, o + 8) of a tile row as two words, from three aligned
// 32-bit loads and two funnel shifts.
__device__ __forceinline__ uint2 row8(const uint8_t *row, int o) {
  const uint32_t *w = reinterpret_cast<const uint32_t *>(row) + (o >> 2);
  const uint32_t sh = (uint32_t)(o & 3) * 8u;
  const uint32_t w0 = w[0], w1 = w[1], w2 = w[2];
  return make_uint2(__funnelshift_r(w0, w1, sh), __funnelshift_r(w1, w2, sh));
}

__device__ __forceinline__ int level_reach(int lev, int radius) {
  int r = radius;
  for (int l = kFlowLevels - 1; l > lev; --l) r = 2 * r + 1;
  return r;
}

__global__ void __launch_bounds__(kFlowThreads, 3) k_flow_match(const FlowParams P, int lev, int radius) {
  const int pair = blockIdx.y >> 1, dir = blockIdx.y & 1;
  const int w = P.lev[lev].w[pair], h = P.lev[lev].h[pair];
  const int ntx = (w + kMX - 1) / kMX;
  if ((int)blockIdx.x >= ntx * ((h + kMY - 1) / kMY)) return;     // block-uniform
  const int bx0 = (blockIdx.x % ntx) * kMX, by0 = (blockIdx.x / ntx) * kMY;
  const uint8_t *A = P.Y + P.lev[lev].y_off[pair][dir];        // the image that moves
  const uint8_t *B = P.Y + P.lev[lev].y_off[pair][dir ^ 1];    // the target
  const bool top = lev == kFlowLevels - 1;
  const int reach = level_reach(lev, radius);
  const int ha = kWin + reach;
  __shared__ MatchTile2 T;
  load_rect<kMAWP>(T.a, A, w, h, bx0 - ha, by0 - ha, kMX + 2 * ha, kMY + 2 * ha);
  load_rect<kMBWP>(T.b, B, w, h, bx0 - kWin, by0 - kWin, kMBW, kMBH);
  __syncthreads();
  // the thread's 2 x 2 block: columns lx, lx + 1 and rows ly, ly + 1 of the tile
  const int lx = 2 * (threadIdx.x % (kMX / 2)), ly = 2 * (threadIdx.x / (kMX / 2));
  const int x = bx0 + lx, y = by0 + ly;
  if (x >= w || y >= h) return;
  int sx = 0, sy = 0;
  if (!top) {
    const int wu = P.lev[lev + 1].w[pair];
    const size_t j = P.lev[lev + 1].d_off[pair][dir] + (size_t)(y >> 1) * wu + (x >> 1);
    sx = 2 * P.dx[j];
    sy = 2 * P.dy[j];
  }
  const int n_cand = top ? P.n_cand_top : 9;
  const int8_t *cand = top ? P.cand_top : P.cand_fine;
  const int lim = reach;
  // the target's eight rows over both pixel rows, eight bytes over both columns
  uint2 tb[2 * kWin + 2];
#pragma unroll
  for (int k = 0; k < 2 * kWin + 2; ++k) tb[k] = row8(T.b[ly + k], lx);
  int best[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
  int bxs[4] = {sx, sx, sx, sx}, bys[4] = {sy, sy, sy, sy};
  for (int c = 0; c < n_cand; ++c) {
    // the search never leaves the reach; the clamp only guards the tile
    const int dx = clampi(sx + cand[2 * c], -lim, lim), dy = clampi(sy + cand[2 * c + 1], -lim, lim);
    const int o = lx + ha - kWin + dx;
    const uint8_t(*ra)[kMAWP] = T.a + (ly + ha - kWin + dy);
    // costs of (left, right) x (upper, lower): window rows 0-6 and 1-7
    unsigned c00 = 0u, c01 = 0u, c10 = 0u, c11 = 0u;
#pragma unroll
    for (int k = 0; k < 2 * kWin + 2; ++k) {
      const uint2 a = row8(ra[k], o);
      const unsigned d0 = __vabsdiffu4(a.x, tb[k].x), d1 = __vabsdiffu4(a.y, tb[k].y);
      // left pixel: bytes 0-6; right pixel: bytes 1-7
      const unsigned sl = __dp4a(d1, 0x00010101u, __dp4a(d0, 0x01010101u, 0u));
      const unsigned sr = __dp4a(d1, 0x01010101u, __dp4a(d0, 0x01010100u, 0u));
      if (k < 2 * kWin + 1) { c00 += sl; c01 += sr; }
      if (k > 0) { c10 += sl; c11 += sr; }
    }
    const unsigned cs[4] = {c00, c01, c10, c11};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if ((int)cs[q] < best[q]) {
        best[q] = (int)cs[q];
        bxs[q] = dx;
        bys[q] = dy;
      }
    }
  }
  const size_t base = P.lev[lev].d_off[pair][dir];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int xq = x + (q & 1), yq = y + (q >> 1);
    if (xq >= w || yq >= h) continue;
    const size_t i = (size_t)yq * w + xq;
    P.dx[base + i] = (int16_t)bxs[q];
    P.dy[base + i] = (int16_t)bys[q];
  }
}

__device__ __forceinline__ float subpixel(int cm, int c0, int cp) {
  const float num = (float)(cm - cp);
  const float den = __fmul_rn(2.0f, (float)(cm - 2 * c0 + cp));
  const float off = den > 0.0f ? __fdiv_rn(num, den) : 0.0f;
  return fminf(fmaxf(off, -0.5f), 0.5f);
}

// The full level with the sub-pixel step: the 2 x 2 matcher over the nine
// refinement candidates, then per pixel the parabolas through the costs of
// its displacement d and of d -/+ (1, 0), d -/+ (0, 1). Neighbours that were
// candidates reuse their cost (the same window sums); the others are summed
// from the tile, whose halo covers d +- 1.
__device__ __forceinline__ int pixel_cost(const MatchTile2 &T, const uint2 (&tb)[2 * kWin + 2], int ha, int lx,
                                          int ly, int qx, int qy, int dx, int dy) {
  const int o = lx + ha - kWin + dx;
  const uint8_t(*ra)[kMAWP] = T.a + (ly + ha - kWin + dy + qy);
  const unsigned m0 = qx ? 0x01010100u : 0x01010101u, m1 = qx ? 0x01010101u : 0x00010101u;
  unsigned c = 0u;
#pragma unroll
  for (int k = 0; k < 2 * kWin + 1; ++k) {
    const uint2 a = row8(ra[k], o);
    const uint2 t = qy ? tb[k + 1] : tb[k];
    c = __dp4a(__vabsdiffu4(a.x, t.x), m0, c);
    c = __dp4a(__vabsdiffu4(a.y, t.y), m1, c);
  }
  return (int)c;
}

__global__ void __launch_bounds__(kFlowThreads, 2) k_flow_match_final(const FlowParams P, int radius) {
  const int pair = blockIdx.y >> 1, dir = blockIdx.y & 1;
  const int w = P.lev[0].w[pair], h = P.lev[0].h[pair];
  const int ntx = (w + kMX - 1) / kMX;
  if ((int)blockIdx.x >= ntx * ((h + kMY - 1) / kMY)) return;     // block-uniform
  const int bx0 = (blockIdx.x % ntx) * kMX, by0 = (blockIdx.x / ntx) * kMY;
  const uint8_t *A = P.Y + P.lev[0].y_off[pair][dir];
  const uint8_t *B = P.Y + P.lev[0].y_off[pair][dir ^ 1];
  const int reach = level_reach(0, radius);
  const int ha = kWin + reach + 1;                              // the chosen d and its neighbours
  __shared__ MatchTile2 T;
  load_rect<kMAWP>(T.a, A, w, h, bx0 - ha, by0 - ha, kMX + 2 * ha, kMY + 2 * ha);
  load_rect<kMBWP>(T.b, B, w, h, bx0 - kWin, by0 - kWin, kMBW, kMBH);
  __syncthreads();
  const int lx = 2 * (threadIdx.x % (kMX / 2)), ly = 2 * (threadIdx.x / (kMX / 2));
  const int x = bx0 + lx, y = by0 + ly;
  if (x >= w || y >= h) return;
  const int wu = P.lev[1].w[pair];
  const size_t j = P.lev[1].d_off[pair][dir] + (size_t)(y >> 1) * wu + (x >> 1);
  const int sx = 2 * P.dx[j], sy = 2 * P.dy[j];
  const int lim = reach;
  uint2 tb[2 * kWin + 2];
#pragma unroll
  for (int k = 0; k < 2 * kWin + 2; ++k) tb[k] = row8(T.b[ly + k], lx);
  int best[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
  int bxs[4] = {sx, sx, sx, sx}, bys[4] = {sy, sy, sy, sy};
  int cst[4][9], cdx[9], cdy[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const int dx = clampi(sx + P.cand_fine[2 * c], -lim, lim), dy = clampi(sy + P.cand_fine[2 * c + 1], -lim, lim);
    cdx[c] = dx;
    cdy[c] = dy;
    const int o = lx + ha - kWin + dx;
    const uint8_t(*ra)[kMAWP] = T.a + (ly + ha - kWin + dy);
    unsigned c00 = 0u, c01 = 0u, c10 = 0u, c11 = 0u;
#pragma unroll
    for (int k = 0; k < 2 * kWin + 2; ++k) {
      const uint2 a = row8(ra[k], o);
      const unsigned d0 = __vabsdiffu4(a.x, tb[k].x), d1 = __vabsdiffu4(a.y, tb[k].y);
      const unsigned sl = __dp4a(d1, 0x00010101u, __dp4a(d0, 0x01010101u, 0u));
      const unsigned sr = __dp4a(d1, 0x01010101u, __dp4a(d0, 0x01010100u, 0u));
      if (k < 2 * kWin + 1) { c00 += sl; c01 += sr; }
      if (k > 0) { c10 += sl; c11 += sr; }
    }
    const unsigned cs[4] = {c00, c01, c10, c11};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      cst[q][c] = (int)cs[q];
      if ((int)cs[q] < best[q]) {
        best[q] = (int)cs[q];
        bxs[q] = dx;
        bys[q] = dy;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int xq = x + (q & 1), yq = y + (q >> 1);
    if (xq >= w || yq >= h) continue;
    const int dx = bxs[q], dy = bys[q];
    // costs of d, d -/+ (1, 0), d -/+ (0, 1)
    int cc[5];
    cc[0] = best[q];
#pragma unroll
    for (int e = 1; e < 5; ++e) {
      const int nx = dx + (e == 1 ? -1 : (e == 2 ? 1 : 0)), ny = dy + (e == 3 ? -1 : (e == 4 ? 1 : 0));
      int v = -1;
#pragma unroll
      for (int c = 0; c < 9; ++c)
        if (cdx[c] == nx && cdy[c] == ny) v = cst[q][c];
      cc[e] = v >= 0 ? v : pixel_cost(T, tb, ha, lx, ly, q & 1, q >> 1, nx, ny);
    }
    const float ox = subpixel(cc[1], cc[0], cc[2]);
    const float oy = subpixel(cc[3], cc[0], cc[4]);
    float2 *out = dir == 0 ? P.out_ij[pair] : P.out_ji[pair];
    out[(size_t)yq * w + xq] = make_float2(__fadd_rn((float)dx, ox), __fadd_rn((float)dy, oy));
  }
}

dim3 flow_tiles(const FlowParams &p, int lev, int tx, int ty) {
  int most = 0;
  for (int i = 0; i < p.n_pairs; ++i)
    most = std::max(most, ((p.lev[lev].w[i] + tx - 1) / tx) * ((p.lev[lev].h[i] + ty - 1) / ty));
  return dim3(std::max(1, most), 2 * p.n_pairs);
}

dim3 flow_grid(const FlowParams &p, int lev) {
  int most = 0;
  for (int i = 0; i < p.n_pairs; ++i) most = std::max(most, p.lev[lev].w[i] * p.lev[lev].h[i]);
  return dim3(std::max(1, std::min(1024, (most + kFlowThreads - 1) / kFlowThreads)), 2 * p.n_pairs);
}

}  // namespace

cudaError_t launch_flow(const FlowParams &p, int radius, cudaStream_t s) {
  if (p.n_pairs <= 0) return cudaSuccess;
  if (radius < 1 || radius > kFlowMaxRadius) return cudaErrorInvalidValue;
  static_assert(kMX * kMY == 4 * kFlowThreads && kFlowLevels >= 2, "2 x 2 pixels per thread; a level above the finest");
  for (int lev = 1; lev < kFlowLevels; ++lev) k_flow_down<<<flow_grid(p, lev), kFlowThreads, 0, s>>>(p, lev);
  for (int lev = kFlowLevels - 1; lev >= 1; --lev)
    k_flow_match<<<flow_tiles(p, lev, kMX, kMY), kFlowThreads, 0, s>>>(p, lev, radius);
  k_flow_match_final<<<flow_tiles(p, 0, kMX, kMY), kFlowThreads, 0, s>>>(p, radius);
  return cudaGetLastError();
}

}  // namespace stitch
