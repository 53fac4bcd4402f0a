// Optical flow between the pre-warped images of every pair over its blend
// band (paper section 3.2: the flow that drives the local warping of Eq.
// 17-18). The paper takes it from a library routine; this is a
// coarse-to-fine block matcher on integer luminance:
//
// luminance:    Y = round-half-even(clamp((R + 2G + B) / 4, 0, 255)) of both
//               cameras' float32 pre-warped band samples (uint8; R + 2G + B of
//               each tap interpolated once), and the pyramid's next levels,
//               (a + b + c + d + 2) >> 2 over 2 x 2 blocks, the last row /
//               column repeated for odd sizes: all written by the band
//               pre-warp itself (k_prewarp_band, kFlagPwLuma), each 64 x 32
//               piece building its share of levels 1 and 2 in shared memory.
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
// at a time, summed per pixel column with byte-masked dot products). The
// candidates are taken in strips of three along d_y, which share their rows
// of the moving image, and the scan's choice is kept as the minimum of
// (cost, tie-break rank) packed into one integer. At the full level the
// matcher (k_flow_match_final) ends with the sub-pixel step, reusing the costs
// of the 3 x 3 candidates among d's four neighbours.
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
// in image coordinates, clamped into the image. Where every column lies
// inside the image with a word to spare, thread i writes word i % nw of rows
// i / nw, i / nw + rows per pass, ... (nw words per tile row), each from the
// two aligned image words that hold its bytes; the reads stay inside the
// image's rows. Elsewhere the same per byte, with the columns clamped.
template <int kPitch>
__device__ __forceinline__ void load_rect(uint8_t (*t)[kPitch], const uint8_t *__restrict__ img, int w, int h, int x0,
                                          int y0, int cols, int rows) {
  static_assert(kPitch % 4 == 0, "tile rows hold whole words");
  const int nt = blockDim.x;
  const int nw = (cols + 3) >> 2;
  if (x0 >= 0 && x0 + 4 * nw + 4 <= w && nw <= nt) {
    const int rpp = nt / nw;
    const int r = (int)threadIdx.x / nw;
    const int c = (int)threadIdx.x - r * nw;
    if (r >= rpp) return;
    for (int rr = r; rr < rows; rr += rpp) {
      const uintptr_t a = reinterpret_cast<uintptr_t>(img + (size_t)clampi(y0 + rr, 0, h - 1) * w + x0 + 4 * c);
      const uint32_t *q = reinterpret_cast<const uint32_t *>(a & ~(uintptr_t)3);
      reinterpret_cast<uint32_t *>(t[rr])[c] = __funnelshift_r(__ldg(q), __ldg(q + 1), (uint32_t)(a & 3u) * 8u);
    }
    return;
  }
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

// The tie-break rank of candidate start + (ex, ey): |e|^2, then e_y, then e_x,
// as one integer (|e|^2 in bits 10-17, e_y + 16 in bits 5-9, e_x + 16 in bits
// 0-4). The packed value (cost << 18) | rank of one candidate is below
// another's exactly when it has the smaller cost, or the same cost and an
// earlier place in the order; so the minimum of the packed values is the
// candidate that the in-order scan with strict replacement keeps, in
// whatever order the costs are summed, and the rank gives back e.
__device__ __forceinline__ uint32_t cand_rank(int ex, int ey) {
  return ((uint32_t)(ex * ex + ey * ey) << 10) | ((uint32_t)(ey + 16) << 5) | (uint32_t)(ex + 16);
}
static_assert((2 * kWin + 1) * (2 * kWin + 1) * 255 < (1 << 14), "a window cost fits in 14 bits");
static_assert(2 * kFlowMaxRadius * kFlowMaxRadius < 256 && kFlowMaxRadius < 16, "a rank fits in 18 bits");
__device__ __forceinline__ int rank_ex(uint32_t v) { return (int)(v & 31u) - 16; }
__device__ __forceinline__ int rank_ey(uint32_t v) { return (int)((v >> 5) & 31u) - 16; }

// Costs of the thread's 2 x 2 pixels for the three displacements (dx, dy0 +
// j), j = 0, 1, 2. Ten rows of the moving tile, read once at dx's column
// offset, serve all three: candidate j pairs moving row j + k with target row
// k. Per row pair two SIMD differences give the bytes of both pixel columns,
// and byte-masked dot products add bytes 0-6 (left pixel) and 1-7 (right
// pixel) onto running sums; rows 1-6 belong to the upper and the lower pixel
// row alike, row 0 ends the upper window and row 7 the lower one.
// cs[j][q]: q = 0 upper left, 1 upper right, 2 lower left, 3 lower right.
__device__ __forceinline__ void strip_costs(const MatchTile2 &T, const uint2 (&tb)[2 * kWin + 2], int ha, int lx,
                                            int ly, int dx, int dy0, uint32_t (&cs)[3][4]) {
  constexpr uint32_t kL0 = 0x01010101u, kL1 = 0x00010101u, kR0 = 0x01010100u, kR1 = 0x01010101u;
  const int o = lx + ha - kWin + dx;
  const uint8_t(*ra)[kMAWP] = T.a + (ly + ha - kWin + dy0);
  uint2 a[2 * kWin + 4];
#pragma unroll
  for (int r = 0; r < 2 * kWin + 4; ++r) a[r] = row8(ra[r], o);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    uint32_t ml = 0u, mr = 0u;
#pragma unroll
    for (int k = 1; k < 2 * kWin + 1; ++k) {
      const uint32_t d0 = __vabsdiffu4(a[j + k].x, tb[k].x), d1 = __vabsdiffu4(a[j + k].y, tb[k].y);
      ml = __dp4a(d1, kL1, __dp4a(d0, kL0, ml));
      mr = __dp4a(d1, kR1, __dp4a(d0, kR0, mr));
    }
    constexpr int kLast = 2 * kWin + 1;
    const uint32_t u0 = __vabsdiffu4(a[j].x, tb[0].x), u1 = __vabsdiffu4(a[j].y, tb[0].y);
    const uint32_t w0 = __vabsdiffu4(a[j + kLast].x, tb[kLast].x), w1 = __vabsdiffu4(a[j + kLast].y, tb[kLast].y);
    cs[j][0] = __dp4a(u1, kL1, __dp4a(u0, kL0, ml));
    cs[j][1] = __dp4a(u1, kR1, __dp4a(u0, kR0, mr));
    cs[j][2] = __dp4a(w1, kL1, __dp4a(w0, kL0, ml));
    cs[j][3] = __dp4a(w1, kR1, __dp4a(w0, kR0, mr));
  }
}

// Per thread: the 2 x 2 block's start displacement from the level above (0
// at the coarsest level). The level above keeps |d| within its reach, so
// |2 d| <= lim - 1 and every candidate stays within this level's reach; the
// clamp only guards the tile against a corrupted displacement buffer.
__device__ __forceinline__ void block_start(const FlowParams &P, int lev, int pair, int dir, int x, int y, int lim,
                                            int &sx, int &sy) {
  const int wu = P.lev[lev + 1].w[pair];
  const size_t j = P.lev[lev + 1].d_off[pair][dir] + (size_t)(y >> 1) * wu + (x >> 1);
  sx = clampi(2 * P.dx[j], 1 - lim, lim - 1);
  sy = clampi(2 * P.dy[j], 1 - lim, lim - 1);
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
  if (!top) block_start(P, lev, pair, dir, x, y, reach, sx, sy);
  const int r = top ? radius : 1;                               // candidates start + [-r, r]^2
  // the target's eight rows over both pixel rows, eight bytes over both columns
  uint2 tb[2 * kWin + 2];
#pragma unroll
  for (int k = 0; k < 2 * kWin + 2; ++k) tb[k] = row8(T.b[ly + k], lx);
  uint32_t best[4] = {UINT_MAX, UINT_MAX, UINT_MAX, UINT_MAX};
  // strips of three candidates per column e_x; the last strip of a column
  // moves up to end at e_y = r (a candidate summed twice keeps its value)
  for (int ex = -r; ex <= r; ++ex) {
    for (int ey0 = -r;; ey0 += 3) {
      const int e0 = min(ey0, r - 2);
      uint32_t cs[3][4];
      strip_costs(T, tb, ha, lx, ly, sx + ex, sy + e0, cs);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const uint32_t rk = cand_rank(ex, e0 + j);
#pragma unroll
        for (int q = 0; q < 4; ++q) best[q] = min(best[q], (cs[j][q] << 18) | rk);
      }
      if (e0 + 3 > r) break;
    }
  }
  const size_t base = P.lev[lev].d_off[pair][dir];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int xq = x + (q & 1), yq = y + (q >> 1);
    if (xq >= w || yq >= h) continue;
    const size_t i = (size_t)yq * w + xq;
    P.dx[base + i] = (int16_t)(sx + rank_ex(best[q]));
    P.dy[base + i] = (int16_t)(sy + rank_ey(best[q]));
  }
}

__device__ __forceinline__ float subpixel(int cm, int c0, int cp) {
  const float num = (float)(cm - cp);
  const float den = __fmul_rn(2.0f, (float)(cm - 2 * c0 + cp));
  const float off = den > 0.0f ? __fdiv_rn(num, den) : 0.0f;
  return fminf(fmaxf(off, -0.5f), 0.5f);
}

// The window costs of the thread's 2 x 2 pixels at one displacement (dx,
// dy), summed from the tile as strip_costs sums one candidate (the tile's
// halo covers the chosen d +- 1).
__device__ __forceinline__ void block_costs(const MatchTile2 &T, const uint2 (&tb)[2 * kWin + 2], int ha, int lx,
                                            int ly, int dx, int dy, uint32_t (&cs)[4]) {
  const int o = lx + ha - kWin + dx;
  const uint8_t(*ra)[kMAWP] = T.a + (ly + ha - kWin + dy);
  uint32_t ml = 0u, mr = 0u;
#pragma unroll
  for (int k = 1; k < 2 * kWin + 1; ++k) {
    const uint2 a = row8(ra[k], o);
    const uint32_t d0 = __vabsdiffu4(a.x, tb[k].x), d1 = __vabsdiffu4(a.y, tb[k].y);
    ml = __dp4a(d1, 0x00010101u, __dp4a(d0, 0x01010101u, ml));
    mr = __dp4a(d1, 0x01010101u, __dp4a(d0, 0x01010100u, mr));
  }
  constexpr int kLast = 2 * kWin + 1;
  const uint2 a0 = row8(ra[0], o), a7 = row8(ra[kLast], o);
  const uint32_t u0 = __vabsdiffu4(a0.x, tb[0].x), u1 = __vabsdiffu4(a0.y, tb[0].y);
  const uint32_t w0 = __vabsdiffu4(a7.x, tb[kLast].x), w1 = __vabsdiffu4(a7.y, tb[kLast].y);
  cs[0] = __dp4a(u1, 0x00010101u, __dp4a(u0, 0x01010101u, ml));
  cs[1] = __dp4a(u1, 0x01010101u, __dp4a(u0, 0x01010100u, mr));
  cs[2] = __dp4a(w1, 0x00010101u, __dp4a(w0, 0x01010101u, ml));
  cs[3] = __dp4a(w1, 0x01010101u, __dp4a(w0, 0x01010100u, mr));
}

// The neighbours of the pixels' choices that lie outside the 3 x 3: along x
// for a pixel whose e_x is -1 or 1 (the neighbour at e_x -/+ 2), along y
// likewise. Each distinct displacement among the eight is summed once for
// the whole block (block_costs), so the warp runs as many passes as its
// busiest thread has distinct displacements, usually one or two.
// out[q] holds pixel q's x neighbour, out[4 + q] its y neighbour.
__device__ __forceinline__ void outer_costs(const MatchTile2 &T, const uint2 (&tb)[2 * kWin + 2], int ha, int lx,
                                            int ly, int sx, int sy, const int (&ex)[4], const int (&ey)[4],
                                            uint32_t (&out)[8]) {
  int disp[8];                 // start-relative displacement, (o_x + 8) | (o_y + 8) << 4
  uint32_t need = 0u;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    out[q] = out[4 + q] = 0u;
    disp[q] = (2 * ex[q] + 8) | ((ey[q] + 8) << 4);
    disp[4 + q] = (ex[q] + 8) | ((2 * ey[q] + 8) << 4);
    need |= (ex[q] != 0 ? 1u : 0u) << q;
    need |= (ey[q] != 0 ? 1u : 0u) << (4 + q);
  }
  while (need) {
    const int b = __ffs(need) - 1;
    int d = disp[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) d = b == k ? disp[k] : d;
    uint32_t cs[4];
    block_costs(T, tb, ha, lx, ly, sx + (d & 15) - 8, sy + (d >> 4) - 8, cs);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (((need >> k) & 1u) && disp[k] == d) {
        out[k] = cs[k & 3];
        need &= ~(1u << k);
      }
    }
  }
}

// The full level with the sub-pixel step: the 2 x 2 matcher over the 3 x 3
// refinement (three strips, one per e_x), then per pixel the parabolas
// through the costs of its displacement d and of d -/+ (1, 0), d -/+ (0, 1).
// Neighbours inside the 3 x 3 reuse its costs (the same window sums); the
// others are summed from the tile (outer_costs).
__global__ void __launch_bounds__(kFlowThreads, 3) k_flow_match_final(const FlowParams P, int radius) {
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
  __shared__ uint32_t cst[3][3][4][kFlowThreads];   // [e_y + 1][e_x + 1][pixel][thread]
  load_rect<kMAWP>(T.a, A, w, h, bx0 - ha, by0 - ha, kMX + 2 * ha, kMY + 2 * ha);
  load_rect<kMBWP>(T.b, B, w, h, bx0 - kWin, by0 - kWin, kMBW, kMBH);
  __syncthreads();
  const int tid = threadIdx.x;
  const int lx = 2 * (tid % (kMX / 2)), ly = 2 * (tid / (kMX / 2));
  const int x = bx0 + lx, y = by0 + ly;
  if (x >= w || y >= h) return;
  int sx, sy;
  block_start(P, 0, pair, dir, x, y, reach, sx, sy);
  uint2 tb[2 * kWin + 2];
#pragma unroll
  for (int k = 0; k < 2 * kWin + 2; ++k) tb[k] = row8(T.b[ly + k], lx);
  uint32_t best[4] = {UINT_MAX, UINT_MAX, UINT_MAX, UINT_MAX};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    uint32_t cs[3][4];
    strip_costs(T, tb, ha, lx, ly, sx + c - 1, sy - 1, cs);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const uint32_t rk = cand_rank(c - 1, j - 1);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        cst[j][c][q][tid] = cs[j][q];
        best[q] = min(best[q], (cs[j][q] << 18) | rk);
      }
    }
  }
  int ex[4], ey[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    ex[q] = rank_ex(best[q]);
    ey[q] = rank_ey(best[q]);
  }
  uint32_t oc[8];
  outer_costs(T, tb, ha, lx, ly, sx, sy, ex, ey, oc);
  float2 *out = dir == 0 ? P.out_ij[pair] : P.out_ji[pair];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int xq = x + (q & 1), yq = y + (q >> 1);
    if (xq >= w || yq >= h) continue;
    const int dx = sx + ex[q], dy = sy + ey[q];
    const int c0 = (int)(best[q] >> 18);
    // d -/+ (1, 0) and d -/+ (0, 1): from the 3 x 3 where they lie in it
    const int cl = (int)(ex[q] > -1 ? cst[ey[q] + 1][ex[q]][q][tid] : oc[q]);
    const int cr = (int)(ex[q] < 1 ? cst[ey[q] + 1][ex[q] + 2][q][tid] : oc[q]);
    const int cu = (int)(ey[q] > -1 ? cst[ey[q]][ex[q] + 1][q][tid] : oc[4 + q]);
    const int cd = (int)(ey[q] < 1 ? cst[ey[q] + 2][ex[q] + 1][q][tid] : oc[4 + q]);
    const float ox = subpixel(cl, c0, cr);
    const float oy = subpixel(cu, c0, cd);
    out[(size_t)yq * w + xq] = make_float2(__fadd_rn((float)dx, ox), __fadd_rn((float)dy, oy));
  }
}

dim3 flow_tiles(const FlowParams &p, int lev, int tx, int ty) {
  int most = 0;
  for (int i = 0; i < p.n_pairs; ++i)
    most = std::max(most, ((p.lev[lev].w[i] + tx - 1) / tx) * ((p.lev[lev].h[i] + ty - 1) / ty));
  return dim3(std::max(1, most), 2 * p.n_pairs);
}

}  // namespace

cudaError_t launch_flow(const FlowParams &p, int radius, cudaStream_t s) {
  if (p.n_pairs <= 0) return cudaSuccess;
  if (radius < 1 || radius > kFlowMaxRadius) return cudaErrorInvalidValue;
  static_assert(kMX * kMY == 4 * kFlowThreads && kFlowLevels >= 2, "2 x 2 pixels per thread; a level above the finest");
  for (int lev = kFlowLevels - 1; lev >= 1; --lev)
    k_flow_match<<<flow_tiles(p, lev, kMX, kMY), kFlowThreads, 0, s>>>(p, lev, radius);
  k_flow_match_final<<<flow_tiles(p, 0, kMX, kMY), kFlowThreads, 0, s>>>(p, radius);
  return cudaGetLastError();
}

}  // namespace stitch
