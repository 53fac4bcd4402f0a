// K3 -- pre-warp, local warping, colour transfer, blend and balance
// (paper section 3.1 pre-warp; section 3.2 Eq. 15-18; Eq. 4; Eq. 5).
//
// Kernels of one frame:
//
// k_prewarp_band: the pre-warped image of section 3.1 over each pair's blend
//   band, for BOTH cameras of the pair, computed once per band pixel and kept
//   in a small intermediate. It does not depend on the colour estimate. In
//   the frame path the intermediate holds v - 128 (the offset form below) as
//   halves, which hold the half2 bilinear's results exactly;
//   STITCH_FP16_INTERMEDIATE selects half2 instead of float32 arithmetic for
//   the remap that reads them. (The flow and the correspondence fit use a
//   float32 intermediate of the plain pre-warped image.)
//
// k_fuse_own: the fully covered own tiles (columns of one camera k, every
//   pixel seen by k with a margin), about three quarters of a rig's tiles.
//   The source window that a tile maps to through H_k^-1 (planar) or through
//   the cylinder's ray and H_k^-1 is staged in shared memory as one RGBX word
//   per pixel whose fourth byte is 0x64, so that one byte permute turns the
//   same channel of two pixels into a half2 pair (1024 + v0, 1024 + v1).
//   A thread takes its pixels two at a time:
//   * s = H_k^-1 q for both in packed float32 (f32x2 FMA), relative to the
//     window and shifted by half a pixel, one reciprocal per pixel;
//   * integer tap and fraction by the round-to-nearest magic constant;
//   * the bilinear sample (Eq. 18's kernel, section 3.1) in half2 on v - 128:
//     a + fx (b - a) + fy ((d - a) + fx ((e - d) - (b - a))), exact tap
//     differences, every rounding within 1/32 of a grey level of the exact
//     interpolant for the fraction rounded to half precision;
//   * v . M (Eq. 4) in packed float32 with the offset folded into a per-
//     channel bias, the last product saturating to [0, 1] (M is pre-scaled by
//     1/255), which is the clamp to [0, 255];
//   * balance (Eq. 5) and rounding through the colour slot's output table:
//     byte = table[round(4080 u)], the curve evaluated at the fused value
//     rounded to a sixteenth of a grey level.
//
// k_fuse: the band tiles and the partly covered own tiles.
//   * Pixels of a band rectangle: theta_j = (x - x0 + 0.5) / (x1 - x0),
//     theta_i = 1 - theta_j (Eq. 16 read as a ramp), X_i = q + theta_j
//     clamp(flow_ij), X_j = q + theta_i clamp(flow_ji) (Eq. 17, continuous
//     reading; the printed weights under STITCH_FLOW_WEIGHTS_PRINTED), X
//     clamped into the band (skipped for tiles whose reach stays inside it),
//     the bilinear sample of the pre-warped intermediate (Eq. 18), then
//     out = theta_i P_i(X_i) M_i + theta_j P_j(X_j) M_j through the table.
//   * Other pixels (own columns beside the band, band columns outside the
//     band rows, partly covered tiles) take the general float32 path: staged
//     windows of both cameras, coverage tests, Eq. 15's one-image fallbacks
//     (k, then k - 1, then k + 1), blending both cameras without flow where
//     both cover a band-column pixel, uncovered pixels 0.
//   Pixels go to a shared-memory tile and leave as 16-byte stores per plane.
//
// Both fuse kernels are persistent: a block loads the colour matrices and
// the 12 KB output table once and then takes tiles with a fixed stride.
//
// k_prewarp_multi / k_fuse_multi / k_fuse_own_multi: the same work over the
// tiles of several independent rigs in one launch each; the fuse kernels
// take tiles from a work counter and reload the colour constants when the
// rig changes. When the rigs' tile shapes differ, the *_mixed forms run
// every tile with its rig's shape.
#include <algorithm>
#include <cstddef>
#include <cuda_fp16.h>

#include "stitch_internal.h"

namespace stitch {

namespace {

constexpr float kMagicRound = 12582912.0f;   // 1.5 * 2^23: x + kMagicRound rounds x to an integer (RNE)
constexpr uint32_t kMagicRoundBits = 0x4B400000u;
constexpr float kMagicByte = 8388608.0f;     // 2^23: the float with bits 0x4B0000bb is 2^23 + bb
constexpr uint32_t kXByte = 0x64u;           // fourth byte of a staged word: [v, 0x64] is the half 1024 + v
constexpr float kHalfOffset = 1152.0f;       // 1024 + 128: half (1024 + v) minus this is v - 128

// Source windows: a fixed row stride per tile shape (tap offsets become
// immediates); windows wider or taller than the capacity fall back to
// per-pixel global gathers and are counted (windows clipped by the frame to a
// sliver, or with a corner behind the camera, take the same path uncounted).
template <int TW, int TH>
struct WinGeom {
  static constexpr int kStride = TW + TW / 2;          // words per staged row
  static constexpr int kRows = TH + 16 + (TW >= 128 ? 8 : 0);   // a wide tile spans more rotated rows
  static constexpr int kAlloc = kStride * kRows + kStride + 8;   // + a guard row for zero-weight taps
  static_assert(kStride % 4 == 0, "window rows are staged four pixels at a time");
};

// Approximate reciprocal (the hardware's one-instruction rcp.approx, flushing
// subnormals: within one ulp; a camera's w is near 1 wherever it is used).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

__device__ __forceinline__ __half2 as_h2(uint32_t v) {
  __half2 h;
  *reinterpret_cast<uint32_t *>(&h) = v;
  return h;
}
__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<const uint32_t *>(&h); }

// s = H^-1 q for panorama point (x, y) given as floats relative to the origin.
// Cylindrical panorama: q stands for the ray (sin theta, h, cos theta) with
// theta = (x - cx) / f and h = (y - cy) / f (the origin is 0 there).
__device__ __forceinline__ void cam_map_f(const CamDev &c, float dx, float dy, float &sx, float &sy, float &nw) {
  float nx, ny;
  if (c.cyl) {
    const float th = (dx - c.cyl_cx) * c.cyl_finv;
    const float hh = (dy - c.cyl_cy) * c.cyl_finv;
    float sn, cs;
    sincosf(th, &sn, &cs);
    nx = fmaf(c.h[0], sn, fmaf(c.h[1], hh, c.h[2] * cs));
    ny = fmaf(c.h[3], sn, fmaf(c.h[4], hh, c.h[5] * cs));
    nw = fmaf(c.h[6], sn, fmaf(c.h[7], hh, c.h[8] * cs));
  } else {
    nx = fmaf(c.h[0], dx, fmaf(c.h[1], dy, c.h[2]));
    ny = fmaf(c.h[3], dx, fmaf(c.h[4], dy, c.h[5]));
    nw = fmaf(c.h[6], dx, fmaf(c.h[7], dy, c.h[8]));
  }
  const float r = rcp_approx(nw);
  sx = __fmul_rn(nx, r);
  sy = __fmul_rn(ny, r);
}

// Integer part and fraction of s with fraction in [0, 1]; for integer s the
// pair (s - 1, 1) may come back instead of (s, 0): both give the same bilinear
// sample, and the right-hand tap then never passes the last row / column.
__device__ __forceinline__ void split(float s, int &i, float &f) {
  const float r = (s - 0.5f) + kMagicRound;
  i = __float_as_int(r) - (int)kMagicRoundBits;
  f = s - (r - kMagicRound);
}

// Channel c (0..2) of an RGBX word as 2^23 + value (exact).
__device__ __forceinline__ float mbyte(uint32_t w, int c) {
  return __int_as_float(__byte_perm(w, 0x4B000000u, 0x7440u + c));
}

// Bilinear of four RGBX words with fractions (fx, fy), float32.
__device__ __forceinline__ float3 bilerp_words(uint32_t a, uint32_t b, uint32_t d, uint32_t e, float fx, float fy) {
  float o[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float A = mbyte(a, c), B = mbyte(b, c), D = mbyte(d, c), E = mbyte(e, c);
    const float top = fmaf(fx, B - A, A - kMagicByte);
    const float bot = fmaf(fx, E - D, D - kMagicByte);
    o[c] = fmaf(fy, bot - top, top);
  }
  return make_float3(o[0], o[1], o[2]);
}

__device__ __forceinline__ float3 load_rgb(const uint8_t *__restrict__ p) {
  return make_float3((float)__ldg(p), (float)__ldg(p + 1), (float)__ldg(p + 2));
}

// Bilinear sample of a packed-RGB frame in global memory at (sx, sy) inside
// the frame (the general path, used where no staged window applies).
__device__ __forceinline__ float3 src_bilinear(const uint8_t *__restrict__ src, const CamDev &c, float sx, float sy) {
  int ix, iy;
  float fx, fy;
  split(sx, ix, fx);
  split(sy, iy, fy);
  ix = min(max(ix, 0), c.w - 1);
  iy = min(max(iy, 0), c.h_px - 1);
  const int ix1 = min(ix + 1, c.w - 1), iy1 = min(iy + 1, c.h_px - 1);
  const uint8_t *r0 = src + (size_t)iy * c.pitch;
  const uint8_t *r1 = src + (size_t)iy1 * c.pitch;
  const float3 a = load_rgb(r0 + 3 * ix), b = load_rgb(r0 + 3 * ix1);
  const float3 d = load_rgb(r1 + 3 * ix), e = load_rgb(r1 + 3 * ix1);
  float3 t, u, o;
  t.x = fmaf(fx, b.x - a.x, a.x); t.y = fmaf(fx, b.y - a.y, a.y); t.z = fmaf(fx, b.z - a.z, a.z);
  u.x = fmaf(fx, e.x - d.x, d.x); u.y = fmaf(fx, e.y - d.y, d.y); u.z = fmaf(fx, e.z - d.z, d.z);
  o.x = fmaf(fy, u.x - t.x, t.x); o.y = fmaf(fy, u.y - t.y, t.y); o.z = fmaf(fy, u.z - t.z, t.z);
  return o;
}

// ---------------------------------------------------------------------------
// Source windows in shared memory.
// ---------------------------------------------------------------------------

struct Window {
  int x0, y0, w, h, ok;
  int a16;                           // staged in 16-pixel groups from 16-byte aligned rows (x0 % 16 == 0)
  int over;                          // a proper window (in front, at least 2 x 2) beyond the capacity
};

// Rows of the frame start on 16-byte boundaries (base and pitch), so a
// 16-pixel group starting at a multiple of 16 pixels is three aligned
// 16-byte words.
__device__ __forceinline__ bool rows16(const uint8_t *src, const CamDev &c) {
  return ((reinterpret_cast<uintptr_t>(src) | (uintptr_t)c.pitch) & 15u) == 0;
}

// Source window of the panorama rectangle [rx0, rx1] x [ry0, ry1] (inclusive)
// in camera c: the bounding box of the mapped corners plus one pixel of margin
// and the right / bottom tap, clipped to the frame. Computed by one warp (lane
// & 3 picks a corner); every lane returns the same window. ok = 0 when a corner
// maps behind the camera, the box is empty or it exceeds the capacity. With
// a16 (rows16) the left edge moves down to a multiple of 16 pixels when the
// wider window still fits, so that staging takes aligned 16-pixel groups.
template <int kStride, int kRows>
__device__ Window warp_window(const CamDev &c, int rx0, int ry0, int rx1, int ry1, bool a16) {
  const int k = threadIdx.x & 3;
  const int px = (k & 1) ? rx1 : rx0;
  const int py = (k & 2) ? ry1 : ry0;
  float sx, sy, nw;
  cam_map_f(c, (float)(px - c.ox), (float)(py - c.oy), sx, sy, nw);
  int front = (nw > 0.0f && sx == sx && sy == sy) ? 1 : 0;
  float lo_x = sx, hi_x = sx, lo_y = sy, hi_y = sy;
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    lo_x = fminf(lo_x, __shfl_xor_sync(0xffffffffu, lo_x, o));
    hi_x = fmaxf(hi_x, __shfl_xor_sync(0xffffffffu, hi_x, o));
    lo_y = fminf(lo_y, __shfl_xor_sync(0xffffffffu, lo_y, o));
    hi_y = fmaxf(hi_y, __shfl_xor_sync(0xffffffffu, hi_y, o));
    front &= __shfl_xor_sync(0xffffffffu, front, o);
  }
  lo_x = fmaxf(lo_x, -4.0f);
  lo_y = fmaxf(lo_y, -4.0f);
  hi_x = fminf(hi_x, c.wm1 + 4.0f);
  hi_y = fminf(hi_y, c.hm1 + 4.0f);
  Window W;
  W.x0 = max(0, (int)floorf(lo_x) - 1);
  W.y0 = max(0, (int)floorf(lo_y) - 1);
  const int x1 = min(c.w - 1, (int)floorf(hi_x) + 2);
  const int y1 = min(c.h_px - 1, (int)floorf(hi_y) + 2);
  // aligned: 16 ceil((w + 1) / 16) words per row (the word past the window included)
  W.a16 = (kStride % 16 == 0 && a16 && x1 - (W.x0 & ~15) + 1 <= kStride - 1) ? 1 : 0;
  if (W.a16) W.x0 &= ~15;
  W.w = x1 - W.x0 + 1;
  W.h = y1 - W.y0 + 1;
  const bool proper = front && W.w >= 2 && W.h >= 2;
  W.ok = (proper && W.w <= kStride && W.h <= kRows) ? 1 : 0;
  W.over = (proper && !W.ok) ? 1 : 0;
  return W;
}

__device__ __forceinline__ Window no_window() {
  Window W;
  W.x0 = W.y0 = W.w = W.h = W.ok = W.a16 = W.over = 0;
  return W;
}

// Stage the window as RGBX words (fourth byte 0x64): four pixels (12 bytes)
// per step, read as aligned 32-bit words and realigned with funnel shifts.
// Every row also gets the word just past the window (a real pixel, or 0x64
// past the frame) and the row below the window is filled with 0x64 words:
// a tap with zero weight there still reads a finite value.
template <int kStride>
__device__ void stage_window(const uint8_t *__restrict__ src, const CamDev &c, const Window &W, uint32_t *s) {
  for (int i = threadIdx.x; i < kStride + 4; i += blockDim.x) s[W.h * kStride + i] = kXByte << 24;
  if (W.a16) {
    // 16 pixels (48 bytes, three aligned 16-byte words) per step; groups that
    // reach past the frame's right edge are read byte by byte (0x64 words
    // past the edge).
    const int G16 = (W.w + 16) >> 4;               // <= kStride / 16 (warp_window checked)
    const float inv16 = rcp_approx((float)G16);
    const int rpp16 = (int)(((float)kFuseThreads + 0.5f) * inv16);
    const int rf = (int)(((float)threadIdx.x + 0.5f) * inv16);
    const int g16 = threadIdx.x - rf * G16;
    if (rf >= rpp16 || rf >= W.h) return;
    const int px = W.x0 + 16 * g16;
    const int nv = min(16, max(0, c.w - px));      // pixels of the group inside the frame
    const uint8_t *row = src + (size_t)(W.y0 + rf) * c.pitch + 3 * px;
    const size_t rstep = (size_t)rpp16 * (size_t)c.pitch;
    uint32_t *dst = s + rf * kStride + 16 * g16;
    for (int r = rf; r < W.h; r += rpp16, row += rstep, dst += rpp16 * kStride) {
      uint32_t q[12];
      if (nv == 16) {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(row));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(row) + 1);
        const uint4 d = __ldg(reinterpret_cast<const uint4 *>(row) + 2);
        q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
        q[4] = b.x; q[5] = b.y; q[6] = b.z; q[7] = b.w;
        q[8] = d.x; q[9] = d.y; q[10] = d.z; q[11] = d.w;
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) q[k] = 0u;
#pragma unroll
        for (int j = 0; j < 48; ++j)
          if (j < 3 * nv) q[j >> 2] |= (uint32_t)__ldg(row + j) << ((j & 3) * 8);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t q0 = q[3 * k], q1 = q[3 * k + 1], q2 = q[3 * k + 2];
        const uint32_t p0 = __byte_perm(q0, kXByte, 0x4210u);
        const uint32_t p1 = (__byte_perm(q0, q1, 0x0543u) & 0x00ffffffu) | (kXByte << 24);
        const uint32_t p2 = (__byte_perm(q1, q2, 0x0432u) & 0x00ffffffu) | (kXByte << 24);
        const uint32_t p3 = __byte_perm(q2, kXByte, 0x4321u);
        *reinterpret_cast<uint4 *>(dst + 4 * k) = make_uint4(p0, p1, p2, p3);
      }
    }
    return;
  }
  const int G = min((W.w + 4) >> 2, kStride >> 2);
  // G <= kStride / 4 <= blockDim.x: thread i takes group i % G of rows i / G,
  // i / G + rows_per_pass, ... The quotients come from an approximate
  // reciprocal: floor((i + 1/2) / G) = floor(i / G), and (i + 1/2) / G lies at
  // least 1 / (2 G) >= 1/128 from an integer, far beyond the reciprocal's error.
  const float inv_g = rcp_approx((float)G);
  const int rpp = (int)(((float)kFuseThreads + 0.5f) * inv_g);
  const int r_first = (int)(((float)threadIdx.x + 0.5f) * inv_g);
  const int g = threadIdx.x - r_first * G;
  if (r_first >= rpp || r_first >= W.h) return;
  const int px = W.x0 + 4 * g;
  const int nvalid = min(4, c.w - px);              // pixels of the group inside the frame
  const uint32_t col = 3u * (uint32_t)px;           // byte offset of the group in its row
  // With a pitch that is a multiple of 4, every row's group has the same
  // misalignment; the four aligned words from there hold its 12 bytes.
  const uintptr_t B = reinterpret_cast<uintptr_t>(src + (size_t)(W.y0 + r_first) * c.pitch + col);
  const uint32_t lead = (uint32_t)(B & 3u), sh = lead * 8u;
  const uint32_t *wrow = reinterpret_cast<const uint32_t *>(B - lead);
  const size_t wstep = (size_t)rpp * (size_t)c.pitch / 4;
  const bool vec_ok = nvalid == 4 && (c.pitch & 3) == 0;
  // On the frame's last row the 16 bytes read must end inside its 3 w bytes.
  const int last_vec_row = (col - lead + 16u <= 3u * (uint32_t)c.w) ? c.h_px - 1 : c.h_px - 2;
  uint32_t *dst = s + r_first * kStride + 4 * g;
  for (int r = r_first; r < W.h; r += rpp, wrow += wstep, dst += rpp * kStride) {
    uint32_t p0, p1, p2, p3;
    if (vec_ok && W.y0 + r <= last_vec_row) {
      const uint32_t w0 = __ldg(wrow), w1 = __ldg(wrow + 1), w2 = __ldg(wrow + 2), w3 = __ldg(wrow + 3);
      const uint32_t q0 = __funnelshift_r(w0, w1, sh);
      const uint32_t q1 = __funnelshift_r(w1, w2, sh);
      const uint32_t q2 = __funnelshift_r(w2, w3, sh);
      p0 = __byte_perm(q0, kXByte, 0x4210u);
      p1 = (__byte_perm(q0, q1, 0x0543u) & 0x00ffffffu) | (kXByte << 24);
      p2 = (__byte_perm(q1, q2, 0x0432u) & 0x00ffffffu) | (kXByte << 24);
      p3 = __byte_perm(q2, kXByte, 0x4321u);
    } else {
      const uint8_t *b = src + (size_t)(W.y0 + r) * c.pitch + col;
      uint32_t q[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < nvalid)
          q[k] = (uint32_t)__ldg(b + 3 * k) | ((uint32_t)__ldg(b + 3 * k + 1) << 8) |
                 ((uint32_t)__ldg(b + 3 * k + 2) << 16);
      p0 = q[0] | (kXByte << 24); p1 = q[1] | (kXByte << 24);
      p2 = q[2] | (kXByte << 24); p3 = q[3] | (kXByte << 24);
    }
    *reinterpret_cast<uint4 *>(dst) = make_uint4(p0, p1, p2, p3);
  }
}

// Bilinear sample from a staged window (taps clamped into the window), float32.
template <int kStride>
__device__ __forceinline__ float3 win_bilinear(const uint32_t *s, const Window &W, float sx, float sy) {
  int ix, iy;
  float fx, fy;
  split(sx, ix, fx);
  split(sy, iy, fy);
  int lx = ix - W.x0, ly = iy - W.y0;
  // A sample exactly on the window's last column / row, (last, 0), is the
  // same as (last - 1, 1); the clamps below only guard memory.
  if (lx > W.w - 2) { lx = W.w - 2; fx = 1.0f; }
  if (ly > W.h - 2) { ly = W.h - 2; fy = 1.0f; }
  lx = max(lx, 0);
  ly = max(ly, 0);
  const uint32_t *p = s + ly * kStride + lx;
  return bilerp_words(p[0], p[1], p[kStride], p[kStride + 1], fx, fy);
}

// Luminance sum L = R + 2G + B of an RGBX word (exact, one dot product).
__device__ __forceinline__ float luma_word(uint32_t w) {
  return (float)__dp4a(w, 0x00010201u, 0u);
}

// The bilinear sample of L at (sx, sy) from a staged window (taps clamped
// into the window as in win_bilinear): L of each tap, interpolated once,
// which is the interpolated channels' R + 2G + B with fewer roundings.
template <int kStride>
__device__ __forceinline__ float win_luma(const uint32_t *s, const Window &W, float sx, float sy) {
  int ix, iy;
  float fx, fy;
  split(sx, ix, fx);
  split(sy, iy, fy);
  int lx = ix - W.x0, ly = iy - W.y0;
  if (lx > W.w - 2) { lx = W.w - 2; fx = 1.0f; }
  if (ly > W.h - 2) { ly = W.h - 2; fy = 1.0f; }
  lx = max(lx, 0);
  ly = max(ly, 0);
  const uint32_t *p = s + ly * kStride + lx;
  const float A = luma_word(p[0]), B = luma_word(p[1]), D = luma_word(p[kStride]), E = luma_word(p[kStride + 1]);
  const float top = fmaf(fx, B - A, A);
  const float bot = fmaf(fx, E - D, D);
  return fmaf(fy, bot - top, top);
}

// The same from the frame in global memory (windows that did not fit).
__device__ __forceinline__ float src_luma(const uint8_t *__restrict__ src, const CamDev &c, float sx, float sy) {
  int ix, iy;
  float fx, fy;
  split(sx, ix, fx);
  split(sy, iy, fy);
  ix = min(max(ix, 0), c.w - 1);
  iy = min(max(iy, 0), c.h_px - 1);
  const int ix1 = min(ix + 1, c.w - 1), iy1 = min(iy + 1, c.h_px - 1);
  const uint8_t *r0 = src + (size_t)iy * c.pitch;
  const uint8_t *r1 = src + (size_t)iy1 * c.pitch;
  auto L = [](const uint8_t *q) { return (float)((int)__ldg(q) + 2 * (int)__ldg(q + 1) + (int)__ldg(q + 2)); };
  const float A = L(r0 + 3 * ix), B = L(r0 + 3 * ix1), D = L(r1 + 3 * ix), E = L(r1 + 3 * ix1);
  const float top = fmaf(fx, B - A, A);
  const float bot = fmaf(fx, E - D, D);
  return fmaf(fy, bot - top, top);
}

// ---------------------------------------------------------------------------
// Shared memory common to every fuse kernel: colour constants, window
// descriptors, the output table and (multi-rig kernels) the rig's parameters.
// ---------------------------------------------------------------------------

struct BlockColor {
  float M[kMaxCams][9];      // M / 255, so fused values land in [0, 1]
  float bias[kMaxCams][3];   // 128 * sum_c M[c][k] / 255: the correction for taps held as v - 128
  // per camera and output channel k, as register pairs for the f32x2 path:
  // (M[6+k], M[6+k], bias[k], bias[k]) and (M[3+k], M[3+k], M[k], M[k])
  float4 pr[kMaxCams][3][2];
  // per camera and output channel k: (M[k], M[3+k], M[6+k], bias[k])
  float4 col[kMaxCams][3];
};

struct __align__(16) SmemHead {
  FuseParams sp;             // multi-rig kernels: the current rig's parameters
  BlockColor bc;
  Window sW[2];
  int item;
  int rig;
  __align__(16) uint8_t lut[kLutBytes];
  uint32_t ohist[3 * 256];   // STITCH_BALANCE_OUTPUT: the block's share of the pre-balance histogram
};

template <int TW, int TH, int NW>
struct __align__(16) SmemTile {
  __align__(16) uint32_t win[NW][WinGeom<TW, TH>::kAlloc];
  __align__(16) uint8_t out[3][TH][TW];
};

// Shared memory of the single-rig band pre-warp: the two cameras' window
// descriptors and staged windows only (no colour constants or tables), so
// that a one-wave grid fits.
struct __align__(16) SmemPw {
  Window sW[2];
  __align__(16) uint32_t win[2][WinGeom<kTileW, kTileH>::kAlloc];
  uint8_t lum[kTileH][kTileW];            // kFlagPwLuma: the piece's luminance, level 0
  uint8_t lum1[kTileH / 2][kTileW / 2];   // and level 1
};

// The same for the multi-rig band pre-warp, with the item's rig parameters.
struct __align__(16) SmemPwMulti {
  FuseParams sp;
  SmemPw pw;
};

template <int TW, int TH, int NW>
constexpr size_t smem_bytes() {
  return (sizeof(SmemHead) + 15) / 16 * 16 + sizeof(SmemTile<TW, TH, NW>);
}

template <int TW, int TH, int NW>
__device__ __forceinline__ SmemTile<TW, TH, NW> &tile_smem(unsigned char *base) {
  return *reinterpret_cast<SmemTile<TW, TH, NW> *>(base + (sizeof(SmemHead) + 15) / 16 * 16);
}

// The colour constants and the output table of a rig (all threads; the
// caller synchronises before use).
__device__ void load_color(const FuseParams &P, SmemHead &h) {
  const int t = threadIdx.x;
  if (t < kMaxCams * 9) h.bc.M[t / 9][t % 9] = P.color->M[t / 9][t % 9] * (1.0f / 255.0f);
  if (t >= 96 && t < 96 + kMaxCams * 3) {
    const int k = (t - 96) / 3, c = (t - 96) % 3;
    const float *M = P.color->M[k];
    const float m0 = M[c] * (1.0f / 255.0f), m3 = M[3 + c] * (1.0f / 255.0f), m6 = M[6 + c] * (1.0f / 255.0f);
    const float b = (128.0f / 255.0f) * (M[c] + M[3 + c] + M[6 + c]);
    h.bc.bias[k][c] = b;
    h.bc.pr[k][c][0] = make_float4(m6, m6, b, b);
    h.bc.pr[k][c][1] = make_float4(m3, m3, m0, m0);
    h.bc.col[k][c] = make_float4(m0, m3, m6, b);
  }
  const uint4 *src = reinterpret_cast<const uint4 *>(P.lut);
  uint4 *dst = reinterpret_cast<uint4 *>(h.lut);
  for (int i = t; i < kLutBytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
}

// Table index of a fused value u in [0, 1]: round(4080 u), as the low bits of
// u * 4080 + 1.5 * 2^23.
__device__ __forceinline__ uint32_t lut_index(float u) {
  return __float_as_uint(fmaf(u, kLutTop, kMagicRound)) - kMagicRoundBits;
}

// Pre-balance histogram bin of a table index q (the grid of sixteenths):
// floor((q + 8) / 16).
__device__ __forceinline__ uint32_t hist_bin(uint32_t q) { return (q + 8u) >> 4; }

// One pixel's bytes from its fused value v (already scaled by 1/255): the
// saturation is the clamp to [0, 255], the table applies Eq. 5 and rounds.
// hist (or null): the block's pre-balance histogram of covered pixels.
template <int TW, int TH>
__device__ __forceinline__ void put_px(uint8_t (*out)[TH][TW], const uint8_t *lut, int lx, int ly, bool cov, float3 v,
                                       uint32_t *hist = nullptr) {
  uint32_t o0 = 0u, o1 = 0u, o2 = 0u;
  if (cov) {
    const uint32_t q0 = lut_index(__saturatef(v.x)), q1 = lut_index(__saturatef(v.y));
    const uint32_t q2 = lut_index(__saturatef(v.z));
    o0 = lut[q0];
    o1 = lut[kLutEntries + q1];
    o2 = lut[2 * kLutEntries + q2];
    if (hist) {
      atomicAdd(&hist[hist_bin(q0)], 1u);
      atomicAdd(&hist[256 + hist_bin(q1)], 1u);
      atomicAdd(&hist[512 + hist_bin(q2)], 1u);
    }
  }
  out[0][ly][lx] = (uint8_t)o0;
  out[1][ly][lx] = (uint8_t)o1;
  out[2][ly][lx] = (uint8_t)o2;
}

// The piece's chunks of the tile (columns [16 c0, 16 c1)) as 16-byte stores.
template <int TW, int TH>
__device__ __forceinline__ void store_tile(const FuseParams &P, int tx0, int ty0, const uint8_t (*s_out)[TH][TW],
                                           int c0, int c1) {
  constexpr int kPieces = TW / 16;
  for (int t = threadIdx.x; t < 3 * TH * kPieces; t += blockDim.x) {
    const int c = t / (TH * kPieces);
    const int r = (t / kPieces) % TH;
    const int q = t % kPieces;
    const int y = ty0 + r, x = tx0 + 16 * q;
    if (q < c0 || q >= c1 || y >= P.pano_h || x >= P.pano_pitch) continue;
    const uint4 v = *reinterpret_cast<const uint4 *>(&s_out[c][r][16 * q]);
    *reinterpret_cast<uint4 *>(P.out + (size_t)c * P.pano_pitch * P.pano_h + (size_t)y * P.pano_pitch + x) = v;
  }
}

// ---------------------------------------------------------------------------
// The paired fast path: two pixels per step, half2 / f32x2 arithmetic.
// ---------------------------------------------------------------------------

// Thread -> pixel pairs of a TW x TH tile. Warp w owns rows
// [w TH / 8, (w + 1) TH / 8). With TW >= 64 a pair is columns (l + 64 cp,
// l + 64 cp + 32) of one row (lane l; bank-conflict-free tap reads); with TW =
// 32 it is column l of two consecutive rows.
template <int TW, int TH>
struct PairMap {
  static constexpr int kG = TW / 32;
  static constexpr int kRPW = TH / 8;
  static constexpr bool kRowPairs = kG == 1;
  static constexpr int kCP = kRowPairs ? 1 : kG / 2;
  static constexpr int kSteps = kRowPairs ? kRPW / 2 : kRPW;
  static constexpr float kDy = kRowPairs ? 2.0f : 1.0f;
  static_assert(TW % 32 == 0 && TH % 16 == 0 && (kG == 1 || kG % 2 == 0), "tile shape");
  __device__ static int lx0(int lane, int cp) { return kRowPairs ? lane : lane + 64 * cp; }
  __device__ static int lx1(int lane, int cp) { return kRowPairs ? lane : lane + 64 * cp + 32; }
  __device__ static int ly0(int warp, int s) { return kRPW * warp + (kRowPairs ? 2 * s : s); }
  __device__ static int ly1(int warp, int s) { return ly0(warp, s) + (kRowPairs ? 1 : 0); }
};

// The half-shifted camera map (hm) of a pixel pair: n = col + row * hy with
// components (x, y, w) and s' = (n.x / n.w, n.y / n.w) = s - (1/2, 1/2), the
// same products in the same order as cam_point. col holds a column's share
// (planar: the camera-relative panorama column; cylinder: its sin / cos),
// row the row coordinate (planar: the camera-relative row, exact; cylinder:
// (y - cy) / f, formed from the exact row for every step).
struct PairCoords {
  float2 cx[2], cy[2], cw[2];   // per column pair: both pixels' column shares
  float2 y0;                    // both pixels' panorama row at step 0 (exact)
};

template <int TW, int TH>
__device__ __forceinline__ PairCoords pair_coords(const CamDev &c, int tx0, int ty0, int lane, int warp) {
  using PM = PairMap<TW, TH>;
  PairCoords pc;
#pragma unroll
  for (int cp = 0; cp < 2; ++cp) {
    if (cp >= PM::kCP) break;
    float a0, b0, a1, b1;   // (first, second) column factors of both pixels
    const int x0 = tx0 + PM::lx0(lane, cp), x1 = tx0 + PM::lx1(lane, cp);
    if (c.cyl) {
      sincosf(((float)x0 - c.cyl_cx) * c.cyl_finv, &a0, &b0);
      sincosf(((float)x1 - c.cyl_cx) * c.cyl_finv, &a1, &b1);
    } else {
      a0 = (float)(x0 - c.ox);
      a1 = (float)(x1 - c.ox);
      b0 = b1 = 1.0f;
    }
    pc.cx[cp] = f2(fmaf(c.hm[0], a0, c.hm[2] * b0), fmaf(c.hm[0], a1, c.hm[2] * b1));
    pc.cy[cp] = f2(fmaf(c.hm[3], a0, c.hm[5] * b0), fmaf(c.hm[3], a1, c.hm[5] * b1));
    pc.cw[cp] = f2(fmaf(c.hm[6], a0, c.hm[8] * b0), fmaf(c.hm[6], a1, c.hm[8] * b1));
  }
  pc.y0 = f2((float)(ty0 + PM::ly0(warp, 0)), (float)(ty0 + PM::ly1(warp, 0)));
  return pc;
}

// Row coordinate of both pixels from their exact panorama rows.
__device__ __forceinline__ float2 pair_row(const CamDev &c, float2 y) {
  if (c.cyl) return __fmul2_rn(__fadd2_rn(y, f2(-c.cyl_cy)), f2(c.cyl_finv));
  return __fadd2_rn(y, f2(-(float)c.oy));
}

// s' of a pixel pair (the division skipped for an affine camera).
__device__ __forceinline__ void pair_point(const CamDev &c, const PairCoords &pc, int cp, float2 row, float2 &ux,
                                           float2 &uy) {
  const float2 nx = __ffma2_rn(row, f2(c.hm[1]), pc.cx[cp]);
  const float2 ny = __ffma2_rn(row, f2(c.hm[4]), pc.cy[cp]);
  if (c.affine) {
    ux = nx;
    uy = ny;
  } else {
    const float2 nw = __ffma2_rn(row, f2(c.hm[7]), pc.cw[cp]);
    const float2 rw = f2(rcp_approx(nw.x), rcp_approx(nw.y));
    ux = __fmul2_rn(nx, rw);
    uy = __fmul2_rn(ny, rw);
  }
}

// Half-shifted source points um of a pixel pair -> the magic-rounded floats
// (whose bits are kMagicRoundBits + tap index) and the fractions in half
// precision.
__device__ __forceinline__ void split_pair(float2 um, float2 &r, __half2 &f) {
  r = __fadd2_rn(um, f2(kMagicRound));
  const float2 n = __fadd2_rn(r, f2(-kMagicRound));
  const float2 d = __ffma2_rn(n, f2(-1.0f), um);   // um - round(um), in [-1/2, 1/2], exact
  f = __float22half2_rn(__fadd2_rn(d, f2(0.5f)));
}

// Half2 channel pair (1024 + v of pixel 0, 1024 + v of pixel 1) from two RGBX
// words with the fourth byte 0x64.
template <int C>
__device__ __forceinline__ __half2 chan_pair(uint32_t w0, uint32_t w1) {
  return as_h2(__byte_perm(w0, w1, 0x7430u + 0x0101u * C));
}

// Bilinear of a pixel pair per channel, in half2 on v - 128:
// a + fx (b - a) + fy ((d - a) + fx ((e - d) - (b - a))).
__device__ __forceinline__ void bilerp_pair(const uint32_t (&t0)[4], const uint32_t (&t1)[4], __half2 fx, __half2 fy,
                                            float2 (&v)[3]) {
  const __half2 off = __float2half2_rn(kHalfOffset);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    __half2 A, B, D, E;
    if (c == 0) {
      A = chan_pair<0>(t0[0], t1[0]); B = chan_pair<0>(t0[1], t1[1]);
      D = chan_pair<0>(t0[2], t1[2]); E = chan_pair<0>(t0[3], t1[3]);
    } else if (c == 1) {
      A = chan_pair<1>(t0[0], t1[0]); B = chan_pair<1>(t0[1], t1[1]);
      D = chan_pair<1>(t0[2], t1[2]); E = chan_pair<1>(t0[3], t1[3]);
    } else {
      A = chan_pair<2>(t0[0], t1[0]); B = chan_pair<2>(t0[1], t1[1]);
      D = chan_pair<2>(t0[2], t1[2]); E = chan_pair<2>(t0[3], t1[3]);
    }
    const __half2 dx = __hsub2(B, A);
    const __half2 dy = __hsub2(D, A);
    const __half2 dxy = __hsub2(__hsub2(E, D), dx);
    const __half2 a = __hsub2(A, off);
    const __half2 u = __hfma2(fx, dxy, dy);
    const __half2 t = __hfma2(fx, dx, a);
    v[c] = __half22float2(__hfma2(fy, u, t));
  }
}

// The four taps of a pixel at word index i of a window with row stride S.
// The index is clamped to the window's allocation (kMax = kAlloc - S - 2), so
// that no coordinate, however wrong, reads outside it.
template <int S, int kMax>
__device__ __forceinline__ void taps(const uint32_t *w, uint32_t i, uint32_t (&t)[4]) {
  i = min(i, (uint32_t)kMax);
  t[0] = w[i];
  t[1] = w[i + 1];
  t[2] = w[i + S];
  t[3] = w[i + S + 1];
}

// v . M + bias through the table for a pixel pair (v held as v - 128), the
// products in cam_value's order; pr holds the camera's colour pairs (in
// shared memory or registers).
template <int TW, int TH, typename PR>
__device__ __forceinline__ void finish_pair(const float2 (&v)[3], const PR &pr, const uint8_t *lut,
                                            uint8_t (*out)[TH][TW], int lx0, int ly0, int lx1, int ly1, bool in0,
                                            bool in1, uint32_t *hist) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 a = pr[k][0], b = pr[k][1];
    float2 acc = __ffma2_rn(v[2], f2(a.x, a.y), f2(a.z, a.w));
    acc = __ffma2_rn(v[1], f2(b.x, b.y), acc);
    const float u0 = __saturatef(fmaf(v[0].x, b.z, acc.x));
    const float u1 = __saturatef(fmaf(v[0].y, b.w, acc.y));
    const float2 q = __ffma2_rn(f2(u0, u1), f2(kLutTop), f2(kMagicRound));
    const uint32_t q0 = __float_as_uint(q.x) - kMagicRoundBits, q1 = __float_as_uint(q.y) - kMagicRoundBits;
    if (in0) out[k][ly0][lx0] = lut[k * kLutEntries + q0];
    if (in1) out[k][ly1][lx1] = lut[k * kLutEntries + q1];
    if (hist) {
      if (in0) atomicAdd(&hist[256 * k + hist_bin(q0)], 1u);
      if (in1) atomicAdd(&hist[256 * k + hist_bin(q1)], 1u);
    }
  }
}

// Every pixel of a fully covered own tile from its staged window (W.ok): the
// tile lies inside camera k with a margin, so every tap is a frame pixel of
// the window and the result equals cam_value's for each pixel. kAll: the
// piece holds every column of the tile (no column tests); kHist: the block's
// pre-balance histogram is kept.
template <int TW, int TH, bool kAll, bool kHist>
__device__ __forceinline__ void own_pairs(const CamDev &c, const Window &W, const uint32_t *win, const BlockColor &bc,
                                          int k, const uint8_t *lut, uint8_t (*out)[TH][TW], int tx0, int ty0,
                                          int cx0, int cx1, uint32_t *hist) {
  using PM = PairMap<TW, TH>;
  constexpr int S = WinGeom<TW, TH>::kStride;
  constexpr int kMax = WinGeom<TW, TH>::kAlloc - S - 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // word index of tap (ix, iy) = bits(ry) S + bits(rx) - off
  const uint32_t off = kMagicRoundBits * (uint32_t)(S + 1) + (uint32_t)W.y0 * (uint32_t)S + (uint32_t)W.x0;
  const PairCoords pc = pair_coords<TW, TH>(c, tx0, ty0, lane, warp);
  float4 prc[3][2];   // the camera's colour pairs, held in registers for the tile
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    prc[q][0] = bc.pr[k][q][0];
    prc[q][1] = bc.pr[k][q][1];
  }
  float2 y = pc.y0;
#pragma unroll 2
  for (int s = 0; s < PM::kSteps; ++s) {
    const float2 row = pair_row(c, y);
#pragma unroll
    for (int cp = 0; cp < PM::kCP; ++cp) {
      float2 ux, uy;
      pair_point(c, pc, cp, row, ux, uy);
      float2 rx, ry;
      __half2 fx, fy;
      split_pair(ux, rx, fx);
      split_pair(uy, ry, fy);
      const uint32_t i0 = __float_as_uint(ry.x) * (uint32_t)S + __float_as_uint(rx.x) - off;
      const uint32_t i1 = __float_as_uint(ry.y) * (uint32_t)S + __float_as_uint(rx.y) - off;
      uint32_t t0[4], t1[4];
      taps<S, kMax>(win, i0, t0);
      taps<S, kMax>(win, i1, t1);
      float2 v[3];
      bilerp_pair(t0, t1, fx, fy, v);
      const int lx0 = PM::lx0(lane, cp), lx1 = PM::lx1(lane, cp);
      finish_pair<TW, TH>(v, prc, lut, out, lx0, PM::ly0(warp, s), lx1, PM::ly1(warp, s),
                          kAll || (lx0 >= cx0 && lx0 < cx1), kAll || (lx1 >= cx0 && lx1 < cx1),
                          kHist ? hist : nullptr);
    }
    y = __fadd2_rn(y, f2(PM::kDy));
  }
}

// ---------------------------------------------------------------------------
// Per-pixel general path: the same arithmetic as the paired path, one pixel
// at a time (its second half2 lane repeats the first), so that a pixel's
// bytes do not depend on the tile shape, the tile kind or the batch.
// ---------------------------------------------------------------------------

// Half-shifted source point s' = s - (1/2, 1/2) of panorama pixel (x, y) in
// camera c, from the half-shifted map hm (the paired path evaluates the same
// products in the same order: column share first, then the row).
__device__ __forceinline__ void cam_point(const CamDev &c, int x, int y, float &sx, float &sy, float &nw) {
  float a, b, rc;
  if (c.cyl) {
    sincosf(((float)x - c.cyl_cx) * c.cyl_finv, &a, &b);
    rc = ((float)y - c.cyl_cy) * c.cyl_finv;
  } else {
    a = (float)(x - c.ox);
    b = 1.0f;
    rc = (float)(y - c.oy);
  }
  const float cx = fmaf(c.hm[0], a, c.hm[2] * b);
  const float cy = fmaf(c.hm[3], a, c.hm[5] * b);
  const float cw = fmaf(c.hm[6], a, c.hm[8] * b);
  const float nx = fmaf(rc, c.hm[1], cx), ny = fmaf(rc, c.hm[4], cy);
  nw = fmaf(rc, c.hm[7], cw);
  if (c.affine) {
    sx = nx;
    sy = ny;
  } else {
    const float r = rcp_approx(nw);
    sx = __fmul_rn(nx, r);
    sy = __fmul_rn(ny, r);
  }
}

// Coverage of Eq. 15 in half-shifted coordinates: 0 <= s <= (w - 1, h - 1).
__device__ __forceinline__ bool covered_m(const CamDev &c, float sx, float sy, float nw) {
  return nw > 0.0f && sx >= -0.5f && sx <= c.wm1 - 0.5f && sy >= -0.5f && sy <= c.hm1 - 0.5f;
}

// One RGBX word (fourth byte 0x64) of frame pixel (x, y) from global memory.
__device__ __forceinline__ uint32_t gword(const uint8_t *__restrict__ src, const CamDev &c, int x, int y) {
  const uint8_t *p = src + (size_t)y * c.pitch + 3 * x;
  return (uint32_t)__ldg(p) | ((uint32_t)__ldg(p + 1) << 8) | ((uint32_t)__ldg(p + 2) << 16) | (kXByte << 24);
}

// Camera k's colour-transferred value at panorama pixel (x, y) in the offset
// form (bias + (P - 128) . M / 255, not yet saturated), or false where k does
// not cover the pixel. Taps: floor(s) and floor(s) + 1, the far tap clamped
// to the last row / column; read from the staged window when all four lie in
// it, else from the frame.
template <int S>
__device__ bool cam_value(const FuseParams &P, const BlockColor &bc, int k, const Window &W, const uint32_t *win,
                          int x, int y, float3 &o) {
  const CamDev &c = P.cam[k];
  float sx, sy, nw;
  cam_point(c, x, y, sx, sy, nw);
  if (!covered_m(c, sx, sy, nw)) return false;
  const float rx = sx + kMagicRound, ry = sy + kMagicRound;
  const float fx = (sx - (rx - kMagicRound)) + 0.5f, fy = (sy - (ry - kMagicRound)) + 0.5f;
  const int ix = max((int)(__float_as_uint(rx) - kMagicRoundBits), 0);
  const int iy = max((int)(__float_as_uint(ry) - kMagicRoundBits), 0);
  const int ix1 = min(ix + 1, c.w - 1), iy1 = min(iy + 1, c.h_px - 1);
  uint32_t t[4];
  const int lx = ix - W.x0, ly = iy - W.y0;
  if (W.ok && lx >= 0 && ly >= 0 && ix1 - W.x0 < W.w && iy1 - W.y0 < W.h) {
    const int dx = ix1 - ix, dy = (iy1 - iy) * S;
    const uint32_t *q = win + ly * S + lx;
    t[0] = q[0]; t[1] = q[dx]; t[2] = q[dy]; t[3] = q[dy + dx];
  } else {
    const uint8_t *src = P.src[k];
    t[0] = gword(src, c, ix, iy); t[1] = gword(src, c, ix1, iy);
    t[2] = gword(src, c, ix, iy1); t[3] = gword(src, c, ix1, iy1);
  }
  float2 v[3];
  bilerp_pair(t, t, __float2half2_rn(fx), __float2half2_rn(fy), v);
  const float *M = bc.M[k], *bias = bc.bias[k];
  o.x = fmaf(v[0].x, M[0], fmaf(v[1].x, M[3], fmaf(v[2].x, M[6], bias[0])));
  o.y = fmaf(v[0].x, M[1], fmaf(v[1].x, M[4], fmaf(v[2].x, M[7], bias[1])));
  o.z = fmaf(v[0].x, M[2], fmaf(v[1].x, M[5], fmaf(v[2].x, M[8], bias[2])));
  return true;
}

// Camera k's value with the one-image fallbacks of Eq. 15 (k, then k - 1,
// then k + 1 when those exist): true when any of them covers the pixel.
template <int S>
__device__ __forceinline__ bool own_value(const FuseParams &P, const BlockColor &bc, int k, int first, int second,
                                          const Window &W, const uint32_t *win, int x, int y, float3 &o) {
  if (cam_value<S>(P, bc, k, W, win, x, y, o)) return true;
  const Window none = no_window();
  if (first >= 0 && first < P.n_cams && cam_value<S>(P, bc, first, none, win, x, y, o)) return true;
  return second >= 0 && second < P.n_cams && cam_value<S>(P, bc, second, none, win, x, y, o);
}

template <int TW, int TH>
__device__ __forceinline__ void ownpart_pairs(const FuseParams &P, const BlockColor &bc, int k, const Window &W,
                                              const uint32_t *win, const uint8_t *lut, uint8_t (*out)[TH][TW],
                                              int tx0, int ty0, int cx0, int cx1, uint32_t *hist) {
  using PM = PairMap<TW, TH>;
  constexpr int S = WinGeom<TW, TH>::kStride;
  constexpr int kMax = WinGeom<TW, TH>::kAlloc - S - 2;
  const CamDev &c = P.cam[k];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t off = kMagicRoundBits * (uint32_t)(S + 1) + (uint32_t)W.y0 * (uint32_t)S + (uint32_t)W.x0;
  const uint32_t wx = (uint32_t)W.w - 1u, wy = (uint32_t)W.h - 1u;   // last window column / row with a right tap
  const float hx = c.wm1 - 0.5f, hy = c.hm1 - 0.5f;
  const PairCoords pc = pair_coords<TW, TH>(c, tx0, ty0, lane, warp);
  float2 y = pc.y0;
#pragma unroll 1
  for (int s = 0; s < PM::kSteps; ++s) {
    const float2 row = pair_row(c, y);
#pragma unroll
    for (int cp = 0; cp < PM::kCP; ++cp) {
      const int lx0 = PM::lx0(lane, cp), lx1 = PM::lx1(lane, cp);
      const int ly0 = PM::ly0(warp, s), ly1 = PM::ly1(warp, s);
      const bool col0 = lx0 >= cx0 && lx0 < cx1, col1 = lx1 >= cx0 && lx1 < cx1;
      const bool in0 = col0 && tx0 + lx0 < P.pano_w && ty0 + ly0 < P.pano_h;
      const bool in1 = col1 && tx0 + lx1 < P.pano_w && ty0 + ly1 < P.pano_h;
      // the piece's pixels past the panorama's last column (row padding) are 0
      if (col0 && !in0) put_px<TW, TH>(out, lut, lx0, ly0, false, make_float3(0.0f, 0.0f, 0.0f));
      if (col1 && !in1) put_px<TW, TH>(out, lut, lx1, ly1, false, make_float3(0.0f, 0.0f, 0.0f));
      float2 ux, uy;
      pair_point(c, pc, cp, row, ux, uy);
      const float2 nw = __ffma2_rn(row, f2(c.hm[7]), pc.cw[cp]);
      float2 rx, ry;
      __half2 fx, fy;
      split_pair(ux, rx, fx);
      split_pair(uy, ry, fy);
      // window-relative taps (unsigned: a tap left of / above the window wraps)
      const uint32_t wx0 = __float_as_uint(rx.x) - kMagicRoundBits - (uint32_t)W.x0;
      const uint32_t wx1 = __float_as_uint(rx.y) - kMagicRoundBits - (uint32_t)W.x0;
      const uint32_t wy0 = __float_as_uint(ry.x) - kMagicRoundBits - (uint32_t)W.y0;
      const uint32_t wy1 = __float_as_uint(ry.y) - kMagicRoundBits - (uint32_t)W.y0;
      const bool ok0 = nw.x > 0.0f && ux.x >= -0.5f && ux.x <= hx && uy.x >= -0.5f && uy.x <= hy && wx0 < wx && wy0 < wy;
      const bool ok1 = nw.y > 0.0f && ux.y >= -0.5f && ux.y <= hx && uy.y >= -0.5f && uy.y <= hy && wx1 < wx && wy1 < wy;
      if (W.ok && (ok0 || !in0) && (ok1 || !in1)) {
        const uint32_t i0 = __float_as_uint(ry.x) * (uint32_t)S + __float_as_uint(rx.x) - off;
        const uint32_t i1 = __float_as_uint(ry.y) * (uint32_t)S + __float_as_uint(rx.y) - off;
        uint32_t t0[4], t1[4];
        taps<S, kMax>(win, i0, t0);
        taps<S, kMax>(win, i1, t1);
        float2 v[3];
        bilerp_pair(t0, t1, fx, fy, v);
        finish_pair<TW, TH>(v, bc.pr[k], lut, out, lx0, ly0, lx1, ly1, in0, in1, hist);
      } else {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const bool in = q ? in1 : in0;
          if (!in) continue;
          const int lx = q ? lx1 : lx0, ly = q ? ly1 : ly0;
          float3 v = make_float3(0.0f, 0.0f, 0.0f);
          const bool cov = own_value<S>(P, bc, k, k - 1, k + 1, W, win, tx0 + lx, ty0 + ly, v);
          put_px<TW, TH>(out, lut, lx, ly, cov, v, hist);
        }
      }
    }
    y = __fadd2_rn(y, f2(PM::kDy));
  }
}

// ---------------------------------------------------------------------------
// Band intermediate of the frame path: v - 128 per band pixel and side as
// four halves (R, G, B, 0). The values are exact halves (the half2 bilinear's
// results), so the float32 remap reads them without loss.
// ---------------------------------------------------------------------------

// Bilinear of four intermediate taps (a, b: row ly; d, e: row ly + 1) with
// fractions (gx, gy), float32: the three channels.
__device__ __forceinline__ float3 lerp4(float4 a, float4 b, float4 d, float4 e, float gx, float gy) {
  const float2 A = f2(a.x, a.y), B = f2(b.x, b.y), D = f2(d.x, d.y), E = f2(e.x, e.y);
  const float2 dx = __ffma2_rn(A, f2(-1.0f), B);
  const float2 dy = __ffma2_rn(A, f2(-1.0f), D);
  const float2 dxy = __ffma2_rn(dx, f2(-1.0f), __ffma2_rn(D, f2(-1.0f), E));
  const float2 o = __ffma2_rn(f2(gy), __ffma2_rn(f2(gx), dxy, dy), __ffma2_rn(f2(gx), dx, A));
  const float bx = b.z - a.z, by = d.z - a.z, bxy = (e.z - d.z) - bx;
  const float oz = fmaf(gy, fmaf(gx, bxy, by), fmaf(gx, bx, a.z));
  return make_float3(o.x, o.y, oz);
}

// The same for half taps (four halves R, G, B, 0 per tap), in half2.
__device__ __forceinline__ float3 lerp_h(uint2 a, uint2 b, uint2 d, uint2 e, float gx, float gy) {
  const __half2 hx = __float2half2_rn(gx), hy = __float2half2_rn(gy);
  float2 o[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const __half2 A = as_h2(h ? a.y : a.x), B = as_h2(h ? b.y : b.x);
    const __half2 D = as_h2(h ? d.y : d.x), E = as_h2(h ? e.y : e.x);
    const __half2 dx = __hsub2(B, A), dy = __hsub2(D, A);
    const __half2 dxy = __hsub2(__hsub2(E, D), dx);
    o[h] = __half22float2(__hfma2(hy, __hfma2(hx, dxy, dy), __hfma2(hx, dx, A)));
  }
  return make_float3(o[0].x, o[0].y, o[1].x);
}

// A half tap as the float32 intermediate holds it (exact).
__device__ __forceinline__ float4 h4f(uint2 u) {
  const float2 rg = __half22float2(as_h2(u.x));
  return make_float4(rg.x, rg.y, __low2float(as_h2(u.y)), 0.0f);
}

// Bilinear of the intermediate at band-relative tap (lx, ly) with fractions
// (gx, gy); the neighbours are (lx1, ly1). kHalf: half2 arithmetic
// (STITCH_FP16_INTERMEDIATE), else float32. Returns the three channels.
template <bool kHalf>
__device__ __forceinline__ float3 pw_lerp(const uint2 *pw, int bw, int lx, int ly, int lx1, int ly1, float gx,
                                          float gy) {
  const uint2 a = __ldg(pw + (size_t)ly * bw + lx), b = __ldg(pw + (size_t)ly * bw + lx1);
  const uint2 d = __ldg(pw + (size_t)ly1 * bw + lx), e = __ldg(pw + (size_t)ly1 * bw + lx1);
  if (kHalf) return lerp_h(a, b, d, e, gx, gy);
  return lerp4(h4f(a), h4f(b), h4f(d), h4f(e), gx, gy);
}

// Tap of a remap sample: the band-relative tap (lx, ly), the step to its
// right / lower neighbour (0 where clamped at the band's last column / row)
// and the fractions; band_sample's arithmetic.
struct BandTap {
  int lx, ly, dx, dy;
  float gx, gy;
};

template <bool kClamp>
__device__ __forceinline__ BandTap band_tap_of(float2 qm, int bw, int bh) {
  if (kClamp) {
    qm.x = fminf(fmaxf(qm.x, -0.5f), (float)bw - 1.5f);
    qm.y = fminf(fmaxf(qm.y, -0.5f), (float)bh - 1.5f);
  }
  const float2 r = __fadd2_rn(qm, f2(kMagicRound));
  const float2 d = __ffma2_rn(__fadd2_rn(r, f2(-kMagicRound)), f2(-1.0f), qm);
  BandTap t;
  t.lx = (int)(__float_as_uint(r.x) - kMagicRoundBits);
  t.ly = (int)(__float_as_uint(r.y) - kMagicRoundBits);
  t.gx = d.x + 0.5f;
  t.gy = d.y + 0.5f;
  t.dx = 1;
  t.dy = 1;
  if (kClamp) {
    if (t.lx < 0) { t.lx = 0; t.gx = 0.0f; }
    if (t.ly < 0) { t.ly = 0; t.gy = 0.0f; }
    t.lx = min(t.lx, bw - 1);
    t.ly = min(t.ly, bh - 1);
    t.dx = min(t.lx + 1, bw - 1) - t.lx;
    t.dy = min(t.ly + 1, bh - 1) - t.ly;
  }
  return t;
}

// Remap sample P_k(X) (Eq. 18) of a band's intermediate at the band-relative,
// half-shifted point qm = X - (x0, y0) - 1/2. kClamp: X may lie outside the
// band (clamped into it first) and taps may fall on its last row / column.
template <bool kHalf, bool kClamp>
__device__ __forceinline__ float3 band_sample(const uint2 *pw, int bw, int bh, float2 qm) {
  const BandTap t = band_tap_of<kClamp>(qm, bw, bh);
  return pw_lerp<kHalf>(pw, bw, t.lx, t.ly, t.lx + t.dx, t.ly + t.dy, t.gx, t.gy);
}

// A band pixel (x, y) inside the band rectangle of pair p (Eq. 16-18 and the
// weighted mean of Eq. 15), as the fused value scaled by 1/255.
template <bool kHalf, bool kClamp>
__device__ __forceinline__ float3 band_pixel(const FuseParams &P, const BlockColor &bc, int p, int x, int y,
                                             bool printed) {
  using PT = uint2;
  const BandDev B = P.band[p];
  const int bw = B.x1 - B.x0, bh = B.y1 - B.y0;
  const float mf = P.max_flow;
  const size_t fi = (size_t)(y - B.y0) * bw + (x - B.x0);
  float2 fa = __ldg(P.flow_ij[p] + fi);
  float2 fb = __ldg(P.flow_ji[p] + fi);
  fa.x = fmaxf(fminf(fa.x, mf), -mf); fa.y = fmaxf(fminf(fa.y, mf), -mf);
  fb.x = fmaxf(fminf(fb.x, mf), -mf); fb.y = fmaxf(fminf(fb.y, mf), -mf);
  const float tb = __fmul_rn((float)(x - B.x0) + 0.5f, B.inv_bw);
  const float ta = 1.0f - tb;
  const float wa = printed ? ta : tb;
  const float wb = printed ? tb : ta;
  const float2 base = f2((float)(x - B.x0) - 0.5f, (float)(y - B.y0) - 0.5f);
  const PT *pwa = reinterpret_cast<const PT *>(P.pw) + P.pw_off[p][0];
  const PT *pwb = reinterpret_cast<const PT *>(P.pw) + P.pw_off[p][1];
  const float3 Pa = band_sample<kHalf, kClamp>(pwa, bw, bh, __ffma2_rn(f2(wa), fa, base));
  const float3 Pb = band_sample<kHalf, kClamp>(pwb, bw, bh, __ffma2_rn(f2(wb), fb, base));
  const float *Ma = bc.M[p], *Mb = bc.M[p + 1];
  const float *ba = bc.bias[p], *bb = bc.bias[p + 1];
  float3 o;
  o.x = fmaf(tb, fmaf(Pb.x, Mb[0], fmaf(Pb.y, Mb[3], fmaf(Pb.z, Mb[6], bb[0]))),
             ta * fmaf(Pa.x, Ma[0], fmaf(Pa.y, Ma[3], fmaf(Pa.z, Ma[6], ba[0]))));
  o.y = fmaf(tb, fmaf(Pb.x, Mb[1], fmaf(Pb.y, Mb[4], fmaf(Pb.z, Mb[7], bb[1]))),
             ta * fmaf(Pa.x, Ma[1], fmaf(Pa.y, Ma[4], fmaf(Pa.z, Ma[7], ba[1]))));
  o.z = fmaf(tb, fmaf(Pb.x, Mb[2], fmaf(Pb.y, Mb[5], fmaf(Pb.z, Mb[8], bb[2]))),
             ta * fmaf(Pa.x, Ma[2], fmaf(Pa.y, Ma[5], fmaf(Pa.z, Ma[8], ba[2]))));
  return o;
}

// ---------------------------------------------------------------------------
// Tiles.
// ---------------------------------------------------------------------------

// Shared memory of a band piece: only the output tile.
template <int TW, int TH>
struct __align__(16) SmemBand {
  __align__(16) uint8_t out[3][TH][TW];
};

template <int TW, int TH>
constexpr size_t band_smem_bytes() {
  return (sizeof(SmemHead) + 15) / 16 * 16 + sizeof(SmemBand<TW, TH>);
}

// A fully covered own piece (kTileOwn): window of its columns, staging,
// paired per-pixel work, stores. Pieces whose window does not fit take the
// general per-pixel path with taps from the frame.
template <int TW, int TH>
__device__ __forceinline__ void fuse_own_tile(const FuseParams &P, const TileDesc t, SmemHead &h,
                                              SmemTile<TW, TH, 1> &st) {
  using G = WinGeom<TW, TH>;
  const int tx0 = t.tx * TW, ty0 = t.ty * TH;
  const int cx0 = 16 * t.c0, cx1 = 16 * t.c1;
  const int ty1 = min(ty0 + TH, P.pano_h) - 1;
  const int warp = threadIdx.x >> 5;
  const int k = t.idx;
  const CamDev &c = P.cam[k];
  if (warp == 0) {
    const Window W = warp_window<G::kStride, G::kRows>(c, tx0 + cx0, ty0, tx0 + cx1 - 1, ty1, rows16(P.src[k], c));
    if ((threadIdx.x & 31) == 0) {
      h.sW[0] = W;
      if (W.over && P.win_fallback) atomicAdd(P.win_fallback, 1u);
    }
  }
  __syncthreads();
  const Window W0 = h.sW[0];
  if (W0.ok) {
    stage_window<G::kStride>(P.src[k], c, W0, st.win[0]);
    __syncthreads();
    const bool all = t.c0 == 0 && t.c1 == TW / 16;
    if (P.out_hist) {
      if (all)
        own_pairs<TW, TH, true, true>(c, W0, st.win[0], h.bc, k, h.lut, st.out, tx0, ty0, cx0, cx1, h.ohist);
      else
        own_pairs<TW, TH, false, true>(c, W0, st.win[0], h.bc, k, h.lut, st.out, tx0, ty0, cx0, cx1, h.ohist);
    } else {
      if (all)
        own_pairs<TW, TH, true, false>(c, W0, st.win[0], h.bc, k, h.lut, st.out, tx0, ty0, cx0, cx1, nullptr);
      else
        own_pairs<TW, TH, false, false>(c, W0, st.win[0], h.bc, k, h.lut, st.out, tx0, ty0, cx0, cx1, nullptr);
    }
  } else {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < (TW / 32) * (TH / 8); ++j) {
      const int lx = lane + 32 * (j % (TW / 32)), ly = (TH / 8) * warp + j / (TW / 32);
      if (lx < cx0 || lx >= cx1) continue;
      float3 v = make_float3(0.0f, 0.0f, 0.0f);
      const bool cov = cam_value<G::kStride>(P, h.bc, k, W0, st.win[0], tx0 + lx, ty0 + ly, v);
      put_px<TW, TH>(st.out, h.lut, lx, ly, cov, v, P.out_hist ? h.ohist : nullptr);
    }
  }
  __syncthreads();
  store_tile<TW, TH>(P, tx0, ty0, st.out, t.c0, t.c1);
}

// One remap sample (Eq. 18) of a band's intermediate at the band-relative,
// half-shifted point qm (inside the band when !kClamp), returned in the
// intermediate's units; the same arithmetic as band_sample.
template <bool kHalf, bool kClamp>
__device__ __forceinline__ float3 band_tap(const uint2 *pw, int bw, int bh, float2 qm) {
  return band_sample<kHalf, kClamp>(pw, bw, bh, qm);
}

// Every pixel of a piece inside a band rectangle (kTileBand): a band pixel of
// Eq. 16-18 from the band's pre-warped intermediate; no windows. A thread
// walks its columns (theta, the flow column and the band-relative column are
// fixed there) down its rows, with the next pixel's flows loaded before the
// current pixel's remap taps; both cameras' colour constants stay in
// registers. The clamps into the band are skipped when the piece's reach
// (max_flow + 1 pixels around it) stays inside the band.
template <bool kHalf, bool kClamp, int TW, int TH>
__device__ __forceinline__ void band_rows(const FuseParams &P, const BlockColor &bc, int p, int tx0, int ty0, int cx0,
                                          int cx1, const uint8_t *lut, uint8_t (*out)[TH][TW], uint32_t *hist) {
  using PT = uint2;
  constexpr int kGroups = TW / 32, kRPW = TH / 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const BandDev B = P.band[p];
  const int bw = B.x1 - B.x0, bh = B.y1 - B.y0;
  const float mf = P.max_flow;
  const bool printed = (P.flags & STITCH_FLOW_WEIGHTS_PRINTED) != 0;
  const PT *pwa = reinterpret_cast<const PT *>(P.pw) + P.pw_off[p][0];
  const PT *pwb = reinterpret_cast<const PT *>(P.pw) + P.pw_off[p][1];
  const float4 *ca = bc.col[p], *cb = bc.col[p + 1];
  const int ly0 = kRPW * warp;
  const int row0 = ty0 + ly0 - B.y0;       // band-relative row of the thread's first pixel
#pragma unroll 1
  for (int gi = 0; gi < kGroups; ++gi) {
    const int lx = lane + 32 * gi;
    if (lx < cx0 || lx >= cx1) continue;
    const int col = tx0 + lx - B.x0;       // band-relative column
    const float tb = __fmul_rn((float)col + 0.5f, B.inv_bw);
    const float ta = 1.0f - tb;
    const float wa = printed ? ta : tb;
    const float wb = printed ? tb : ta;
    const float2 *fa_p = P.flow_ij[p] + (size_t)row0 * bw + col;
    const float2 *fb_p = P.flow_ji[p] + (size_t)row0 * bw + col;
    float2 base = f2((float)col - 0.5f, (float)row0 - 0.5f);
    float2 fa = __ldg(fa_p), fb = __ldg(fb_p);
#pragma unroll
    for (int r = 0; r < kRPW; ++r) {
      float2 na, nb;
      if (r + 1 < kRPW) {
        na = __ldg(fa_p + (size_t)(r + 1) * bw);
        nb = __ldg(fb_p + (size_t)(r + 1) * bw);
      }
      fa.x = fmaxf(fminf(fa.x, mf), -mf); fa.y = fmaxf(fminf(fa.y, mf), -mf);
      fb.x = fmaxf(fminf(fb.x, mf), -mf); fb.y = fmaxf(fminf(fb.y, mf), -mf);
      const float3 Pa = band_tap<kHalf, kClamp>(pwa, bw, bh, __ffma2_rn(f2(wa), fa, base));
      const float3 Pb = band_tap<kHalf, kClamp>(pwb, bw, bh, __ffma2_rn(f2(wb), fb, base));
      float o[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float4 A = ca[k], Bq = cb[k];
        o[k] = fmaf(tb, fmaf(Pb.x, Bq.x, fmaf(Pb.y, Bq.y, fmaf(Pb.z, Bq.z, Bq.w))),
                    ta * fmaf(Pa.x, A.x, fmaf(Pa.y, A.y, fmaf(Pa.z, A.z, A.w))));
      }
      put_px<TW, TH>(out, lut, lx, ly0 + r, true, make_float3(o[0], o[1], o[2]), hist);
      base.y += 1.0f;
      if (r + 1 < kRPW) {
        fa = na;
        fb = nb;
      }
    }
  }
}

template <bool kHalf, int TW, int TH>
__device__ __forceinline__ void fuse_band_piece(const FuseParams &P, const TileDesc t, SmemHead &h,
                                                uint8_t (*out)[TH][TW]) {
  const int tx0 = t.tx * TW, ty0 = t.ty * TH;
  const int cx0 = 16 * t.c0, cx1 = 16 * t.c1;
  const int p = t.idx;
  const BandDev B = P.band[p];
  const int reach = (int)ceilf(P.max_flow) + 1;
  const bool interior = tx0 + cx0 - reach >= B.x0 && tx0 + cx1 - 1 + reach + 1 < B.x1 && ty0 - reach >= B.y0 &&
                        ty0 + TH - 1 + reach + 1 < B.y1;
  uint32_t *hist = P.out_hist ? h.ohist : nullptr;
  if (interior)
    band_rows<kHalf, false, TW, TH>(P, h.bc, p, tx0, ty0, cx0, cx1, h.lut, out, hist);
  else
    band_rows<kHalf, true, TW, TH>(P, h.bc, p, tx0, ty0, cx0, cx1, h.lut, out, hist);
  __syncthreads();
  store_tile<TW, TH>(P, tx0, ty0, out, t.c0, t.c1);
}

// A general piece: own columns of camera idx seen only in part
// (kTileOwnPart), or band columns of pair idx with other pixels
// (kTileBandPart: the chunk holding a band edge, rows outside the band
// rectangle). Every pixel takes the per-pixel general path.
template <bool kHalf, int TW, int TH>
__device__ __forceinline__ void fuse_tile(const FuseParams &P, const TileDesc t, SmemHead &h,
                                          SmemTile<TW, TH, 2> &st) {
  using G = WinGeom<TW, TH>;
  constexpr int S = G::kStride;
  const int tx0 = t.tx * TW, ty0 = t.ty * TH;
  const int cx0 = 16 * t.c0, cx1 = 16 * t.c1;
  const int px0 = tx0 + cx0;
  const int px1 = min(tx0 + cx1, P.pano_w) - 1, ty1 = min(ty0 + TH, P.pano_h) - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool empty = px0 > px1 || ty0 > ty1;
  const BlockColor &bc = h.bc;

  // Source windows: warp 0 for the piece's camera (or a band's left camera),
  // warp 1 for a band's right camera, only where its pixels need them.
  if (warp < 2) {
    Window W = no_window();
    bool need = false;
    if (!empty) {
      if (t.kind == kTileOwnPart) {
        need = warp == 0;
        if (need) W = warp_window<S, G::kRows>(P.cam[t.idx], px0, ty0, px1, ty1, rows16(P.src[t.idx], P.cam[t.idx]));
      } else {
        const BandDev B = P.band[t.idx];
        const bool rows_out = ty0 < B.y0 || ty1 >= B.y1;
        need = warp == 0 ? (px0 < B.x0 || (rows_out && px1 >= B.x0)) : (px1 >= B.x1 || (rows_out && px0 < B.x1));
        if (need)
          W = warp_window<S, G::kRows>(P.cam[t.idx + warp], px0, ty0, px1, ty1,
                                       rows16(P.src[t.idx + warp], P.cam[t.idx + warp]));
      }
    }
    if (lane == 0) {
      h.sW[warp] = W;
      if (need && W.over && P.win_fallback) atomicAdd(P.win_fallback, 1u);
    }
  }
  __syncthreads();
  const Window W0 = h.sW[0], W1 = h.sW[1];
  if (W0.ok) stage_window<S>(P.src[t.idx], P.cam[t.idx], W0, st.win[0]);
  if (W1.ok) stage_window<S>(P.src[t.idx + 1], P.cam[t.idx + 1], W1, st.win[1]);
  __syncthreads();

  if (t.kind == kTileOwnPart) {
    ownpart_pairs<TW, TH>(P, bc, t.idx, W0, st.win[0], h.lut, st.out, tx0, ty0, cx0, cx1,
                          P.out_hist ? h.ohist : nullptr);
  } else {
    const int p = t.idx;
    const BandDev B = P.band[p];
    const bool printed = (P.flags & STITCH_FLOW_WEIGHTS_PRINTED) != 0;
    // The block's threads take the piece's own pixels (a band-edge chunk is
    // 16 columns wide): pixel i of the piece is column cx0 + i % pw of row
    // i / pw; the row comes from an approximate reciprocal of pw / 16
    // (floor((i / 16 + 1/2) / n) = floor(i / (16 n)), far from rounding).
    const int n16 = t.c1 - t.c0, pw = 16 * n16;
    const float inv_n = rcp_approx((float)n16);
#pragma unroll 1
    for (int i = threadIdx.x; i < pw * TH; i += kFuseThreads) {
      const int ly = (int)(((float)(i >> 4) + 0.5f) * inv_n);
      const int lx = cx0 + (i - ly * pw);
      const int x = tx0 + lx, y = ty0 + ly;
      float3 v = make_float3(0.0f, 0.0f, 0.0f);
      bool cov = false;
      if (x < P.pano_w && y < P.pano_h) {
        if (x < B.x0) {
          cov = own_value<S>(P, bc, p, p - 1, p + 1, W0, st.win[0], x, y, v);
        } else if (x >= B.x1) {
          cov = own_value<S>(P, bc, p + 1, p, p + 2, W1, st.win[1], x, y, v);
        } else if (y < B.y0 || y >= B.y1) {
          const float tb = __fmul_rn((float)(x - B.x0) + 0.5f, B.inv_bw);
          const float ta = 1.0f - tb;
          float3 va, vb;
          const bool ca = cam_value<S>(P, bc, p, W0, st.win[0], x, y, va);
          const bool cb = cam_value<S>(P, bc, p + 1, W1, st.win[1], x, y, vb);
          if (ca && cb) {
            v = make_float3(fmaf(ta, va.x, tb * vb.x), fmaf(ta, va.y, tb * vb.y), fmaf(ta, va.z, tb * vb.z));
          } else if (ca) {
            v = va;
          } else if (cb) {
            v = vb;
          }
          cov = ca || cb;
        } else {
          v = band_pixel<kHalf, true>(P, bc, p, x, y, printed);
          cov = true;
        }
      }
      put_px<TW, TH>(st.out, h.lut, lx, ly, cov, v, P.out_hist ? h.ohist : nullptr);
    }
  }
  __syncthreads();
  store_tile<TW, TH>(P, tx0, ty0, st.out, t.c0, t.c1);
}

// One band pre-warp piece (kTileW x kTileH) of pair pt.pair, both cameras,
// s clamped into the frame (the band lies inside both cameras' coverage, so
// the clamp only removes float32 noise). Under kFlagPwOffset (the frame path)
// the samples are the paired half2 bilinear of the staged windows and the
// intermediate holds v - 128; otherwise (the flow and the correspondence fit,
// which want the plain pre-warped image) a float32 bilinear of v.
template <bool kHalf>
__device__ __forceinline__ void prewarp_piece(const FuseParams &P, const PwTile pt, SmemPw &sp) {
  Window *sW = sp.sW;
  uint32_t (*win)[WinGeom<kTileW, kTileH>::kAlloc] = sp.win;
  using G = WinGeom<kTileW, kTileH>;
  using PM = PairMap<kTileW, kTileH>;
  constexpr int S = G::kStride;
  constexpr int kMax = G::kAlloc - S - 2;
  const BandDev B = P.band[pt.pair];
  const int bw = B.x1 - B.x0;
  const int rx0 = pt.x0, ry0 = pt.y0;
  const int rx1 = min(rx0 + kTileW, B.x1) - 1, ry1 = min(ry0 + kTileH, B.y1) - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < 2) {
    const Window W = warp_window<S, G::kRows>(P.cam[pt.pair + warp], rx0, ry0, rx1, ry1,
                                               rows16(P.src[pt.pair + warp], P.cam[pt.pair + warp]));
    if (lane == 0) {
      sW[warp] = W;
      if (W.over && P.win_fallback) atomicAdd(P.win_fallback, 1u);
    }
  }
  __syncthreads();
  const bool offset = (P.flags & kFlagPwOffset) != 0;
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    const Window W = sW[side];
    const int k = pt.pair + side;
    const CamDev &c = P.cam[k];
    if (W.ok) stage_window<S>(P.src[k], c, W, win[side]);
    __syncthreads();
    // the frame path (offset form) and STITCH_FP16_INTERMEDIATE store halves,
    // the flow and the correspondence fit float32 values
    const bool hstore = kHalf || offset;
    const bool luma = !offset && (P.flags & kFlagPwLuma) != 0;
    uint2 *dst2 = reinterpret_cast<uint2 *>(P.pw) + P.pw_off[pt.pair][side];
    float4 *dst4 = reinterpret_cast<float4 *>(P.pw) + P.pw_off[pt.pair][side];
    uint8_t *dsty = reinterpret_cast<uint8_t *>(P.pw) + P.pw_off[pt.pair][side];
    if (offset && W.ok) {
      // Every clamped point of the piece lies in the window (clipped to the
      // frame); a far tap past the frame reads the staged 0x64 column / row
      // with weight zero.
      const uint32_t off = kMagicRoundBits * (uint32_t)(S + 1) + (uint32_t)W.y0 * (uint32_t)S + (uint32_t)W.x0;
      const float hx = c.wm1 - 0.5f, hy = c.hm1 - 0.5f;
      const PairCoords pc = pair_coords<kTileW, kTileH>(c, rx0, ry0, lane, warp);
      float2 yy = pc.y0;
#pragma unroll 2
      for (int s = 0; s < PM::kSteps; ++s) {
        float2 ux, uy;
        pair_point(c, pc, 0, pair_row(c, yy), ux, uy);
        ux = f2(fminf(fmaxf(ux.x, -0.5f), hx), fminf(fmaxf(ux.y, -0.5f), hx));
        uy = f2(fminf(fmaxf(uy.x, -0.5f), hy), fminf(fmaxf(uy.y, -0.5f), hy));
        float2 rx, ry;
        __half2 fx, fy;
        split_pair(ux, rx, fx);
        split_pair(uy, ry, fy);
        const uint32_t i0 = __float_as_uint(ry.x) * (uint32_t)S + __float_as_uint(rx.x) - off;
        const uint32_t i1 = __float_as_uint(ry.y) * (uint32_t)S + __float_as_uint(rx.y) - off;
        uint32_t t0[4], t1[4];
        taps<S, kMax>(win[side], i0, t0);
        taps<S, kMax>(win[side], i1, t1);
        float2 v[3];
        bilerp_pair(t0, t1, fx, fy, v);
        const int y = ry0 + PM::ly0(warp, s);
        const int x0 = rx0 + PM::lx0(lane, 0), x1 = rx0 + PM::lx1(lane, 0);
        if (y <= ry1) {
          const size_t o = (size_t)(y - B.y0) * bw;
          if (x0 <= rx1)
            dst2[o + (x0 - B.x0)] = make_uint2(h2_bits(__floats2half2_rn(v[0].x, v[1].x)),
                                               h2_bits(__floats2half2_rn(v[2].x, 0.0f)));
          if (x1 <= rx1)
            dst2[o + (x1 - B.x0)] = make_uint2(h2_bits(__floats2half2_rn(v[0].y, v[1].y)),
                                               h2_bits(__floats2half2_rn(v[2].y, 0.0f)));
        }
        yy = __fadd2_rn(yy, f2(PM::kDy));
      }
    } else {
      for (int j = 0; j < 8; ++j) {
        const int x = rx0 + lane + 32 * (j & 1);
        const int y = ry0 + 4 * warp + (j >> 1);
        if (x > rx1 || y > ry1) continue;
        const size_t o = (size_t)(y - B.y0) * bw + (x - B.x0);
        float3 v;
        if (offset) {
          // window did not fit: the same arithmetic with taps from the frame
          float sx, sy, nw;
          cam_point(c, x, y, sx, sy, nw);
          sx = fminf(fmaxf(sx, -0.5f), c.wm1 - 0.5f);
          sy = fminf(fmaxf(sy, -0.5f), c.hm1 - 0.5f);
          const float rxs = sx + kMagicRound, rys = sy + kMagicRound;
          const float fx = (sx - (rxs - kMagicRound)) + 0.5f, fy = (sy - (rys - kMagicRound)) + 0.5f;
          const int ix = max((int)(__float_as_uint(rxs) - kMagicRoundBits), 0);
          const int iy = max((int)(__float_as_uint(rys) - kMagicRoundBits), 0);
          const int ix1 = min(ix + 1, c.w - 1), iy1 = min(iy + 1, c.h_px - 1);
          uint32_t t[4] = {gword(P.src[k], c, ix, iy), gword(P.src[k], c, ix1, iy), gword(P.src[k], c, ix, iy1),
                           gword(P.src[k], c, ix1, iy1)};
          float2 vv[3];
          bilerp_pair(t, t, __float2half2_rn(fx), __float2half2_rn(fy), vv);
          v = make_float3(vv[0].x, vv[1].x, vv[2].x);
        } else {
          float sx, sy, nw;
          cam_map_f(c, (float)(x - c.ox), (float)(y - c.oy), sx, sy, nw);
          sx = fminf(fmaxf(sx, 0.0f), c.wm1);
          sy = fminf(fmaxf(sy, 0.0f), c.hm1);
          if (luma) {
            // the flow's luminance: round-half-even(clamp((R + 2G + B) / 4, 0, 255))
            const float L = W.ok ? win_luma<S>(win[side], W, sx, sy) : src_luma(P.src[k], c, sx, sy);
            const uint8_t yv = (uint8_t)__float2int_rn(fminf(fmaxf(L * 0.25f, 0.0f), 255.0f));
            dsty[o] = yv;
            sp.lum[y - ry0][x - rx0] = yv;
            continue;
          }
          v = W.ok ? win_bilinear<S>(win[side], W, sx, sy) : src_bilinear(P.src[k], c, sx, sy);
        }
        if (hstore) {
          dst2[o] = make_uint2(h2_bits(__floats2half2_rn(v.x, v.y)), h2_bits(__floats2half2_rn(v.z, 0.0f)));
        } else {
          dst4[o] = make_float4(v.x, v.y, v.z, 0.0f);
        }
      }
    }
    if (luma) {
      // Levels 1 and 2 of the flow's pyramid over this piece: (a + b + c +
      // d + 2) >> 2 over 2 x 2 blocks, the last row / column repeated for odd
      // sizes. Pieces start at multiples of 64 x 32 band pixels, so every
      // block of both levels lies inside one piece, and the piece's clipped
      // extent is where the band's odd last row / column repeats.
      __syncthreads();
      const int bx = rx0 - B.x0, by = ry0 - B.y0;          // band-relative origin (even, a multiple of 4)
      const int nx0 = rx1 - rx0 + 1, ny0 = ry1 - ry0 + 1;
      const int nx1 = (nx0 + 1) >> 1, ny1 = (ny0 + 1) >> 1;
      uint8_t *d1 = reinterpret_cast<uint8_t *>(P.pw) + P.lum_off[0][pt.pair][side];
      const int w1 = P.lum_w[0][pt.pair];
      for (int i = threadIdx.x; i < nx1 * ny1; i += blockDim.x) {
        const int yy = i / nx1, xx = i - yy * nx1;
        const int xa = 2 * xx, ya = 2 * yy, xb = min(xa + 1, nx0 - 1), yb = min(ya + 1, ny0 - 1);
        const int v = (sp.lum[ya][xa] + sp.lum[yb][xa] + sp.lum[ya][xb] + sp.lum[yb][xb] + 2) >> 2;
        sp.lum1[yy][xx] = (uint8_t)v;
        d1[(size_t)((by >> 1) + yy) * w1 + (bx >> 1) + xx] = (uint8_t)v;
      }
      __syncthreads();
      const int nx2 = (nx1 + 1) >> 1, ny2 = (ny1 + 1) >> 1;
      uint8_t *d2 = reinterpret_cast<uint8_t *>(P.pw) + P.lum_off[1][pt.pair][side];
      const int w2 = P.lum_w[1][pt.pair];
      for (int i = threadIdx.x; i < nx2 * ny2; i += blockDim.x) {
        const int yy = i / nx2, xx = i - yy * nx2;
        const int xa = 2 * xx, ya = 2 * yy, xb = min(xa + 1, nx1 - 1), yb = min(ya + 1, ny1 - 1);
        const int v = (sp.lum1[ya][xa] + sp.lum1[yb][xa] + sp.lum1[ya][xb] + sp.lum1[yb][xb] + 2) >> 2;
        d2[(size_t)((by >> 2) + yy) * w2 + (bx >> 2) + xx] = (uint8_t)v;
      }
      __syncthreads();   // the next side rewrites the tiles
    }
  }
}

// Copy one rig's parameters into shared memory (16-byte words).
__device__ __forceinline__ void copy_params(FuseParams &dst, const FuseParams *src) {
  static_assert(sizeof(FuseParams) % 16 == 0, "parameter block must be a whole number of 16-byte words");
  const int4 *s = reinterpret_cast<const int4 *>(src);
  int4 *d = reinterpret_cast<int4 *>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(FuseParams) / 16); i += blockDim.x) d[i] = __ldg(s + i);
}

// STITCH_BALANCE_OUTPUT: the block's histogram starts at zero and is added
// to the frame's histogram once, when the persistent block is done.
__device__ __forceinline__ void ohist_zero(const FuseParams &P, SmemHead &h) {
  if (P.out_hist)
    for (int i = threadIdx.x; i < 3 * 256; i += blockDim.x) h.ohist[i] = 0u;
}
__device__ __forceinline__ void ohist_flush(const FuseParams &P, SmemHead &h) {
  if (!P.out_hist) return;
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * 256; i += blockDim.x) {
    const uint32_t c = h.ohist[i];
    if (c) atomicAdd(P.out_hist + i, c);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Kernels.
// ---------------------------------------------------------------------------

template <bool kHalf>
__global__ void __launch_bounds__(kFuseThreads) k_prewarp_band(const FuseParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemPw &sp = *reinterpret_cast<SmemPw *>(smem);
  prewarp_piece<kHalf>(P, P.pw_tiles[blockIdx.x], sp);
}

// General pieces (the first n_tiles - n_band - n_full of the list),
// persistent: block b takes pieces b, b + grid, ...
template <bool kHalf, int TW, int TH>
__global__ void __launch_bounds__(kFuseThreads, 3) k_fuse(const FuseParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemHead &h = *reinterpret_cast<SmemHead *>(smem);
  load_color(P, h);
  ohist_zero(P, h);
  const int n = P.n_tiles - P.n_band - P.n_full;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    __syncthreads();
    fuse_tile<kHalf, TW, TH>(P, P.tiles[i], h, tile_smem<TW, TH, 2>(smem));
  }
  ohist_flush(P, h);
}

// Band pieces (the n_band before the fully covered ones), persistent.
template <bool kHalf, int TW, int TH>
__global__ void __launch_bounds__(kFuseThreads, 4) k_fuse_band(const FuseParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemHead &h = *reinterpret_cast<SmemHead *>(smem);
  SmemBand<TW, TH> &sb = *reinterpret_cast<SmemBand<TW, TH> *>(smem + (sizeof(SmemHead) + 15) / 16 * 16);
  load_color(P, h);
  ohist_zero(P, h);
  const int base = P.n_tiles - P.n_full - P.n_band;
  for (int i = blockIdx.x; i < P.n_band; i += gridDim.x) {
    __syncthreads();
    fuse_band_piece<kHalf, TW, TH>(P, P.tiles[base + i], h, sb.out);
  }
  ohist_flush(P, h);
}

// The fully covered own pieces, which close the list (P.n_full of them).
template <int TW, int TH>
__global__ void __launch_bounds__(kFuseThreads, 4) k_fuse_own(const FuseParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemHead &h = *reinterpret_cast<SmemHead *>(smem);
  load_color(P, h);
  ohist_zero(P, h);
  const int base = P.n_tiles - P.n_full;
  for (int i = blockIdx.x; i < P.n_full; i += gridDim.x) {
    __syncthreads();
    fuse_own_tile<TW, TH>(P, P.tiles[base + i], h, tile_smem<TW, TH, 1>(smem));
  }
  ohist_flush(P, h);
}

// Band pre-warp of several rigs in one launch (the frame path: launched
// without the flow's luminance tiles): block b takes item b.
template <bool kHalf>
__global__ void __launch_bounds__(kFuseThreads) k_prewarp_multi(const MultiParams M) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemPwMulti &sm = *reinterpret_cast<SmemPwMulti *>(smem);
  const MultiItem it = M.items[blockIdx.x];
  copy_params(sm.sp, M.params + M.base + it.rig);
  __syncthreads();
  prewarp_piece<kHalf>(sm.sp, it.pw, sm.pw);
}

// Next item of a persistent multi-rig launch; reloads the rig's parameters
// and colour constants when the rig changes. Returns false when none is left.
__device__ __forceinline__ bool next_item(const MultiParams &M, SmemHead &h, MultiItem &it) {
  __syncthreads();
  if (threadIdx.x == 0) h.item = atomicAdd(M.counter, 1);
  __syncthreads();
  const int item = h.item;
  if (item >= M.n_items) return false;
  it = M.items[item];
  if (it.rig != h.rig) {
    copy_params(h.sp, M.params + M.base + it.rig);
    __syncthreads();
    load_color(h.sp, h);
    __syncthreads();
    if (threadIdx.x == 0) h.rig = it.rig;
    __syncthreads();
  }
  return true;
}

// One tile of a multi-rig launch in its own call frame, so that each shape's
// code gets its own register allocation inside the mixed-shape kernels.
template <bool kHalf, int TW, int TH>
__device__ __forceinline__ void any_tile(SmemHead &h, const TileDesc t, unsigned char *smem) {
  if (t.kind == kTileBand)
    fuse_band_piece<kHalf, TW, TH>(h.sp, t, h, tile_smem<TW, TH, 2>(smem).out);
  else
    fuse_tile<kHalf, TW, TH>(h.sp, t, h, tile_smem<TW, TH, 2>(smem));
}
template <bool kHalf, int TW, int TH>
__device__ __noinline__ void multi_tile(SmemHead &h, const TileDesc t, unsigned char *smem) {
  any_tile<kHalf, TW, TH>(h, t, smem);
}
template <int TW, int TH>
__device__ __noinline__ void multi_own_tile(SmemHead &h, const TileDesc t, unsigned char *smem) {
  fuse_own_tile<TW, TH>(h.sp, t, h, tile_smem<TW, TH, 1>(smem));
}

// Persistent fuse over the tiles of several rigs: each block takes the next
// item from a work counter until none is left (dynamic balance of uneven tile
// costs). k_fuse_multi serves batches whose rigs share one tile shape;
// k_fuse_multi_mixed runs every item with its rig's own shape.
template <bool kHalf, int TW, int TH>
__global__ void __launch_bounds__(kFuseThreads, 3) k_fuse_multi(const MultiParams M) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemHead &h = *reinterpret_cast<SmemHead *>(smem);
  if (threadIdx.x == 0) h.rig = -1;
  MultiItem it;
  while (next_item(M, h, it)) any_tile<kHalf, TW, TH>(h, it.tile, smem);
}

template <bool kHalf>
__global__ void __launch_bounds__(kFuseThreads, 3) k_fuse_multi_mixed(const MultiParams M) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemHead &h = *reinterpret_cast<SmemHead *>(smem);
  if (threadIdx.x == 0) h.rig = -1;
  MultiItem it;
  while (next_item(M, h, it)) {
    switch (it.shape) {
      case 0: multi_tile<kHalf, 64, 32>(h, it.tile, smem); break;
      case 1: multi_tile<kHalf, 64, 16>(h, it.tile, smem); break;
      case 2: multi_tile<kHalf, 32, 32>(h, it.tile, smem); break;
      case 3: multi_tile<kHalf, 128, 16>(h, it.tile, smem); break;
      case 4: multi_tile<kHalf, 32, 16>(h, it.tile, smem); break;
      default: multi_tile<kHalf, 128, 32>(h, it.tile, smem); break;
    }
  }
}

// Persistent fuse over the band pieces of several rigs that share one tile
// shape (the single-rig band kernel's register budget and shared memory).
template <bool kHalf, int TW, int TH>
__global__ void __launch_bounds__(kFuseThreads, 4) k_fuse_band_multi(const MultiParams M) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemHead &h = *reinterpret_cast<SmemHead *>(smem);
  SmemBand<TW, TH> &sb = *reinterpret_cast<SmemBand<TW, TH> *>(smem + (sizeof(SmemHead) + 15) / 16 * 16);
  if (threadIdx.x == 0) h.rig = -1;
  MultiItem it;
  while (next_item(M, h, it)) fuse_band_piece<kHalf, TW, TH>(h.sp, it.tile, h, sb.out);
}

// Persistent fuse over the fully covered own tiles of several rigs (one shape
// for all rigs, or each rig's own).
template <int TW, int TH>
__global__ void __launch_bounds__(kFuseThreads, 4) k_fuse_own_multi(const MultiParams M) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemHead &h = *reinterpret_cast<SmemHead *>(smem);
  if (threadIdx.x == 0) h.rig = -1;
  MultiItem it;
  while (next_item(M, h, it)) fuse_own_tile<TW, TH>(h.sp, it.tile, h, tile_smem<TW, TH, 1>(smem));
}

__global__ void __launch_bounds__(kFuseThreads, 4) k_fuse_own_multi_mixed(const MultiParams M) {
  extern __shared__ __align__(16) unsigned char smem[];
  SmemHead &h = *reinterpret_cast<SmemHead *>(smem);
  if (threadIdx.x == 0) h.rig = -1;
  MultiItem it;
  while (next_item(M, h, it)) {
    switch (it.shape) {
      case 0: multi_own_tile<64, 32>(h, it.tile, smem); break;
      case 1: multi_own_tile<64, 16>(h, it.tile, smem); break;
      case 2: multi_own_tile<32, 32>(h, it.tile, smem); break;
      case 3: multi_own_tile<128, 16>(h, it.tile, smem); break;
      case 4: multi_own_tile<32, 16>(h, it.tile, smem); break;
      default: multi_own_tile<128, 32>(h, it.tile, smem); break;
    }
  }
}

// ---------------------------------------------------------------------------
// Host side: shared-memory sizes, attributes, launches.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kPwSmem = sizeof(SmemPw);                      // single-rig band pre-warp (the flow's, with
                                                                 // its luminance tiles)
constexpr size_t kPwSmemFrame = (offsetof(SmemPw, lum) + 15) / 16 * 16;   // without them: only kFlagPwLuma uses them
constexpr size_t kPwMultiSmem = offsetof(SmemPwMulti, pw) + kPwSmemFrame;   // multi-rig (frame path): the rig's
                                                                              // parameters too
constexpr size_t kMixSmem =
    cmax(cmax(cmax(smem_bytes<64, 32, 2>(), smem_bytes<64, 16, 2>()), cmax(smem_bytes<32, 32, 2>(), smem_bytes<128, 16, 2>())),
         cmax(smem_bytes<32, 16, 2>(), smem_bytes<128, 32, 2>()));
constexpr size_t kMixOwnSmem =
    cmax(cmax(cmax(smem_bytes<64, 32, 1>(), smem_bytes<64, 16, 1>()), cmax(smem_bytes<32, 32, 1>(), smem_bytes<128, 16, 1>())),
         cmax(smem_bytes<32, 16, 1>(), smem_bytes<128, 32, 1>()));

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int TW, int TH>
cudaError_t setup_shape() {
  cudaError_t e = set_smem(k_fuse<false, TW, TH>, smem_bytes<TW, TH, 2>());
  if (e == cudaSuccess) e = set_smem(k_fuse<true, TW, TH>, smem_bytes<TW, TH, 2>());
  if (e == cudaSuccess) e = set_smem(k_fuse_band<false, TW, TH>, band_smem_bytes<TW, TH>());
  if (e == cudaSuccess) e = set_smem(k_fuse_band<true, TW, TH>, band_smem_bytes<TW, TH>());
  if (e == cudaSuccess) e = set_smem(k_fuse_own<TW, TH>, smem_bytes<TW, TH, 1>());
  if (e == cudaSuccess) e = set_smem(k_fuse_multi<false, TW, TH>, smem_bytes<TW, TH, 2>());
  if (e == cudaSuccess) e = set_smem(k_fuse_multi<true, TW, TH>, smem_bytes<TW, TH, 2>());
  if (e == cudaSuccess) e = set_smem(k_fuse_own_multi<TW, TH>, smem_bytes<TW, TH, 1>());
  if (e == cudaSuccess) e = set_smem(k_fuse_band_multi<false, TW, TH>, band_smem_bytes<TW, TH>());
  if (e == cudaSuccess) e = set_smem(k_fuse_band_multi<true, TW, TH>, band_smem_bytes<TW, TH>());
  return e;
}

// Resident blocks per SM of a persistent kernel, cached per kernel.
template <typename K>
int per_sm(K kernel, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kFuseThreads, smem) != cudaSuccess) n = 1;
  return n < 1 ? 1 : n;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
  }
  return n;
}

// Persistent grid for n tiles: one full wave of resident blocks (every SM
// holds as many blocks as fit, which hides the kernels' load latency).
int persistent_grid(int n, int resident) {
  if (n <= 0) return 0;
  return std::min(n, resident * sm_count());
}

// The three fuse launches of a frame (general pieces, band pieces, fully
// covered own pieces), each a persistent grid of at most one resident wave.
template <int TW, int TH>
void fuse_by_half(const FuseParams &p, cudaStream_t s) {
  static int res_gen[2] = {0, 0}, res_band[2] = {0, 0}, res_own = 0;
  const int gen = p.n_tiles - p.n_band - p.n_full;
  const bool half = (p.flags & STITCH_FP16_INTERMEDIATE) != 0;
  constexpr size_t kGen = smem_bytes<TW, TH, 2>(), kBand = band_smem_bytes<TW, TH>(), kOwn = smem_bytes<TW, TH, 1>();
  if (gen > 0) {
    if (half) {
      if (!res_gen[1]) res_gen[1] = per_sm(k_fuse<true, TW, TH>, kGen);
      k_fuse<true, TW, TH><<<persistent_grid(gen, res_gen[1]), kFuseThreads, kGen, s>>>(p);
    } else {
      if (!res_gen[0]) res_gen[0] = per_sm(k_fuse<false, TW, TH>, kGen);
      k_fuse<false, TW, TH><<<persistent_grid(gen, res_gen[0]), kFuseThreads, kGen, s>>>(p);
    }
  }
  if (p.n_band > 0) {
    if (half) {
      if (!res_band[1]) res_band[1] = per_sm(k_fuse_band<true, TW, TH>, kBand);
      k_fuse_band<true, TW, TH><<<persistent_grid(p.n_band, res_band[1]), kFuseThreads, kBand, s>>>(p);
    } else {
      if (!res_band[0]) res_band[0] = per_sm(k_fuse_band<false, TW, TH>, kBand);
      k_fuse_band<false, TW, TH><<<persistent_grid(p.n_band, res_band[0]), kFuseThreads, kBand, s>>>(p);
    }
  }
  if (p.n_full > 0) {
    if (!res_own) res_own = per_sm(k_fuse_own<TW, TH>, kOwn);
    k_fuse_own<TW, TH><<<persistent_grid(p.n_full, res_own), kFuseThreads, kOwn, s>>>(p);
  }
}

template <int TW, int TH>
void band_multi_by_half(const MultiParams &m, bool half, int grid, cudaStream_t s) {
  if (half)
    k_fuse_band_multi<true, TW, TH><<<grid, kFuseThreads, band_smem_bytes<TW, TH>(), s>>>(m);
  else
    k_fuse_band_multi<false, TW, TH><<<grid, kFuseThreads, band_smem_bytes<TW, TH>(), s>>>(m);
}

template <int TW, int TH>
int band_multi_per_sm(bool half) {
  return half ? per_sm(k_fuse_band_multi<true, TW, TH>, band_smem_bytes<TW, TH>())
              : per_sm(k_fuse_band_multi<false, TW, TH>, band_smem_bytes<TW, TH>());
}

template <int TW, int TH>
void fuse_multi_by_half(const MultiParams &m, bool half, int grid, cudaStream_t s) {
  if (half)
    k_fuse_multi<true, TW, TH><<<grid, kFuseThreads, smem_bytes<TW, TH, 2>(), s>>>(m);
  else
    k_fuse_multi<false, TW, TH><<<grid, kFuseThreads, smem_bytes<TW, TH, 2>(), s>>>(m);
}

}  // namespace

static_assert(kNumTileShapes == 6 && kTileShapes[0].w == 64 && kTileShapes[0].h == 32 && kTileShapes[1].w == 64 &&
                  kTileShapes[1].h == 16 && kTileShapes[2].w == 32 && kTileShapes[2].h == 32 &&
                  kTileShapes[3].w == 128 && kTileShapes[3].h == 16 && kTileShapes[4].w == 32 &&
                  kTileShapes[4].h == 16 && kTileShapes[5].w == 128 && kTileShapes[5].h == 32,
              "the shape table and the kernel instantiations below must agree");

size_t prewarp_elem_bytes(bool fp16) { return fp16 ? sizeof(uint2) : sizeof(float4); }

// Once per device, outside any stream capture: every fuse kernel uses more
// than the default 48 KB of dynamic shared memory.
cudaError_t fuse_setup_attributes(int) {
  cudaError_t e = set_smem(k_prewarp_band<false>, kPwSmem);
  if (e == cudaSuccess) e = set_smem(k_prewarp_band<true>, kPwSmem);
  if (e == cudaSuccess) e = set_smem(k_prewarp_multi<false>, kPwMultiSmem);
  if (e == cudaSuccess) e = set_smem(k_prewarp_multi<true>, kPwMultiSmem);
  if (e == cudaSuccess) e = setup_shape<64, 32>();
  if (e == cudaSuccess) e = setup_shape<64, 16>();
  if (e == cudaSuccess) e = setup_shape<32, 32>();
  if (e == cudaSuccess) e = setup_shape<128, 16>();
  if (e == cudaSuccess) e = setup_shape<32, 16>();
  if (e == cudaSuccess) e = setup_shape<128, 32>();
  if (e == cudaSuccess) e = set_smem(k_fuse_multi_mixed<false>, kMixSmem);
  if (e == cudaSuccess) e = set_smem(k_fuse_multi_mixed<true>, kMixSmem);
  if (e == cudaSuccess) e = set_smem(k_fuse_own_multi_mixed, kMixOwnSmem);
  return e;
}

cudaError_t launch_prewarp(const FuseParams &p, cudaStream_t s) {
  if (p.n_pw_tiles <= 0) return cudaSuccess;
  const size_t smem = (p.flags & kFlagPwLuma) ? kPwSmem : kPwSmemFrame;
  if (p.flags & STITCH_FP16_INTERMEDIATE)
    k_prewarp_band<true><<<p.n_pw_tiles, kFuseThreads, smem, s>>>(p);
  else
    k_prewarp_band<false><<<p.n_pw_tiles, kFuseThreads, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_fuse(const FuseParams &p, int shape, cudaStream_t s) {
  if (p.n_tiles <= 0) return cudaSuccess;
  switch (shape) {
    case 0: fuse_by_half<64, 32>(p, s); break;
    case 1: fuse_by_half<64, 16>(p, s); break;
    case 2: fuse_by_half<32, 32>(p, s); break;
    case 3: fuse_by_half<128, 16>(p, s); break;
    case 4: fuse_by_half<32, 16>(p, s); break;
    case 5: fuse_by_half<128, 32>(p, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_prewarp_multi(const MultiParams &m, bool half, cudaStream_t s) {
  if (m.n_items <= 0) return cudaSuccess;
  if (half)
    k_prewarp_multi<true><<<m.n_items, kFuseThreads, kPwMultiSmem, s>>>(m);
  else
    k_prewarp_multi<false><<<m.n_items, kFuseThreads, kPwMultiSmem, s>>>(m);
  return cudaGetLastError();
}

size_t fuse_mixed_smem(const int *shapes, int n, int windows) {
  size_t most = 0;
  for (int i = 0; i < n; ++i) {
    size_t b = windows == 2 ? kMixSmem : kMixOwnSmem;
    switch (shapes[i]) {
      case 0: b = windows == 2 ? smem_bytes<64, 32, 2>() : smem_bytes<64, 32, 1>(); break;
      case 1: b = windows == 2 ? smem_bytes<64, 16, 2>() : smem_bytes<64, 16, 1>(); break;
      case 2: b = windows == 2 ? smem_bytes<32, 32, 2>() : smem_bytes<32, 32, 1>(); break;
      case 3: b = windows == 2 ? smem_bytes<128, 16, 2>() : smem_bytes<128, 16, 1>(); break;
      case 4: b = windows == 2 ? smem_bytes<32, 16, 2>() : smem_bytes<32, 16, 1>(); break;
      case 5: b = windows == 2 ? smem_bytes<128, 32, 2>() : smem_bytes<128, 32, 1>(); break;
      default: break;
    }
    most = std::max(most, b);
  }
  return most;
}

cudaError_t launch_fuse_multi(const MultiParams &m, bool half, int shape, int grid, cudaStream_t s,
                              size_t mixed_smem) {
  if (m.n_items <= 0) return cudaSuccess;
  const size_t mix = mixed_smem ? mixed_smem : kMixSmem;
  switch (shape) {
    case -1:
      if (half)
        k_fuse_multi_mixed<true><<<grid, kFuseThreads, mix, s>>>(m);
      else
        k_fuse_multi_mixed<false><<<grid, kFuseThreads, mix, s>>>(m);
      break;
    case 0: fuse_multi_by_half<64, 32>(m, half, grid, s); break;
    case 1: fuse_multi_by_half<64, 16>(m, half, grid, s); break;
    case 2: fuse_multi_by_half<32, 32>(m, half, grid, s); break;
    case 3: fuse_multi_by_half<128, 16>(m, half, grid, s); break;
    case 4: fuse_multi_by_half<32, 16>(m, half, grid, s); break;
    case 5: fuse_multi_by_half<128, 32>(m, half, grid, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fuse_own_multi(const MultiParams &m, int shape, int grid, cudaStream_t s, size_t mixed_smem) {
  if (m.n_items <= 0) return cudaSuccess;
  switch (shape) {
    case -1: k_fuse_own_multi_mixed<<<grid, kFuseThreads, mixed_smem ? mixed_smem : kMixOwnSmem, s>>>(m); break;
    case 0: k_fuse_own_multi<64, 32><<<grid, kFuseThreads, smem_bytes<64, 32, 1>(), s>>>(m); break;
    case 1: k_fuse_own_multi<64, 16><<<grid, kFuseThreads, smem_bytes<64, 16, 1>(), s>>>(m); break;
    case 2: k_fuse_own_multi<32, 32><<<grid, kFuseThreads, smem_bytes<32, 32, 1>(), s>>>(m); break;
    case 3: k_fuse_own_multi<128, 16><<<grid, kFuseThreads, smem_bytes<128, 16, 1>(), s>>>(m); break;
    case 4: k_fuse_own_multi<32, 16><<<grid, kFuseThreads, smem_bytes<32, 16, 1>(), s>>>(m); break;
    case 5: k_fuse_own_multi<128, 32><<<grid, kFuseThreads, smem_bytes<128, 32, 1>(), s>>>(m); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fuse_band_multi(const MultiParams &m, bool half, int shape, int grid, cudaStream_t s) {
  if (m.n_items <= 0) return cudaSuccess;
  switch (shape) {
    case 0: band_multi_by_half<64, 32>(m, half, grid, s); break;
    case 1: band_multi_by_half<64, 16>(m, half, grid, s); break;
    case 2: band_multi_by_half<32, 32>(m, half, grid, s); break;
    case 3: band_multi_by_half<128, 16>(m, half, grid, s); break;
    case 4: band_multi_by_half<32, 16>(m, half, grid, s); break;
    case 5: band_multi_by_half<128, 32>(m, half, grid, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int fuse_band_multi_blocks_per_sm(bool half, int shape) {
  switch (shape) {
    case 0: return band_multi_per_sm<64, 32>(half);
    case 1: return band_multi_per_sm<64, 16>(half);
    case 2: return band_multi_per_sm<32, 32>(half);
    case 3: return band_multi_per_sm<128, 16>(half);
    case 4: return band_multi_per_sm<32, 16>(half);
    case 5: return band_multi_per_sm<128, 32>(half);
    default: return 0;
  }
}

int fuse_own_multi_blocks_per_sm(int shape, size_t mixed_smem) {
  switch (shape) {
    case -1: return per_sm(k_fuse_own_multi_mixed, mixed_smem ? mixed_smem : kMixOwnSmem);
    case 0: return per_sm(k_fuse_own_multi<64, 32>, smem_bytes<64, 32, 1>());
    case 1: return per_sm(k_fuse_own_multi<64, 16>, smem_bytes<64, 16, 1>());
    case 2: return per_sm(k_fuse_own_multi<32, 32>, smem_bytes<32, 32, 1>());
    case 3: return per_sm(k_fuse_own_multi<128, 16>, smem_bytes<128, 16, 1>());
    case 4: return per_sm(k_fuse_own_multi<32, 16>, smem_bytes<32, 16, 1>());
    case 5: return per_sm(k_fuse_own_multi<128, 32>, smem_bytes<128, 32, 1>());
    default: return 0;
  }
}

int fuse_multi_blocks_per_sm(bool half, int shape, size_t mixed_smem) {
  const size_t mix = mixed_smem ? mixed_smem : kMixSmem;
  switch (shape) {
    case -1: return half ? per_sm(k_fuse_multi_mixed<true>, mix) : per_sm(k_fuse_multi_mixed<false>, mix);
    case 0:
      return half ? per_sm(k_fuse_multi<true, 64, 32>, smem_bytes<64, 32, 2>())
                  : per_sm(k_fuse_multi<false, 64, 32>, smem_bytes<64, 32, 2>());
    case 1:
      return half ? per_sm(k_fuse_multi<true, 64, 16>, smem_bytes<64, 16, 2>())
                  : per_sm(k_fuse_multi<false, 64, 16>, smem_bytes<64, 16, 2>());
    case 2:
      return half ? per_sm(k_fuse_multi<true, 32, 32>, smem_bytes<32, 32, 2>())
                  : per_sm(k_fuse_multi<false, 32, 32>, smem_bytes<32, 32, 2>());
    case 3:
      return half ? per_sm(k_fuse_multi<true, 128, 16>, smem_bytes<128, 16, 2>())
                  : per_sm(k_fuse_multi<false, 128, 16>, smem_bytes<128, 16, 2>());
    case 4:
      return half ? per_sm(k_fuse_multi<true, 32, 16>, smem_bytes<32, 16, 2>())
                  : per_sm(k_fuse_multi<false, 32, 16>, smem_bytes<32, 16, 2>());
    case 5:
      return half ? per_sm(k_fuse_multi<true, 128, 32>, smem_bytes<128, 32, 2>())
                  : per_sm(k_fuse_multi<false, 128, 32>, smem_bytes<128, 32, 2>());
    default: return 0;
  }
}

}  // namespace stitch
