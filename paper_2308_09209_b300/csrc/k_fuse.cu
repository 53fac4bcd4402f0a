// K3 -- pre-warp, local warping, colour transfer, blend and balance
// (paper section 3.1 pre-warp; section 3.2 Eq. 15-18; Eq. 4; Eq. 5).
//
// Two kernels per frame:
//
// k_prewarp_band: the pre-warped image of section 3.1 over each pair's blend
//   band, for BOTH cameras of the pair, computed once per band pixel and kept
//   in a small intermediate (float32 RGB, or float16 with
//   STITCH_FP16_INTERMEDIATE). It does not depend on the colour estimate.
//
// k_fuse: one block per panorama tile (64 x 32 by default; the shape is a
//   template parameter the autotuner picks per rig). The fully covered own
//   tiles (about three quarters of a rig's tiles) run in a second launch,
//   k_fuse_own, whose one-camera code needs fewer registers and no spills.
//   * Own tiles (columns of one camera k): the source window that the tile
//     maps to through H_k^-1 (planar) or through the cylinder's ray and H_k^-1
//     (cylindrical panorama) is staged in shared memory as one RGBX word per
//     pixel; every pixel then computes s = H_k^-1 q (float32, relative to the
//     camera's panorama origin), tests coverage 0 <= s <= (w-1, h-1), reads its
//     four bilinear taps from shared memory and forms v = P . M_k. Pixels that
//     camera k does not cover fall back to k-1, then k+1 (Eq. 15's one-image
//     cases), else 0.
//   * Band tiles: pixels of the band rectangle compute
//       theta_j = (x - x0 + 0.5) / (x1 - x0), theta_i = 1 - theta_j (Eq. 16 read
//       as a ramp), X_i = q + theta_j clamp(flow_ij), X_j = q + theta_i
//       clamp(flow_ji) (Eq. 17, continuous reading; the printed weights under
//       STITCH_FLOW_WEIGHTS_PRINTED), clamp X into the band and sample the
//       pre-warped intermediate bilinearly (Eq. 18):
//       out = theta_i P_i(X_i) M_i + theta_j P_j(X_j) M_j.
//     The tile's other pixels (own columns beside the band, band columns
//     outside the band rows) use the staged windows of both cameras as above,
//     blending both cameras without flow where both cover a band-column pixel.
//   * Each channel is clamped to [0, 255], passed through the piecewise balance
//     curve F (Eq. 5: gamma, linear, gamma) and rounded half to even; pixels
//     go to a shared-memory tile and leave as 16-byte stores per plane.
//
// Thread mapping: lane l of a warp handles columns l + 32 a of the warp's
// rows, so a warp touches 32 consecutive pixels of a row at a time and its
// shared-memory tap reads fall in distinct banks.
//
// k_prewarp_multi / k_fuse_multi / k_fuse_own_multi: the same work over the
// tiles of several independent rigs in one launch each; the fuse kernels are
// persistent (one block per resident slot, tiles taken from a work counter).
// When the rigs' tile shapes differ, the *_mixed forms run every tile with
// its rig's shape.
#include <cuda_fp16.h>

#include "stitch_internal.h"

namespace stitch {

namespace {

constexpr float kMagicRound = 12582912.0f;   // 1.5 * 2^23: x + kMagicRound rounds x to an integer (RNE)
constexpr int kMagicRoundBits = 0x4B400000;
constexpr float kMagicByte = 8388608.0f;     // 2^23: the float with bits 0x4B0000bb is 2^23 + bb
constexpr int kWinCap = 3840;                // staged source pixels per window (15 KB)

// Approximate reciprocal (CUDA's fast division intrinsic: a few ulp).
__device__ __forceinline__ float rcp_approx(float x) { return __fdividef(1.0f, x); }

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
  sx = nx * r;
  sy = ny * r;
}

// Affine camera (no perspective row): s = H^-1 q without a divide.
__device__ __forceinline__ void cam_map_aff(const CamDev &c, float dx, float dy, float &sx, float &sy) {
  sx = fmaf(c.h[0], dx, fmaf(c.h[1], dy, c.h[2]));
  sy = fmaf(c.h[3], dx, fmaf(c.h[4], dy, c.h[5]));
}

__device__ __forceinline__ bool covered(const CamDev &c, float sx, float sy, float nw) {
  return nw > 0.0f && sx >= 0.0f && sx <= c.wm1 && sy >= 0.0f && sy <= c.hm1;
}

// Integer part and fraction of s with fraction in [0, 1]; for integer s the
// pair (s - 1, 1) may come back instead of (s, 0): both give the same bilinear
// sample, and the right-hand tap then never passes the last row / column.
__device__ __forceinline__ void split(float s, int &i, float &f) {
  const float r = (s - 0.5f) + kMagicRound;
  i = __float_as_int(r) - kMagicRoundBits;
  f = s - (r - kMagicRound);
}

// Channel c (0..2) of an RGBX word as 2^23 + value (exact).
__device__ __forceinline__ float mbyte(uint32_t w, int c) {
  return __int_as_float(__byte_perm(w, 0x4B000000u, 0x7440u + c));
}

// Bilinear of four RGBX words with fractions (fx, fy): (1-fy)((1-fx) a + fx b) + fy((1-fx) d + fx e).
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

// Row-vector product v . M (Eq. 4).
__device__ __forceinline__ float3 mulM(const float *M, float3 v) {
  float3 o;
  o.x = fmaf(v.x, M[0], fmaf(v.y, M[3], v.z * M[6]));
  o.y = fmaf(v.x, M[1], fmaf(v.y, M[4], v.z * M[7]));
  o.z = fmaf(v.x, M[2], fmaf(v.y, M[5], v.z * M[8]));
  return o;
}

// ---------------------------------------------------------------------------
// Source windows in shared memory.
// ---------------------------------------------------------------------------

struct Window {
  int x0, y0, w, h, stride, ok;
};

// Source window of the panorama rectangle [rx0, rx1] x [ry0, ry1] (inclusive)
// in camera c: the bounding box of the mapped corners plus one pixel of margin
// and the right / bottom tap, clipped to the frame. Computed by one warp (lane
// & 3 picks a corner); every lane returns the same window. ok = 0 when a corner
// maps behind the camera, the box is empty or it exceeds the capacity.
__device__ Window warp_window(const CamDev &c, int rx0, int ry0, int rx1, int ry1) {
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
  W.w = x1 - W.x0 + 1;
  W.h = y1 - W.y0 + 1;
  W.stride = (W.w + 3) & ~3;
  W.ok = (front && W.w >= 2 && W.h >= 2 && W.stride * W.h <= kWinCap) ? 1 : 0;
  return W;
}

__device__ __forceinline__ Window no_window() {
  Window W;
  W.x0 = W.y0 = W.w = W.h = W.stride = W.ok = 0;
  return W;
}

// Stage the window as RGBX words: four pixels (12 bytes) per step, read as
// aligned 32-bit words and realigned with funnel shifts.
__device__ void stage_window(const uint8_t *__restrict__ src, const CamDev &c, const Window &W, uint32_t *s) {
  const int G = W.stride >> 2;
  const uintptr_t end = reinterpret_cast<uintptr_t>(src) + (uintptr_t)c.pitch * (uintptr_t)(c.h_px - 1) +
                        (uintptr_t)(3 * c.w);
  const int nt = blockDim.x;
  const bool rows = G <= nt;
  const int rpi = rows ? nt / G : 0;
  if (rows && (int)threadIdx.x >= rpi * G) return;
  int r = rows ? (int)threadIdx.x / G : 0;
  int g = rows ? (int)threadIdx.x - r * G : 0;
  int i = threadIdx.x;
  while (true) {
    if (!rows) {
      if (i >= G * W.h) break;
      r = i / G;
      g = i - r * G;
    } else if (r >= W.h) {
      break;
    }
    const int px = W.x0 + 4 * g;
    const uint8_t *b = src + (size_t)(W.y0 + r) * c.pitch + 3 * px;
    const uintptr_t B = reinterpret_cast<uintptr_t>(b);
    const uintptr_t A = B & ~(uintptr_t)3;
    uint32_t p0, p1, p2, p3;
    if (px + 4 <= c.w && A + 16 <= end) {
      const uint32_t *wp = reinterpret_cast<const uint32_t *>(A);
      const uint32_t w0 = __ldg(wp), w1 = __ldg(wp + 1), w2 = __ldg(wp + 2), w3 = __ldg(wp + 3);
      const uint32_t sh = (uint32_t)(B - A) * 8u;
      const uint32_t q0 = __funnelshift_r(w0, w1, sh);
      const uint32_t q1 = __funnelshift_r(w1, w2, sh);
      const uint32_t q2 = __funnelshift_r(w2, w3, sh);
      p0 = __byte_perm(q0, 0u, 0x4210u);
      p1 = __byte_perm(q0, q1, 0x4543u);
      p2 = __byte_perm(q1, q2, 0x4432u);
      p3 = __byte_perm(q2, 0u, 0x4321u);
    } else {
      uint32_t q[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (px + k < c.w)
          q[k] = (uint32_t)__ldg(b + 3 * k) | ((uint32_t)__ldg(b + 3 * k + 1) << 8) |
                 ((uint32_t)__ldg(b + 3 * k + 2) << 16);
      p0 = q[0]; p1 = q[1]; p2 = q[2]; p3 = q[3];
    }
    *reinterpret_cast<uint4 *>(s + r * W.stride + 4 * g) = make_uint4(p0, p1, p2, p3);
    if (rows) r += rpi; else i += nt;
  }
}

// Bilinear sample from a staged window (taps clamped into the window).
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
  const uint32_t *p = s + ly * W.stride + lx;
  return bilerp_words(p[0], p[1], p[W.stride], p[W.stride + 1], fx, fy);
}

// ---------------------------------------------------------------------------
// Colour and balance, prepared once per block.
// ---------------------------------------------------------------------------

struct Tail {       // gamma tails of Eq. 5 on u = v / 255
  float d1, k1, g1; // dark:   F = d1 (u k1)^g1
  float e2, k2, g2; // bright: F = 255 - e2 ((1 - u) k2)^g2
};

struct BlockColor {
  float M[kMaxCams][9];   // M / 255, so fused values land in [0, 1]
  float lo[3], hi[3];     // knots m1/255, m2/255 (outside [0, 1] when there is no tail)
  float mid[3], half[3];  // (lo + hi) / 2, (hi - lo) / 2: a tail is |u - mid| > half
  float A[3], B[3];       // linear part F = A + B u
  Tail tail[3];
};

__device__ void load_block_color(const FuseParams &P, BlockColor &bc) {
  const int t = threadIdx.x;
  if (t < kMaxCams * 9) bc.M[t / 9][t % 9] = P.color->M[t / 9][t % 9] * (1.0f / 255.0f);
  if (t >= 96 && t < 99) {
    const int c = t - 96;
    const Curve cv = P.color->curve[c];
    if ((P.flags & STITCH_BALANCE_OFF) || cv.ident != 0.0f) {
      bc.lo[c] = -1.0f;
      bc.hi[c] = 2.0f;
      bc.A[c] = 0.0f;
      bc.B[c] = 255.0f;
    } else {
      bc.lo[c] = cv.m1 * (1.0f / 255.0f);
      bc.hi[c] = cv.m2 * (1.0f / 255.0f);
      bc.A[c] = cv.d1 - cv.s * cv.m1;
      bc.B[c] = 255.0f * cv.s;
    }
    bc.mid[c] = 0.5f * (bc.lo[c] + bc.hi[c]);
    bc.half[c] = 0.5f * (bc.hi[c] - bc.lo[c]);
    Tail tl;
    tl.d1 = cv.d1;
    tl.k1 = 255.0f * cv.inv_m1;
    tl.g1 = cv.g1;
    tl.e2 = 255.0f - cv.d2;
    tl.k2 = 255.0f * cv.inv_bm;
    tl.g2 = cv.g2;
    bc.tail[c] = tl;
  }
}

// One channel: clamp (saturate), balance (Eq. 5), round half to even; the low
// byte of the result is the output byte. The curve's parameters are read from
// shared memory (keeping them in registers costs more in spills than the
// loads).
__device__ __forceinline__ uint32_t finish(const BlockColor &bc, int c, float v) {
  const float u = __saturatef(v);
  float F = fmaf(bc.B[c], u, bc.A[c]);
  if (fabsf(u - bc.mid[c]) > bc.half[c]) {
    // The side comes from the midpoint: mid -/+ half need not round to the
    // knots exactly, and a value next to a knot must take that knot's tail
    // (both pieces meet there).
    const Tail &t = bc.tail[c];
    F = (u < bc.mid[c]) ? t.d1 * __powf(u * t.k1, t.g1)
                       : 255.0f - t.e2 * __powf((1.0f - u) * t.k2, t.g2);
  }
  return (uint32_t)__float_as_int(F + kMagicRound);
}

// ---------------------------------------------------------------------------
// Per-pixel general paths (global memory).
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool cam_value_g(const FuseParams &P, const BlockColor &bc, int k, int x, int y,
                                            float3 &v) {
  const CamDev &c = P.cam[k];
  float sx, sy, nw;
  cam_map_f(c, (float)(x - c.ox), (float)(y - c.oy), sx, sy, nw);
  if (!covered(c, sx, sy, nw)) return false;
  v = mulM(bc.M[k], src_bilinear(P.src[k], c, sx, sy));
  return true;
}

// Camera k's value at q, from its staged window when there is one (M points
// at the block's shared copy of the camera's matrix).
__device__ __forceinline__ bool cam_value_w(const FuseParams &P, const float *M, int k, const Window &W,
                                            const uint32_t *s, int x, int y, float3 &v) {
  const CamDev &c = P.cam[k];
  float sx, sy, nw;
  cam_map_f(c, (float)(x - c.ox), (float)(y - c.oy), sx, sy, nw);
  if (!covered(c, sx, sy, nw)) return false;
  v = mulM(M, W.ok ? win_bilinear(s, W, sx, sy) : src_bilinear(P.src[k], c, sx, sy));
  return true;
}

template <bool kHalf>
struct PwT;
template <>
struct PwT<false> {
  using T = float4;
  __device__ static void put(float4 *p, size_t i, float3 v) { p[i] = make_float4(v.x, v.y, v.z, 0.0f); }
  __device__ static float3 get(const float4 *p, size_t i) {
    const float4 q = __ldg(p + i);
    return make_float3(q.x, q.y, q.z);
  }
};
template <>
struct PwT<true> {
  using T = uint2;   // four halves
  __device__ static void put(uint2 *p, size_t i, float3 v) {
    const __half2 a = __floats2half2_rn(v.x, v.y);
    const __half2 b = __floats2half2_rn(v.z, 0.0f);
    p[i] = make_uint2(*reinterpret_cast<const uint32_t *>(&a), *reinterpret_cast<const uint32_t *>(&b));
  }
  __device__ static float3 get(const uint2 *p, size_t i) {
    const uint2 q = __ldg(p + i);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&q.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&q.y));
    return make_float3(a.x, a.y, b.x);
  }
};

// Bilinear sample of a band's pre-warped intermediate at X (already inside the band).
template <bool kHalf>
__device__ __forceinline__ float3 pw_bilinear(const typename PwT<kHalf>::T *pw, const BandDev &B, float X, float Y) {
  int ix, iy;
  float gx, gy;
  split(X, ix, gx);
  split(Y, iy, gy);
  // X == x0 (odd) may come back as (x0 - 1, 1): take the tap at x0 instead.
  if (ix < B.x0) { ix = B.x0; gx = 0.0f; }
  if (iy < B.y0) { iy = B.y0; gy = 0.0f; }
  const int bw = B.x1 - B.x0, bh = B.y1 - B.y0;
  const int lx = min(ix - B.x0, bw - 1), ly = min(iy - B.y0, bh - 1);
  const int lx1 = min(lx + 1, bw - 1), ly1 = min(ly + 1, bh - 1);
  const float3 a = PwT<kHalf>::get(pw, (size_t)ly * bw + lx), b = PwT<kHalf>::get(pw, (size_t)ly * bw + lx1);
  const float3 d = PwT<kHalf>::get(pw, (size_t)ly1 * bw + lx), e = PwT<kHalf>::get(pw, (size_t)ly1 * bw + lx1);
  float3 t, u, o;
  t.x = fmaf(gx, b.x - a.x, a.x); t.y = fmaf(gx, b.y - a.y, a.y); t.z = fmaf(gx, b.z - a.z, a.z);
  u.x = fmaf(gx, e.x - d.x, d.x); u.y = fmaf(gx, e.y - d.y, d.y); u.z = fmaf(gx, e.z - d.z, d.z);
  o.x = fmaf(gy, u.x - t.x, t.x); o.y = fmaf(gy, u.y - t.y, t.y); o.z = fmaf(gy, u.z - t.z, t.z);
  return o;
}

template <int TW, int TH>
__device__ __forceinline__ void put_px(uint8_t (*s_out)[TH][TW], int lx, int ly, const BlockColor &bc, bool cov,
                                       float3 v) {
  uint32_t o0 = 0u, o1 = 0u, o2 = 0u;
  if (cov) {
    o0 = finish(bc, 0, v.x);
    o1 = finish(bc, 1, v.y);
    o2 = finish(bc, 2, v.z);
  }
  s_out[0][ly][lx] = (uint8_t)o0;
  s_out[1][ly][lx] = (uint8_t)o1;
  s_out[2][ly][lx] = (uint8_t)o2;
}

template <int TW, int TH>
__device__ __forceinline__ void store_tile(const FuseParams &P, int tx0, int ty0, const uint8_t (*s_out)[TH][TW]) {
  // 3 planes x TH rows x TW / 16 sixteen-byte pieces.
  constexpr int kPieces = TW / 16;
  for (int t = threadIdx.x; t < 3 * TH * kPieces; t += blockDim.x) {
    const int c = t / (TH * kPieces);
    const int r = (t / kPieces) % TH;
    const int q = t % kPieces;
    const int y = ty0 + r, x = tx0 + 16 * q;
    if (y >= P.pano_h || x >= P.pano_pitch) continue;
    const uint4 v = *reinterpret_cast<const uint4 *>(&s_out[c][r][16 * q]);
    *reinterpret_cast<uint4 *>(P.out + (size_t)c * P.pano_pitch * P.pano_h + (size_t)y * P.pano_pitch + x) = v;
  }
}

// Shared memory of one fuse tile.
template <int TW, int TH>
struct FuseSmem {
  BlockColor bc;
  Window sW[2];
  __align__(16) uint32_t s_win[2][kWinCap];
  __align__(16) uint8_t s_out[3][TH][TW];
};

// Thread -> pixel mapping of a TW x TH tile: warp w owns rows
// [w TH / 8, (w + 1) TH / 8), lane l the columns l + 32 a; pixel j of a thread
// is column group j % (TW / 32) of row j / (TW / 32) of its warp's rows.
template <int TW, int TH>
struct Map {
  static constexpr int kGroups = TW / 32;
  static constexpr int kRowsPerWarp = TH / 8;
  static constexpr int kPix = kGroups * kRowsPerWarp;
  static_assert(TW % 32 == 0 && TH % 8 == 0, "tile shape");
  __device__ static int lx(int lane, int j) { return lane + 32 * (j % kGroups); }
  __device__ static int ly(int warp, int j) { return kRowsPerWarp * warp + j / kGroups; }
};

// One panorama tile (see the file header): source windows, per-pixel work,
// then the tile's three planes leave as 16-byte stores.
template <bool kHalf, int TW, int TH>
__device__ __forceinline__ void fuse_tile(const FuseParams &P, const TileDesc t, FuseSmem<TW, TH> &sm) {
  using PT = typename PwT<kHalf>::T;
  using MP = Map<TW, TH>;
  BlockColor &bc = sm.bc;
  const int tx0 = t.tx * TW, ty0 = t.ty * TH;
  const int tx1 = min(tx0 + TW, P.pano_w) - 1, ty1 = min(ty0 + TH, P.pano_h) - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool empty = tx0 > tx1 || ty0 > ty1;
  load_block_color(P, bc);

  // Source windows: warp 0 for the tile's camera (or a band's left camera),
  // warp 1 for a band's right camera, only where tile pixels need them.
  if (warp < 2) {
    Window W = no_window();
    if (!empty) {
      if (t.kind != 1) {
        if (warp == 0) W = warp_window(P.cam[t.idx], tx0, ty0, tx1, ty1);
      } else {
        const BandDev B = P.band[t.idx];
        const bool rows_out = ty0 < B.y0 || ty1 >= B.y1;
        const bool need = warp == 0 ? (tx0 < B.x0 || (rows_out && tx1 >= B.x0))
                                    : (tx1 >= B.x1 || (rows_out && tx0 < B.x1));
        if (need) W = warp_window(P.cam[t.idx + warp], tx0, ty0, tx1, ty1);
      }
    }
    if (lane == 0) sm.sW[warp] = W;
  }
  __syncthreads();
  const Window W0 = sm.sW[0], W1 = sm.sW[1];
  if (W0.ok) stage_window(P.src[t.idx], P.cam[t.idx], W0, sm.s_win[0]);
  if (W1.ok) stage_window(P.src[t.idx + 1], P.cam[t.idx + 1], W1, sm.s_win[1]);
  __syncthreads();

  if (t.kind == 0) {
    // Fully covered own tile: no coverage test, no fallback.
    const int k = t.idx;
    const CamDev &c = P.cam[k];
    const float *M = bc.M[k];
    const float bx = (float)(tx0 - c.ox), by = (float)(ty0 - c.oy);
    if (c.affine && W0.ok) {
#pragma unroll 2
      for (int j = 0; j < MP::kPix; ++j) {
        const int lx = MP::lx(lane, j), ly = MP::ly(warp, j);
        float sx, sy;
        cam_map_aff(c, bx + (float)lx, by + (float)ly, sx, sy);
        put_px<TW, TH>(sm.s_out, lx, ly, bc, true, mulM(M, win_bilinear(sm.s_win[0], W0, sx, sy)));
      }
    } else {
#pragma unroll 2
      for (int j = 0; j < MP::kPix; ++j) {
        const int lx = MP::lx(lane, j), ly = MP::ly(warp, j);
        float sx, sy, nw;
        cam_map_f(c, bx + (float)lx, by + (float)ly, sx, sy, nw);
        const float3 v =
            mulM(M, W0.ok ? win_bilinear(sm.s_win[0], W0, sx, sy) : src_bilinear(P.src[k], c, sx, sy));
        put_px<TW, TH>(sm.s_out, lx, ly, bc, true, v);
      }
    }
  } else if (t.kind == 2) {
    const int k = t.idx;
    const float *M = bc.M[k];
#pragma unroll 2
    for (int j = 0; j < MP::kPix; ++j) {
      const int lx = MP::lx(lane, j), ly = MP::ly(warp, j);
      const int x = tx0 + lx, y = ty0 + ly;
      float3 v = make_float3(0.0f, 0.0f, 0.0f);
      bool cov = false;
      if (x < P.pano_w && y < P.pano_h) {
        cov = cam_value_w(P, M, k, W0, sm.s_win[0], x, y, v);
        if (!cov && k > 0) cov = cam_value_g(P, bc, k - 1, x, y, v);
        if (!cov && k < P.n_cams - 1) cov = cam_value_g(P, bc, k + 1, x, y, v);
      }
      put_px<TW, TH>(sm.s_out, lx, ly, bc, cov, v);
    }
  } else {
    const int p = t.idx;
    const BandDev B = P.band[p];
    const float *Ma = bc.M[p];
    const float *Mb = bc.M[p + 1];
    const PT *pwa = reinterpret_cast<const PT *>(P.pw) + P.pw_off[p][0];
    const PT *pwb = reinterpret_cast<const PT *>(P.pw) + P.pw_off[p][1];
    const bool printed = (P.flags & STITCH_FLOW_WEIGHTS_PRINTED) != 0;
    const float mf = P.max_flow;
    const int bw = B.x1 - B.x0;
#pragma unroll 2
    for (int j = 0; j < MP::kPix; ++j) {
      const int lx = MP::lx(lane, j), ly = MP::ly(warp, j);
      const int x = tx0 + lx, y = ty0 + ly;
      float3 v = make_float3(0.0f, 0.0f, 0.0f);
      bool cov = false;
      if (x < P.pano_w && y < P.pano_h) {
        if (x < B.x0) {
          cov = cam_value_w(P, Ma, p, W0, sm.s_win[0], x, y, v);
          if (!cov && p > 0) cov = cam_value_g(P, bc, p - 1, x, y, v);
          if (!cov) cov = cam_value_g(P, bc, p + 1, x, y, v);
        } else if (x >= B.x1) {
          cov = cam_value_w(P, Mb, p + 1, W1, sm.s_win[1], x, y, v);
          if (!cov) cov = cam_value_g(P, bc, p, x, y, v);
          if (!cov && p + 2 < P.n_cams) cov = cam_value_g(P, bc, p + 2, x, y, v);
        } else {
          const float tb = ((float)(x - B.x0) + 0.5f) * B.inv_bw;
          const float ta = 1.0f - tb;
          if (y < B.y0 || y >= B.y1) {
            float3 va, vb;
            const bool ca = cam_value_w(P, Ma, p, W0, sm.s_win[0], x, y, va);
            const bool cb = cam_value_w(P, Mb, p + 1, W1, sm.s_win[1], x, y, vb);
            if (ca && cb) {
              v = make_float3(fmaf(ta, va.x, tb * vb.x), fmaf(ta, va.y, tb * vb.y), fmaf(ta, va.z, tb * vb.z));
            } else if (ca) {
              v = va;
            } else if (cb) {
              v = vb;
            }
            cov = ca || cb;
          } else {
            const size_t fi = (size_t)(y - B.y0) * bw + (x - B.x0);
            float2 fa = __ldg(P.flow_ij[p] + fi);
            float2 fb = __ldg(P.flow_ji[p] + fi);
            fa.x = fmaxf(fminf(fa.x, mf), -mf); fa.y = fmaxf(fminf(fa.y, mf), -mf);
            fb.x = fmaxf(fminf(fb.x, mf), -mf); fb.y = fmaxf(fminf(fb.y, mf), -mf);
            const float wa = printed ? ta : tb;
            const float wb = printed ? tb : ta;
            const float lo_x = (float)B.x0, hi_x = (float)(B.x1 - 1);
            const float lo_y = (float)B.y0, hi_y = (float)(B.y1 - 1);
            const float Xa = fminf(fmaxf(fmaf(wa, fa.x, (float)x), lo_x), hi_x);
            const float Ya = fminf(fmaxf(fmaf(wa, fa.y, (float)y), lo_y), hi_y);
            const float Xb = fminf(fmaxf(fmaf(wb, fb.x, (float)x), lo_x), hi_x);
            const float Yb = fminf(fmaxf(fmaf(wb, fb.y, (float)y), lo_y), hi_y);
            const float3 Pa = mulM(Ma, pw_bilinear<kHalf>(pwa, B, Xa, Ya));
            const float3 Pb = mulM(Mb, pw_bilinear<kHalf>(pwb, B, Xb, Yb));
            v = make_float3(fmaf(ta, Pa.x, tb * Pb.x), fmaf(ta, Pa.y, tb * Pb.y), fmaf(ta, Pa.z, tb * Pb.z));
            cov = true;
          }
        }
      }
      put_px<TW, TH>(sm.s_out, lx, ly, bc, cov, v);
    }
  }
  __syncthreads();
  store_tile<TW, TH>(P, tx0, ty0, sm.s_out);
}

// Shared memory of a fully covered own tile: one camera, one window.
template <int TW, int TH>
struct FuseOwnSmem {
  BlockColor bc;
  Window sW;
  __align__(16) uint32_t s_win[kWinCap];
  __align__(16) uint8_t s_out[3][TH][TW];
};

// A fully covered own tile (kind 0) on its own: no band, no coverage test, no
// fallback camera; the same arithmetic as that case of fuse_tile, with the
// registers and shared memory of one camera only.
template <int TW, int TH>
__device__ __forceinline__ void fuse_own_tile(const FuseParams &P, const TileDesc t, FuseOwnSmem<TW, TH> &sm) {
  using MP = Map<TW, TH>;
  BlockColor &bc = sm.bc;
  const int tx0 = t.tx * TW, ty0 = t.ty * TH;
  const int tx1 = min(tx0 + TW, P.pano_w) - 1, ty1 = min(ty0 + TH, P.pano_h) - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = t.idx;
  const CamDev &c = P.cam[k];
  load_block_color(P, bc);
  if (warp == 0) {
    const Window W = warp_window(c, tx0, ty0, tx1, ty1);
    if (lane == 0) sm.sW = W;
  }
  __syncthreads();
  const Window W0 = sm.sW;
  if (W0.ok) stage_window(P.src[k], c, W0, sm.s_win);
  __syncthreads();
  const float *M = bc.M[k];
  const float bx = (float)(tx0 - c.ox), by = (float)(ty0 - c.oy);
  if (c.affine && W0.ok) {
#pragma unroll 2
    for (int j = 0; j < MP::kPix; ++j) {
      const int lx = MP::lx(lane, j), ly = MP::ly(warp, j);
      float sx, sy;
      cam_map_aff(c, bx + (float)lx, by + (float)ly, sx, sy);
      put_px<TW, TH>(sm.s_out, lx, ly, bc, true, mulM(M, win_bilinear(sm.s_win, W0, sx, sy)));
    }
  } else {
#pragma unroll 2
    for (int j = 0; j < MP::kPix; ++j) {
      const int lx = MP::lx(lane, j), ly = MP::ly(warp, j);
      float sx, sy, nw;
      cam_map_f(c, bx + (float)lx, by + (float)ly, sx, sy, nw);
      const float3 v = mulM(M, W0.ok ? win_bilinear(sm.s_win, W0, sx, sy) : src_bilinear(P.src[k], c, sx, sy));
      put_px<TW, TH>(sm.s_out, lx, ly, bc, true, v);
    }
  }
  __syncthreads();
  store_tile<TW, TH>(P, tx0, ty0, sm.s_out);
}

// One band pre-warp piece (kTileW x kTileH) of pair pt.pair, both cameras.
template <bool kHalf>
__device__ __forceinline__ void prewarp_piece(const FuseParams &P, const PwTile pt, uint32_t (*s_win)[kWinCap],
                                              Window *sW) {
  using PT = typename PwT<kHalf>::T;
  const BandDev B = P.band[pt.pair];
  const int bw = B.x1 - B.x0;
  const int rx0 = pt.x0, ry0 = pt.y0;
  const int rx1 = min(rx0 + kTileW, B.x1) - 1, ry1 = min(ry0 + kTileH, B.y1) - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < 2) {
    const Window W = warp_window(P.cam[pt.pair + warp], rx0, ry0, rx1, ry1);
    if (lane == 0) sW[warp] = W;
  }
  __syncthreads();
  const Window Wa = sW[0], Wb = sW[1];
  if (Wa.ok) stage_window(P.src[pt.pair], P.cam[pt.pair], Wa, s_win[0]);
  if (Wb.ok) stage_window(P.src[pt.pair + 1], P.cam[pt.pair + 1], Wb, s_win[1]);
  __syncthreads();
  PT *da = reinterpret_cast<PT *>(P.pw) + P.pw_off[pt.pair][0];
  PT *db = reinterpret_cast<PT *>(P.pw) + P.pw_off[pt.pair][1];
  const CamDev &ca = P.cam[pt.pair];
  const CamDev &cb = P.cam[pt.pair + 1];
#pragma unroll 2
  for (int j = 0; j < 8; ++j) {
    const int x = rx0 + lane + 32 * (j & 1);
    const int y = ry0 + 4 * warp + (j >> 1);
    if (x > rx1 || y > ry1) continue;
    const size_t o = (size_t)(y - B.y0) * bw + (x - B.x0);
    float sx, sy, nw;
    // The band lies inside both cameras' coverage: clamp float32 noise away.
    cam_map_f(ca, (float)(x - ca.ox), (float)(y - ca.oy), sx, sy, nw);
    sx = fminf(fmaxf(sx, 0.0f), ca.wm1);
    sy = fminf(fmaxf(sy, 0.0f), ca.hm1);
    PwT<kHalf>::put(da, o, Wa.ok ? win_bilinear(s_win[0], Wa, sx, sy) : src_bilinear(P.src[pt.pair], ca, sx, sy));
    cam_map_f(cb, (float)(x - cb.ox), (float)(y - cb.oy), sx, sy, nw);
    sx = fminf(fmaxf(sx, 0.0f), cb.wm1);
    sy = fminf(fmaxf(sy, 0.0f), cb.hm1);
    PwT<kHalf>::put(db, o, Wb.ok ? win_bilinear(s_win[1], Wb, sx, sy) : src_bilinear(P.src[pt.pair + 1], cb, sx, sy));
  }
}

// Copy one rig's parameters into shared memory (16-byte words).
__device__ __forceinline__ void copy_params(FuseParams &dst, const FuseParams *src) {
  static_assert(sizeof(FuseParams) % 16 == 0, "parameter block must be a whole number of 16-byte words");
  const int4 *s = reinterpret_cast<const int4 *>(src);
  int4 *d = reinterpret_cast<int4 *>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(FuseParams) / 16); i += blockDim.x) d[i] = __ldg(s + i);
}

}  // namespace

// ---------------------------------------------------------------------------
// Kernels.
// ---------------------------------------------------------------------------

template <bool kHalf>
__global__ void __launch_bounds__(kFuseThreads) k_prewarp_band(const FuseParams P) {
  __shared__ __align__(16) uint32_t s_win[2][kWinCap];
  __shared__ Window sW[2];
  prewarp_piece<kHalf>(P, P.pw_tiles[blockIdx.x], s_win, sW);
}

template <bool kHalf, int TW, int TH>
__global__ void __launch_bounds__(kFuseThreads, 4) k_fuse(const FuseParams P) {
  __shared__ FuseSmem<TW, TH> sm;
  fuse_tile<kHalf, TW, TH>(P, P.tiles[blockIdx.x], sm);
}

// The fully covered own tiles, which close the tile list (P.n_full of them).
template <int TW, int TH>
__global__ void __launch_bounds__(kFuseThreads, 4) k_fuse_own(const FuseParams P) {
  __shared__ FuseOwnSmem<TW, TH> sm;
  fuse_own_tile<TW, TH>(P, P.tiles[P.n_tiles - P.n_full + blockIdx.x], sm);
}

// Band pre-warp of several rigs in one launch: block b takes item b.
template <bool kHalf>
__global__ void __launch_bounds__(kFuseThreads) k_prewarp_multi(const MultiParams M) {
  __shared__ __align__(16) uint32_t s_win[2][kWinCap];
  __shared__ Window sW[2];
  __shared__ FuseParams sp;
  const MultiItem it = M.items[blockIdx.x];
  copy_params(sp, M.params + M.base + it.rig);
  __syncthreads();
  prewarp_piece<kHalf>(sp, it.pw, s_win, sW);
}

// Shared memory of the persistent multi-rig kernels: room for any tile shape
// (every rig's tiles use that rig's own shape).
union MultiSmem {
  FuseSmem<64, 32> s0;
  FuseSmem<64, 16> s1;
  FuseSmem<32, 32> s2;
  FuseSmem<128, 16> s3;
};
union MultiOwnSmem {
  FuseOwnSmem<64, 32> s0;
  FuseOwnSmem<64, 16> s1;
  FuseOwnSmem<32, 32> s2;
  FuseOwnSmem<128, 16> s3;
};

// One tile of a multi-rig launch in its own call frame, so that each shape's
// code gets its own register allocation inside the mixed-shape kernels.
template <bool kHalf, int TW, int TH>
__device__ __noinline__ void multi_tile(const FuseParams &P, const TileDesc t, FuseSmem<TW, TH> &sm) {
  fuse_tile<kHalf, TW, TH>(P, t, sm);
}
template <int TW, int TH>
__device__ __noinline__ void multi_own_tile(const FuseParams &P, const TileDesc t, FuseOwnSmem<TW, TH> &sm) {
  fuse_own_tile<TW, TH>(P, t, sm);
}

// Persistent fuse over the tiles of several rigs: each block takes the next
// item from a work counter until none is left (dynamic balance of uneven tile
// costs), loading a rig's parameters into shared memory when the rig changes.
// k_fuse_multi serves batches whose rigs share one tile shape;
// k_fuse_multi_mixed runs every item with its rig's own shape.
template <bool kHalf, int TW, int TH>
__global__ void __launch_bounds__(kFuseThreads, 4) k_fuse_multi(const MultiParams M) {
  __shared__ FuseSmem<TW, TH> sm;
  __shared__ FuseParams sp;
  __shared__ int s_item;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(M.counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= M.n_items) break;
    const MultiItem it = M.items[item];
    if (it.rig != cur) {
      copy_params(sp, M.params + M.base + it.rig);
      cur = it.rig;
    }
    __syncthreads();
    fuse_tile<kHalf, TW, TH>(sp, it.tile, sm);
    __syncthreads();
  }
}

template <bool kHalf>
__global__ void __launch_bounds__(kFuseThreads, 4) k_fuse_multi_mixed(const MultiParams M) {
  __shared__ MultiSmem sm;
  __shared__ FuseParams sp;
  __shared__ int s_item;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(M.counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= M.n_items) break;
    const MultiItem it = M.items[item];
    if (it.rig != cur) {
      copy_params(sp, M.params + M.base + it.rig);
      cur = it.rig;
    }
    __syncthreads();
    switch (it.shape) {
      case 0: multi_tile<kHalf, 64, 32>(sp, it.tile, sm.s0); break;
      case 1: multi_tile<kHalf, 64, 16>(sp, it.tile, sm.s1); break;
      case 2: multi_tile<kHalf, 32, 32>(sp, it.tile, sm.s2); break;
      default: multi_tile<kHalf, 128, 16>(sp, it.tile, sm.s3); break;
    }
    __syncthreads();
  }
}

// Persistent fuse over the fully covered own tiles of several rigs (one shape
// for all rigs, or each rig's own).
template <int TW, int TH>
__global__ void __launch_bounds__(kFuseThreads, 4) k_fuse_own_multi(const MultiParams M) {
  __shared__ FuseOwnSmem<TW, TH> sm;
  __shared__ FuseParams sp;
  __shared__ int s_item;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(M.counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= M.n_items) break;
    const MultiItem it = M.items[item];
    if (it.rig != cur) {
      copy_params(sp, M.params + M.base + it.rig);
      cur = it.rig;
    }
    __syncthreads();
    fuse_own_tile<TW, TH>(sp, it.tile, sm);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kFuseThreads, 4) k_fuse_own_multi_mixed(const MultiParams M) {
  __shared__ MultiOwnSmem sm;
  __shared__ FuseParams sp;
  __shared__ int s_item;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(M.counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= M.n_items) break;
    const MultiItem it = M.items[item];
    if (it.rig != cur) {
      copy_params(sp, M.params + M.base + it.rig);
      cur = it.rig;
    }
    __syncthreads();
    switch (it.shape) {
      case 0: multi_own_tile<64, 32>(sp, it.tile, sm.s0); break;
      case 1: multi_own_tile<64, 16>(sp, it.tile, sm.s1); break;
      case 2: multi_own_tile<32, 32>(sp, it.tile, sm.s2); break;
      default: multi_own_tile<128, 16>(sp, it.tile, sm.s3); break;
    }
    __syncthreads();
  }
}

size_t prewarp_elem_bytes(bool fp16) { return fp16 ? sizeof(uint2) : sizeof(float4); }

cudaError_t fuse_setup_attributes(int) { return cudaSuccess; }

cudaError_t launch_prewarp(const FuseParams &p, cudaStream_t s) {
  if (p.n_pw_tiles <= 0) return cudaSuccess;
  if (p.flags & STITCH_FP16_INTERMEDIATE)
    k_prewarp_band<true><<<p.n_pw_tiles, kFuseThreads, 0, s>>>(p);
  else
    k_prewarp_band<false><<<p.n_pw_tiles, kFuseThreads, 0, s>>>(p);
  return cudaGetLastError();
}

namespace {

// The tiles that touch a band or are partly covered (k_fuse), then the fully
// covered own tiles (k_fuse_own), in one stream.
template <int TW, int TH>
void fuse_multi_by_half(const MultiParams &m, bool half, int grid, cudaStream_t s) {
  if (half)
    k_fuse_multi<true, TW, TH><<<grid, kFuseThreads, 0, s>>>(m);
  else
    k_fuse_multi<false, TW, TH><<<grid, kFuseThreads, 0, s>>>(m);
}

template <int TW, int TH>
int occupancy(bool half) {
  int n = 0;
  if (half)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fuse_multi<true, TW, TH>, kFuseThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fuse_multi<false, TW, TH>, kFuseThreads, 0);
  return n;
}

template <int TW, int TH>
void fuse_by_half(const FuseParams &p, cudaStream_t s) {
  const int mixed = p.n_tiles - p.n_full;
  if (mixed > 0) {
    if (p.flags & STITCH_FP16_INTERMEDIATE)
      k_fuse<true, TW, TH><<<mixed, kFuseThreads, 0, s>>>(p);
    else
      k_fuse<false, TW, TH><<<mixed, kFuseThreads, 0, s>>>(p);
  }
  if (p.n_full > 0) k_fuse_own<TW, TH><<<p.n_full, kFuseThreads, 0, s>>>(p);
}



}  // namespace

static_assert(kTileShapes[0].w == 64 && kTileShapes[0].h == 32 && kTileShapes[1].w == 64 && kTileShapes[1].h == 16 &&
                  kTileShapes[2].w == 32 && kTileShapes[2].h == 32 && kTileShapes[3].w == 128 &&
                  kTileShapes[3].h == 16,
              "the shape table and the kernel instantiations below must agree");

cudaError_t launch_fuse(const FuseParams &p, int shape, cudaStream_t s) {
  if (p.n_tiles <= 0) return cudaSuccess;
  switch (shape) {
    case 0: fuse_by_half<64, 32>(p, s); break;
    case 1: fuse_by_half<64, 16>(p, s); break;
    case 2: fuse_by_half<32, 32>(p, s); break;
    case 3: fuse_by_half<128, 16>(p, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_prewarp_multi(const MultiParams &m, bool half, cudaStream_t s) {
  if (m.n_items <= 0) return cudaSuccess;
  if (half)
    k_prewarp_multi<true><<<m.n_items, kFuseThreads, 0, s>>>(m);
  else
    k_prewarp_multi<false><<<m.n_items, kFuseThreads, 0, s>>>(m);
  return cudaGetLastError();
}

cudaError_t launch_fuse_multi(const MultiParams &m, bool half, int shape, int grid, cudaStream_t s) {
  if (m.n_items <= 0) return cudaSuccess;
  switch (shape) {
    case -1:
      if (half)
        k_fuse_multi_mixed<true><<<grid, kFuseThreads, 0, s>>>(m);
      else
        k_fuse_multi_mixed<false><<<grid, kFuseThreads, 0, s>>>(m);
      break;
    case 0: fuse_multi_by_half<64, 32>(m, half, grid, s); break;
    case 1: fuse_multi_by_half<64, 16>(m, half, grid, s); break;
    case 2: fuse_multi_by_half<32, 32>(m, half, grid, s); break;
    case 3: fuse_multi_by_half<128, 16>(m, half, grid, s); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fuse_own_multi(const MultiParams &m, int shape, int grid, cudaStream_t s) {
  if (m.n_items <= 0) return cudaSuccess;
  switch (shape) {
    case -1: k_fuse_own_multi_mixed<<<grid, kFuseThreads, 0, s>>>(m); break;
    case 0: k_fuse_own_multi<64, 32><<<grid, kFuseThreads, 0, s>>>(m); break;
    case 1: k_fuse_own_multi<64, 16><<<grid, kFuseThreads, 0, s>>>(m); break;
    case 2: k_fuse_own_multi<32, 32><<<grid, kFuseThreads, 0, s>>>(m); break;
    case 3: k_fuse_own_multi<128, 16><<<grid, kFuseThreads, 0, s>>>(m); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int fuse_own_multi_blocks_per_sm(int shape) {
  int n = 0;
  switch (shape) {
    case -1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fuse_own_multi_mixed, kFuseThreads, 0); break;
    case 0: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fuse_own_multi<64, 32>, kFuseThreads, 0); break;
    case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fuse_own_multi<64, 16>, kFuseThreads, 0); break;
    case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fuse_own_multi<32, 32>, kFuseThreads, 0); break;
    case 3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fuse_own_multi<128, 16>, kFuseThreads, 0); break;
    default: break;
  }
  return n;
}

int fuse_multi_blocks_per_sm(bool half, int shape) {
  switch (shape) {
    case -1: {
      int n = 0;
      if (half)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fuse_multi_mixed<true>, kFuseThreads, 0);
      else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fuse_multi_mixed<false>, kFuseThreads, 0);
      return n;
    }
    case 0: return occupancy<64, 32>(half);
    case 1: return occupancy<64, 16>(half);
    case 2: return occupancy<32, 32>(half);
    case 3: return occupancy<128, 16>(half);
    default: return 0;
  }
}

}  // namespace stitch
