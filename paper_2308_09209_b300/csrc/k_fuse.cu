// K3 -- fused pre-warp, local warping, colour transfer, blend and balance
// (paper section 3.1 pre-warp; section 3.2 Eq. 15-18; Eq. 4; Eq. 5).
//
// The panorama is cut into 64 x 16 tiles; each thread produces 4 consecutive
// pixels of one row and writes them as one 4-byte store per colour plane.
//
// Own tiles (columns that belong to one camera k only): s = H_k^-1 q in
// float32 relative to the camera's panorama origin, coverage test
// 0 <= s <= (w-1, h-1), bilinear sample of the packed-RGB source (taps at
// floor(s), floor(s)+1, far tap clamped), v = P . M_k. A pixel camera k does
// not cover falls back to camera k-1, then k+1 (Eq. 15's one-image cases),
// else it is 0.
//
// Band tiles (columns of a pair's blend band): the tile's part of the band
// rectangle, widened by the flow halo and clipped to the band, is pre-warped
// for BOTH cameras into shared memory with M already applied (the pre-warped
// image of section 3.1, stored as float32, or float16 with
// STITCH_FP16_INTERMEDIATE). Each band pixel then computes
//   theta_j = (x - x0 + 0.5) / (x1 - x0), theta_i = 1 - theta_j (Eq. 16 read
//   as a ramp), X_i = q + theta_j clamp(flow_ij), X_j = q + theta_i
//   clamp(flow_ji) (Eq. 17, continuous reading; the printed weights under
//   STITCH_FLOW_WEIGHTS_PRINTED), clamps X into the band and samples the
//   staged tile bilinearly (Eq. 18): out = theta_i P_i(X_i) + theta_j P_j(X_j).
// Pixels of the band columns outside the band rows blend both cameras without
// flow where both cover them, else take the one that does.
//
// Finally each channel is clamped to [0, 255], passed through the piecewise
// balance curve F (Eq. 5: gamma, linear, gamma) and rounded half to even.
#include <cuda_fp16.h>

#include "stitch_internal.h"

namespace stitch {

namespace {

struct Region {
  int x0, y0, w, h;
};

__device__ __forceinline__ bool cam_map(const CamDev &c, int x, int y, float &sx, float &sy) {
  const float dx = (float)(x - c.ox);
  const float dy = (float)(y - c.oy);
  const float nx = fmaf(c.h[0], dx, fmaf(c.h[1], dy, c.h[2]));
  const float ny = fmaf(c.h[3], dx, fmaf(c.h[4], dy, c.h[5]));
  const float nw = fmaf(c.h[6], dx, fmaf(c.h[7], dy, c.h[8]));
  const float r = 1.0f / nw;
  sx = nx * r;
  sy = ny * r;
  return nw > 0.0f && sx >= 0.0f && sx <= c.wm1 && sy >= 0.0f && sy <= c.hm1;
}

__device__ __forceinline__ float3 load_rgb(const uint8_t *__restrict__ p) {
  return make_float3((float)__ldg(p), (float)__ldg(p + 1), (float)__ldg(p + 2));
}

// Bilinear sample of a packed-RGB frame at (sx, sy), assumed inside the frame.
__device__ __forceinline__ float3 src_bilinear(const uint8_t *__restrict__ src, const CamDev &c,
                                               float sx, float sy) {
  const float fx0 = floorf(sx), fy0 = floorf(sy);
  const float fx = sx - fx0, fy = sy - fy0;
  const int ix = (int)fx0, iy = (int)fy0;
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

__device__ __forceinline__ bool cam_value(const FuseParams &P, const ColorOut &col, int k, int x, int y,
                                          float3 &v) {
  float sx, sy;
  if (!cam_map(P.cam[k], x, y, sx, sy)) return false;
  v = mulM(col.M[k], src_bilinear(P.src[k], P.cam[k], sx, sy));
  return true;
}

__device__ __forceinline__ bool own_value(const FuseParams &P, const ColorOut &col, int k, int x, int y,
                                          float3 &v) {
  if (cam_value(P, col, k, x, y, v)) return true;
  if (k > 0 && cam_value(P, col, k - 1, x, y, v)) return true;
  if (k < P.n_cams - 1 && cam_value(P, col, k + 1, x, y, v)) return true;
  return false;
}

// Band columns outside the band rows: Eq. 15 without flow.
__device__ __forceinline__ bool sliver_value(const FuseParams &P, const ColorOut &col, int p, int x, int y,
                                             float3 &v) {
  float3 va, vb;
  const bool ca = cam_value(P, col, p, x, y, va);
  const bool cb = cam_value(P, col, p + 1, x, y, vb);
  if (ca && cb) {
    const float tb = ((float)(x - P.band[p].x0) + 0.5f) * P.band[p].inv_bw;
    const float ta = 1.0f - tb;
    v = make_float3(ta * va.x + tb * vb.x, ta * va.y + tb * vb.y, ta * va.z + tb * vb.z);
    return true;
  }
  if (ca) { v = va; return true; }
  if (cb) { v = vb; return true; }
  return false;
}

__device__ __forceinline__ float balance(const Curve &cv, float x) {
  if (cv.ident != 0.0f) return x;
  if (x < cv.m1) return cv.d1 * __powf(x * cv.inv_m1, cv.g1);
  if (x > cv.m2) return 255.0f - (255.0f - cv.d2) * __powf((255.0f - x) * cv.inv_bm, cv.g2);
  return fmaf(cv.s, x - cv.m1, cv.d1);
}

__device__ __forceinline__ uint32_t to_u8(const Curve &cv, bool bal, float x) {
  x = fminf(fmaxf(x, 0.0f), 255.0f);
  if (bal) x = balance(cv, x);
  const int r = __float2int_rn(x);
  return (uint32_t)min(max(r, 0), 255);
}

template <bool kHalf>
struct StageT;
template <>
struct StageT<false> {
  using T = float;
  __device__ static void put(float *s, int i, float3 v) { s[3 * i] = v.x; s[3 * i + 1] = v.y; s[3 * i + 2] = v.z; }
  __device__ static float3 get(const float *s, int i) { return make_float3(s[3 * i], s[3 * i + 1], s[3 * i + 2]); }
};
template <>
struct StageT<true> {
  using T = __half;
  __device__ static void put(__half *s, int i, float3 v) {
    s[3 * i] = __float2half_rn(v.x); s[3 * i + 1] = __float2half_rn(v.y); s[3 * i + 2] = __float2half_rn(v.z);
  }
  __device__ static float3 get(const __half *s, int i) {
    return make_float3(__half2float(s[3 * i]), __half2float(s[3 * i + 1]), __half2float(s[3 * i + 2]));
  }
};

template <bool kHalf>
__device__ __forceinline__ float3 staged_bilinear(const typename StageT<kHalf>::T *s, const Region &R,
                                                  const BandDev &B, float X, float Y) {
  const float jx = floorf(X), jy = floorf(Y);
  const float gx = X - jx, gy = Y - jy;
  const int ix = (int)jx, iy = (int)jy;
  const int ix1 = min(ix + 1, B.x1 - 1), iy1 = min(iy + 1, B.y1 - 1);
  const int lx0 = min(max(ix - R.x0, 0), R.w - 1), lx1 = min(max(ix1 - R.x0, 0), R.w - 1);
  const int ly0 = min(max(iy - R.y0, 0), R.h - 1), ly1 = min(max(iy1 - R.y0, 0), R.h - 1);
  const float3 a = StageT<kHalf>::get(s, ly0 * R.w + lx0), b = StageT<kHalf>::get(s, ly0 * R.w + lx1);
  const float3 d = StageT<kHalf>::get(s, ly1 * R.w + lx0), e = StageT<kHalf>::get(s, ly1 * R.w + lx1);
  float3 t, u, o;
  t.x = fmaf(gx, b.x - a.x, a.x); t.y = fmaf(gx, b.y - a.y, a.y); t.z = fmaf(gx, b.z - a.z, a.z);
  u.x = fmaf(gx, e.x - d.x, d.x); u.y = fmaf(gx, e.y - d.y, d.y); u.z = fmaf(gx, e.z - d.z, d.z);
  o.x = fmaf(gy, u.x - t.x, t.x); o.y = fmaf(gy, u.y - t.y, t.y); o.z = fmaf(gy, u.z - t.z, t.z);
  return o;
}

__device__ __forceinline__ void store4(const FuseParams &P, int x, int y, const uint32_t (&o)[3]) {
  if (x >= P.pano_pitch || y >= P.pano_h) return;
  const size_t plane = (size_t)P.pano_pitch * P.pano_h;
  uint8_t *base = P.out + (size_t)y * P.pano_pitch + x;
#pragma unroll
  for (int c = 0; c < 3; ++c) *reinterpret_cast<uint32_t *>(base + c * plane) = o[c];
}

__device__ __forceinline__ void load_color(const FuseParams &P, ColorOut &s_col) {
  const int n = (int)(sizeof(ColorOut) / 4);
  const uint32_t *src = reinterpret_cast<const uint32_t *>(P.color);
  uint32_t *dst = reinterpret_cast<uint32_t *>(&s_col);
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

__global__ void __launch_bounds__(kFuseThreads) k_fuse_own(const FuseParams P, int tile0) {
  __shared__ ColorOut s_col;
  load_color(P, s_col);
  __syncthreads();
  const TileDesc t = P.tiles[tile0 + blockIdx.x];
  const int k = t.idx;
  const int x = t.tx * kTileW + (threadIdx.x & 15) * 4;
  const int y = t.ty * kTileH + (threadIdx.x >> 4);
  const bool bal = !(P.flags & STITCH_BALANCE_OFF);
  uint32_t o[3] = {0u, 0u, 0u};
  if (y < P.pano_h) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int xi = x + i;
      float3 v;
      if (xi < P.pano_w && own_value(P, s_col, k, xi, y, v)) {
        o[0] |= to_u8(s_col.curve[0], bal, v.x) << (8 * i);
        o[1] |= to_u8(s_col.curve[1], bal, v.y) << (8 * i);
        o[2] |= to_u8(s_col.curve[2], bal, v.z) << (8 * i);
      }
    }
  }
  store4(P, x, y, o);
}

template <bool kHalf>
__global__ void __launch_bounds__(kFuseThreads) k_fuse_band(const FuseParams P, int tile0) {
  using ST = typename StageT<kHalf>::T;
  __shared__ ColorOut s_col;
  extern __shared__ __align__(16) unsigned char s_raw[];
  load_color(P, s_col);
  const TileDesc t = P.tiles[tile0 + blockIdx.x];
  const int p = t.idx;
  const BandDev B = P.band[p];
  const int tx0 = t.tx * kTileW, ty0 = t.ty * kTileH;
  Region R;
  R.x0 = max(B.x0, tx0 - P.halo);
  R.y0 = max(B.y0, ty0 - P.halo);
  R.w = min(B.x1, tx0 + kTileW + P.halo) - R.x0;
  R.h = min(B.y1, ty0 + kTileH + P.halo) - R.y0;
  const bool staged = R.w > 0 && R.h > 0 && tx0 < B.x1 && tx0 + kTileW > B.x0 && ty0 < B.y1 &&
                      ty0 + kTileH > B.y0;
  ST *sA = reinterpret_cast<ST *>(s_raw);
  ST *sB = sA + (staged ? 3 * R.w * R.h : 0);
  __syncthreads();
  if (staged) {
    const CamDev &ca = P.cam[p];
    const CamDev &cb = P.cam[p + 1];
    for (int i = threadIdx.x; i < R.w * R.h; i += blockDim.x) {
      const int ly = i / R.w;
      const int px = R.x0 + (i - ly * R.w);
      const int py = R.y0 + ly;
      float sx, sy;
      cam_map(ca, px, py, sx, sy);
      sx = fminf(fmaxf(sx, 0.0f), ca.wm1);
      sy = fminf(fmaxf(sy, 0.0f), ca.hm1);
      StageT<kHalf>::put(sA, i, mulM(s_col.M[p], src_bilinear(P.src[p], ca, sx, sy)));
      cam_map(cb, px, py, sx, sy);
      sx = fminf(fmaxf(sx, 0.0f), cb.wm1);
      sy = fminf(fmaxf(sy, 0.0f), cb.hm1);
      StageT<kHalf>::put(sB, i, mulM(s_col.M[p + 1], src_bilinear(P.src[p + 1], cb, sx, sy)));
    }
  }
  __syncthreads();
  const int x = tx0 + (threadIdx.x & 15) * 4;
  const int y = ty0 + (threadIdx.x >> 4);
  const bool bal = !(P.flags & STITCH_BALANCE_OFF);
  const bool printed = (P.flags & STITCH_FLOW_WEIGHTS_PRINTED) != 0;
  const float mf = P.max_flow;
  uint32_t o[3] = {0u, 0u, 0u};
  if (y < P.pano_h) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int xi = x + i;
      if (xi >= P.pano_w) continue;
      float3 v;
      bool cov;
      if (xi < B.x0) {
        cov = own_value(P, s_col, p, xi, y, v);
      } else if (xi >= B.x1) {
        cov = own_value(P, s_col, p + 1, xi, y, v);
      } else if (y < B.y0 || y >= B.y1) {
        cov = sliver_value(P, s_col, p, xi, y, v);
      } else {
        const int bw = B.x1 - B.x0;
        const size_t fi = (size_t)(y - B.y0) * bw + (xi - B.x0);
        float2 fa = __ldg(P.flow_ij[p] + fi);
        float2 fb = __ldg(P.flow_ji[p] + fi);
        fa.x = fmaxf(fminf(fa.x, mf), -mf); fa.y = fmaxf(fminf(fa.y, mf), -mf);
        fb.x = fmaxf(fminf(fb.x, mf), -mf); fb.y = fmaxf(fminf(fb.y, mf), -mf);
        const float tb = ((float)(xi - B.x0) + 0.5f) * B.inv_bw;
        const float ta = 1.0f - tb;
        const float wa = printed ? ta : tb;
        const float wb = printed ? tb : ta;
        const float lo_x = (float)B.x0, hi_x = (float)(B.x1 - 1);
        const float lo_y = (float)B.y0, hi_y = (float)(B.y1 - 1);
        const float Xa = fminf(fmaxf(fmaf(wa, fa.x, (float)xi), lo_x), hi_x);
        const float Ya = fminf(fmaxf(fmaf(wa, fa.y, (float)y), lo_y), hi_y);
        const float Xb = fminf(fmaxf(fmaf(wb, fb.x, (float)xi), lo_x), hi_x);
        const float Yb = fminf(fmaxf(fmaf(wb, fb.y, (float)y), lo_y), hi_y);
        const float3 Pa = staged_bilinear<kHalf>(sA, R, B, Xa, Ya);
        const float3 Pb = staged_bilinear<kHalf>(sB, R, B, Xb, Yb);
        v = make_float3(fmaf(ta, Pa.x, tb * Pb.x), fmaf(ta, Pa.y, tb * Pb.y), fmaf(ta, Pa.z, tb * Pb.z));
        cov = true;
      }
      if (cov) {
        o[0] |= to_u8(s_col.curve[0], bal, v.x) << (8 * i);
        o[1] |= to_u8(s_col.curve[1], bal, v.y) << (8 * i);
        o[2] |= to_u8(s_col.curve[2], bal, v.z) << (8 * i);
      }
    }
  }
  store4(P, x, y, o);
}

}  // namespace

size_t fuse_band_smem_bytes(int halo, bool fp16) {
  const size_t pos = (size_t)(kTileW + 2 * halo) * (size_t)(kTileH + 2 * halo);
  return pos * 2 * 3 * (fp16 ? 2 : 4);
}

cudaError_t fuse_setup_attributes(int max_halo) {
  cudaError_t e = cudaFuncSetAttribute(k_fuse_band<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fuse_band_smem_bytes(max_halo, false));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fuse_band<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)fuse_band_smem_bytes(max_halo, true));
}

cudaError_t launch_fuse(const FuseParams &p, int n_own_tiles, int n_band_tiles, cudaStream_t s) {
  const bool fp16 = (p.flags & STITCH_FP16_INTERMEDIATE) != 0;
  if (n_band_tiles > 0) {
    const size_t smem = fuse_band_smem_bytes(p.halo, fp16);
    if (fp16)
      k_fuse_band<true><<<n_band_tiles, kFuseThreads, smem, s>>>(p, 0);
    else
      k_fuse_band<false><<<n_band_tiles, kFuseThreads, smem, s>>>(p, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (n_own_tiles > 0) {
    k_fuse_own<<<n_own_tiles, kFuseThreads, 0, s>>>(p, n_band_tiles);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

}  // namespace stitch
