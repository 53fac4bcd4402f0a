// Host side of the stitching library: configuration checks, float64 overlap
// geometry (paper section 2.1 step 1, section 3.1), device state, launches and
// the C ABI declared in include/stitch.h.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "stitch_internal.h"

using namespace stitch;

namespace {

thread_local std::string g_last_error;

constexpr double kSnap = 1e-9;
constexpr uint32_t kStateMagic = 0x53544331u;  // "STC1"

// Bounds round inward; values within 1e-9 of an integer snap to it first so
// float64 noise cannot move an integer bound.
int ceil_snap(double v) {
  const double r = std::nearbyint(v);
  if (std::fabs(v - r) < kSnap) return (int)r;
  return (int)std::ceil(v);
}

int floor_snap(double v) {
  const double r = std::nearbyint(v);
  if (std::fabs(v - r) < kSnap) return (int)r;
  return (int)std::floor(v);
}

// 3x3 inverse by the adjugate; false if the determinant is not usable.
bool inv3(const double *m, double *o) {
  const double c00 = m[4] * m[8] - m[5] * m[7];
  const double c01 = m[5] * m[6] - m[3] * m[8];
  const double c02 = m[3] * m[7] - m[4] * m[6];
  const double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
  if (!std::isfinite(det) || std::fabs(det) < 1e-300) return false;
  const double id = 1.0 / det;
  o[0] = c00 * id;
  o[1] = (m[2] * m[7] - m[1] * m[8]) * id;
  o[2] = (m[1] * m[5] - m[2] * m[4]) * id;
  o[3] = c01 * id;
  o[4] = (m[0] * m[8] - m[2] * m[6]) * id;
  o[5] = (m[2] * m[3] - m[0] * m[5]) * id;
  o[6] = c02 * id;
  o[7] = (m[1] * m[6] - m[0] * m[7]) * id;
  o[8] = (m[0] * m[4] - m[1] * m[3]) * id;
  return true;
}

void proj(const double *H, double x, double y, double &X, double &Y, double &W) {
  const double a = H[0] * x + H[1] * y + H[2];
  const double b = H[3] * x + H[4] * y + H[5];
  W = H[6] * x + H[7] * y + H[8];
  X = a / W;
  Y = b / W;
}

// A named NVTX range over a public call (header-only NVTX: a no-op unless a
// profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

struct Geo {
  int n = 0;
  int w[kMaxCams], h[kMaxCams], pitch[kMaxCams];
  double H[kMaxCams][9], Hi[kMaxCams][9];
  int pano_w = 0, pano_h = 0, pano_pitch = 0;
  int ref = 0;
  int band[kMaxPairs][4];            // x0, x1, y0, y1
  int rect[kMaxPairs][2][4];         // [pair][left/right camera] x0, x1, y0, y1
  int pair_i[kMaxPairs], pair_j[kMaxPairs];
  int own_lo[kMaxCams], own_hi[kMaxCams];
  int cyl = 0;                       // cylindrical projection: H = camera pixel -> ray
  double f = 1.0, cx = 0.0, cy = 0.0;  // cylinder: pixels per radian, centre
};

// Panorama point -> camera k (homogeneous: source point and its w; w > 0 in
// front of the camera). Planar: H_k^-1 q. Cylindrical: H_k^-1 applied to the
// ray (sin theta, h, cos theta), theta = (x - cx) / f, h = (y - cy) / f.
void pano_to_cam(const Geo &g, int k, double x, double y, double &sx, double &sy, double &sw) {
  if (!g.cyl) {
    proj(g.Hi[k], x, y, sx, sy, sw);
    return;
  }
  const double th = (x - g.cx) / g.f, hh = (y - g.cy) / g.f;
  const double d0 = std::sin(th), d2 = std::cos(th);
  const double *A = g.Hi[k];
  const double a = A[0] * d0 + A[1] * hh + A[2] * d2;
  const double b = A[3] * d0 + A[4] * hh + A[5] * d2;
  sw = A[6] * d0 + A[7] * hh + A[8] * d2;
  sx = a / sw;
  sy = b / sw;
}

// Camera pixel -> panorama point. Cylindrical: the ray d = H_k (u, v, 1) at
// azimuth atan2(d_x, d_z) and height d_y / sqrt(d_x^2 + d_z^2).
void cam_to_pano(const Geo &g, int k, double u, double v, double &X, double &Y) {
  if (!g.cyl) {
    double W;
    proj(g.H[k], u, v, X, Y, W);
    return;
  }
  const double *C = g.H[k];
  const double d0 = C[0] * u + C[1] * v + C[2];
  const double d1 = C[3] * u + C[4] * v + C[5];
  const double d2 = C[6] * u + C[7] * v + C[8];
  X = g.cx + g.f * std::atan2(d0, d2);
  Y = g.cy + g.f * (d1 / std::sqrt(d0 * d0 + d2 * d2));
}

bool covered64(const Geo &g, int k, double x, double y) {
  double sx, sy, sw;
  pano_to_cam(g, k, x, y, sx, sy, sw);
  return sw > 0 && sx >= 0 && sx <= g.w[k] - 1 && sy >= 0 && sy <= g.h[k] - 1;
}

// Camera corner pixel centres in the panorama: TL, TR, BR, BL.
void corners(const Geo &g, int k, double cx[4], double cy[4]) {
  const double u[4] = {0.0, g.w[k] - 1.0, g.w[k] - 1.0, 0.0};
  const double v[4] = {0.0, 0.0, g.h[k] - 1.0, g.h[k] - 1.0};
  for (int i = 0; i < 4; ++i) {
    double W;
    proj(g.H[k], u[i], v[i], cx[i], cy[i], W);
  }
}

double line_y(double px, double py, double qx, double qy, double x) {
  return py + (qy - py) * (x - px) / (qx - px);
}

#define FAIL(msg)               \
  do {                          \
    err = (msg);                \
    return STITCH_EINVAL;       \
  } while (0)

// The blend band of cameras (a, b = a + 1): columns from the right-most point
// of b's left edge to the left-most point of a's right edge; rows between the
// lowest top edge and the highest bottom edge of both cameras over those
// columns; all bounds rounded inward. The source rectangle of a band in a
// camera is the inward-rounded box spanned by its corners mapped through
// H^-1. Colour pairs point toward the reference camera.
int build_geometry(const stitch_config *cfg, Geo &g, std::string &err) {
  if (!cfg) FAIL("config is NULL");
  if (cfg->n_cams < 2 || cfg->n_cams > kMaxCams) FAIL("n_cams must be in [2, 8]");
  if (!cfg->cam_w || !cfg->cam_h || !cfg->H) FAIL("cam_w, cam_h and H are required");
  if (cfg->projection != STITCH_PROJ_PLANAR && cfg->projection != STITCH_PROJ_CYLINDRICAL)
    FAIL("projection must be STITCH_PROJ_PLANAR or STITCH_PROJ_CYLINDRICAL");
  if (cfg->projection == STITCH_PROJ_CYLINDRICAL &&
      !(std::isfinite(cfg->cyl_focal) && cfg->cyl_focal > 0.0 && std::isfinite(cfg->cyl_cx) &&
        std::isfinite(cfg->cyl_cy)))
    FAIL("the cylindrical projection needs a positive finite cyl_focal and a finite centre");
  if (cfg->pano_w < 1 || cfg->pano_h < 1) FAIL("panorama size must be positive");
  if (cfg->pano_w > 32767 * kTileW || cfg->pano_h > 32767 * kTileH) FAIL("panorama too large");
  if (cfg->pano_pitch < cfg->pano_w || cfg->pano_pitch % 16 != 0)
    FAIL("pano_pitch must be >= pano_w and a multiple of 16");
  if (cfg->window < 1 || cfg->window > kMaxWindow) FAIL("window must be in [1, 16]");
  if (!(cfg->lambda > 0.0 && cfg->lambda < 0.5)) FAIL("lambda must be in (0, 0.5)");
  if (!(cfg->max_flow >= 0.0f && cfg->max_flow <= STITCH_MAX_FLOW)) FAIL("max_flow must be in [0, 16]");
  if (cfg->ref_cam < -1 || cfg->ref_cam >= cfg->n_cams) FAIL("ref_cam out of range");
  if (cfg->flags & ~(STITCH_BALANCE_OFF | STITCH_FP16_INTERMEDIATE | STITCH_FLOW_WEIGHTS_PRINTED | STITCH_LEARNED |
                     STITCH_BALANCE_OUTPUT))
    FAIL("unknown flag");
  g.n = cfg->n_cams;
  g.pano_w = cfg->pano_w;
  g.pano_h = cfg->pano_h;
  g.pano_pitch = cfg->pano_pitch;
  g.ref = cfg->ref_cam < 0 ? cfg->n_cams / 2 : cfg->ref_cam;
  g.cyl = cfg->projection == STITCH_PROJ_CYLINDRICAL ? 1 : 0;
  if (g.cyl) {
    g.f = cfg->cyl_focal;
    g.cx = cfg->cyl_cx;
    g.cy = cfg->cyl_cy;
  }
  long long total_px = 0;
  for (int k = 0; k < g.n; ++k) {
    g.w[k] = cfg->cam_w[k];
    g.h[k] = cfg->cam_h[k];
    if (g.w[k] < 2 || g.h[k] < 2 || g.w[k] > 65535 || g.h[k] > 65535) FAIL("camera size out of range");
    g.pitch[k] = cfg->cam_pitch ? cfg->cam_pitch[k] : 3 * g.w[k];
    if (g.pitch[k] < 3 * g.w[k]) FAIL("camera pitch < 3 * width");
    total_px += (long long)g.w[k] * g.h[k];
    for (int e = 0; e < 9; ++e) {
      g.H[k][e] = cfg->H[k * 9 + e];
      if (!std::isfinite(g.H[k][e])) FAIL("homography has a non-finite entry");
    }
    if (!inv3(g.H[k], g.Hi[k])) FAIL("homography is singular");
  }
  if (total_px >= (1ll << 32)) FAIL("too many camera pixels for 32-bit histograms");
  for (int p = 0; p + 1 < g.n; ++p) {
    const int a = p, b = p + 1;
    int x0, x1, y0, y1;
    if (!g.cyl) {
      double ax[4], ay[4], bx[4], by[4];
      corners(g, a, ax, ay);
      corners(g, b, bx, by);
      x0 = ceil_snap(std::fmax(bx[0], bx[3]));
      x1 = floor_snap(std::fmin(ax[1], ax[2])) + 1;
      const double xl = x0, xr = x1 - 1;
      const double tops[4] = {line_y(ax[0], ay[0], ax[1], ay[1], xl), line_y(ax[0], ay[0], ax[1], ay[1], xr),
                              line_y(bx[0], by[0], bx[1], by[1], xl), line_y(bx[0], by[0], bx[1], by[1], xr)};
      const double bots[4] = {line_y(ax[3], ay[3], ax[2], ay[2], xl), line_y(ax[3], ay[3], ax[2], ay[2], xr),
                              line_y(bx[3], by[3], bx[2], by[2], xl), line_y(bx[3], by[3], bx[2], by[2], xr)};
      double tmax = tops[0], bmin = bots[0];
      for (int i = 1; i < 4; ++i) {
        tmax = std::fmax(tmax, tops[i]);
        bmin = std::fmin(bmin, bots[i]);
      }
      y0 = ceil_snap(tmax);
      y1 = floor_snap(bmin) + 1;
      x0 = std::max(x0, 0);
      y0 = std::max(y0, 0);
      x1 = std::min(x1, g.pano_w);
      y1 = std::min(y1, g.pano_h);
    } else {
      // Cylinder: camera edges map to curves, so the extreme columns come
      // from every pixel of b's left and a's right edge; rows from the
      // coverage of every band column by both cameras.
      double xl_max = -1e300, xr_min = 1e300;
      for (int v = 0; v < g.h[b]; ++v) {
        double X, Y;
        cam_to_pano(g, b, 0.0, (double)v, X, Y);
        xl_max = std::fmax(xl_max, X);
      }
      for (int v = 0; v < g.h[a]; ++v) {
        double X, Y;
        cam_to_pano(g, a, g.w[a] - 1.0, (double)v, X, Y);
        xr_min = std::fmin(xr_min, X);
      }
      x0 = std::max(ceil_snap(xl_max), 0);
      x1 = std::min(floor_snap(xr_min) + 1, g.pano_w);
      if (x1 - x0 < 2) FAIL("an adjacent camera pair has no overlap band");
      y0 = 0;
      y1 = g.pano_h;
      for (int x = x0; x < x1; ++x)
        for (int cam = a; cam <= b; ++cam) {
          int top = 0, bot = g.pano_h - 1;
          while (top < g.pano_h && !covered64(g, cam, x, top)) ++top;
          while (bot >= 0 && !covered64(g, cam, x, bot)) --bot;
          if (top > bot) FAIL("an adjacent camera pair has no overlap band");
          y0 = std::max(y0, top);
          y1 = std::min(y1, bot + 1);
        }
    }
    if (x1 - x0 < 2 || y1 - y0 < 2) FAIL("an adjacent camera pair has no overlap band");
    g.band[p][0] = x0;
    g.band[p][1] = x1;
    g.band[p][2] = y0;
    g.band[p][3] = y1;
    // The band must lie inside both cameras' coverage. Coverage is convex, so
    // testing the band's border pixels suffices.
    for (int cam = a; cam <= b; ++cam) {
      bool ok = true;
      for (int x = x0; x < x1 && ok; ++x) ok = covered64(g, cam, x, y0) && covered64(g, cam, x, y1 - 1);
      for (int y = y0; y < y1 && ok; ++y) ok = covered64(g, cam, x0, y) && covered64(g, cam, x1 - 1, y);
      if (!ok) FAIL("overlap band is not covered by both cameras (homographies too far from a left-to-right rig)");
    }
    for (int side = 0; side < 2; ++side) {
      const int cam = side == 0 ? a : b;
      int rx0, rx1, ry0, ry1;
      if (!g.cyl) {
        const double px[4] = {(double)x0, (double)(x1 - 1), (double)(x1 - 1), (double)x0};
        const double py[4] = {(double)y0, (double)y0, (double)(y1 - 1), (double)(y1 - 1)};
        double sx[4], sy[4];
        for (int i = 0; i < 4; ++i) {
          double W;
          proj(g.Hi[cam], px[i], py[i], sx[i], sy[i], W);
        }
        rx0 = ceil_snap(std::fmax(sx[0], sx[3]));
        rx1 = floor_snap(std::fmin(sx[1], sx[2])) + 1;
        ry0 = ceil_snap(std::fmax(sy[0], sy[1]));
        ry1 = floor_snap(std::fmin(sy[2], sy[3])) + 1;
      } else {
        // every pixel of the band's border: left / right columns, top / bottom rows
        double l = -1e300, r = 1e300, t = -1e300, bo = 1e300, sx, sy, sw;
        for (int y = y0; y < y1; ++y) {
          pano_to_cam(g, cam, x0, y, sx, sy, sw);
          l = std::fmax(l, sx);
          pano_to_cam(g, cam, x1 - 1, y, sx, sy, sw);
          r = std::fmin(r, sx);
        }
        for (int x = x0; x < x1; ++x) {
          pano_to_cam(g, cam, x, y0, sx, sy, sw);
          t = std::fmax(t, sy);
          pano_to_cam(g, cam, x, y1 - 1, sx, sy, sw);
          bo = std::fmin(bo, sy);
        }
        rx0 = ceil_snap(l);
        rx1 = floor_snap(r) + 1;
        ry0 = ceil_snap(t);
        ry1 = floor_snap(bo) + 1;
      }
      rx0 = std::max(rx0, 0);
      ry0 = std::max(ry0, 0);
      rx1 = std::min(rx1, g.w[cam]);
      ry1 = std::min(ry1, g.h[cam]);
      if (rx1 <= rx0 || ry1 <= ry0) rx0 = rx1 = ry0 = ry1 = 0;
      if ((long long)(rx1 - rx0) * (ry1 - ry0) * 255ll >= (1ll << 32)) FAIL("overlap too large for 32-bit sums");
      g.rect[p][side][0] = rx0;
      g.rect[p][side][1] = rx1;
      g.rect[p][side][2] = ry0;
      g.rect[p][side][3] = ry1;
    }
    if (p + 1 <= g.ref) {
      g.pair_i[p] = p;
      g.pair_j[p] = p + 1;
    } else {
      g.pair_i[p] = p + 1;
      g.pair_j[p] = p;
    }
  }
  for (int p = 0; p + 2 < g.n; ++p)
    if (g.band[p][1] > g.band[p + 1][0]) FAIL("overlap bands of successive pairs intersect");
  for (int k = 0; k < g.n; ++k) {
    g.own_lo[k] = k == 0 ? 0 : g.band[k - 1][1];
    g.own_hi[k] = k == g.n - 1 ? g.pano_w : g.band[k][0];
  }
  return STITCH_OK;
}

#undef FAIL

void export_geometry(const Geo &g, int *bands, int *rects) {
  for (int p = 0; p + 1 < g.n; ++p) {
    if (bands)
      for (int e = 0; e < 4; ++e) bands[p * 4 + e] = g.band[p][e];
    if (rects)
      for (int s = 0; s < 2; ++s)
        for (int e = 0; e < 4; ++e) rects[p * 8 + s * 4 + e] = g.rect[p][s][e];
  }
}

}  // namespace

// A pair of events bracketing one stage launch: 0 = stats, 1 = estimate, 2 = fuse, 3 = band pre-warp.
struct ProfPair {
  cudaEvent_t a, b;
  int stage;
};

namespace stitch {

// Launch parameters of the estimate stage (statistics + estimate) for a
// configuration, computed on the host only. Allocates no device memory; the
// caller fills in the frame pointers, the raw-statistics slots and the state.
int prepare_estimate_params(const stitch_config *cfg, StatsParams &sp, int &grid_x, EstimateParams &ep,
                            std::string &err) {
  Geo g;
  const int rc = build_geometry(cfg, g, err);
  if (rc != STITCH_OK) return rc;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long rows = 0;
  int max_h = 0;
  for (int k = 0; k < g.n; ++k) {
    rows += g.h[k];
    max_h = std::max(max_h, g.h[k]);
  }
  // about two statistics blocks per SM: the per-block clearing and flushing
  // of the shared histograms is then a small share of the work
  const int rpb = (int)std::max(1ll, (rows + 2ll * sms - 1) / (2ll * sms));
  sp = StatsParams{};
  sp.n_cams = g.n;
  sp.rows_per_block = rpb;
  for (int k = 0; k < g.n; ++k) {
    sp.w[k] = g.w[k];
    sp.h[k] = g.h[k];
    sp.pitch[k] = g.pitch[k];
  }
  for (int p = 0; p + 1 < g.n; ++p) {
    for (int side = 0; side < 2; ++side) {
      const int cam = side == 0 ? p : p + 1;
      RoleDev r{};
      r.rx0 = g.rect[p][side][0];
      r.rx1 = g.rect[p][side][1];
      r.ry0 = g.rect[p][side][2];
      r.ry1 = g.rect[p][side][3];
      r.pair = p;
      r.is_i = (g.pair_i[p] == cam) ? 1 : 0;
      sp.roles[cam][sp.n_roles[cam]++] = r;
    }
  }
  grid_x = (max_h + rpb - 1) / rpb;
  ep = EstimateParams{};
  ep.n_cams = g.n;
  ep.n_pairs = g.n - 1;
  ep.ref = g.ref;
  ep.window = 1;
  ep.lambda_q = (long long)std::llround(cfg->lambda * 1e6);
  if (ep.lambda_q <= 0 || ep.lambda_q >= 500000) {
    err = "lambda rounds to 0 or 0.5 in millionths";
    return STITCH_EINVAL;
  }
  for (int p = 0; p + 1 < g.n; ++p) {
    ep.pair_i[p] = g.pair_i[p];
    ep.pair_j[p] = g.pair_j[p];
  }
  return STITCH_OK;
}

void record_last_error(const std::string &msg) { g_last_error = msg; }

}  // namespace stitch

struct GraphEntry {
  std::vector<const void *> key;
  int n_frames = 0;
  int parity = 0;
  bool prof = false;
  cudaGraphExec_t exec = nullptr;
  std::vector<ProfPair> pairs;        // events owned by this graph (profiling only)
};

// One slot of the host-memory sequence path: device copies of a frame's
// images and flows and of its panorama, with the events that order the copy
// streams against the compute stream.
struct HostStage {
  uint8_t *frames[kMaxCams] = {};
  float *fij[kMaxPairs] = {};
  float *fji[kMaxPairs] = {};
  uint8_t *pano = nullptr;
  cudaEvent_t in_ready = nullptr;     // inputs copied
  cudaEvent_t computed = nullptr;     // frame computed: inputs free, panorama ready
  cudaEvent_t out_done = nullptr;     // panorama copied out: panorama buffer free
};

// Streams of a recorded sequence: statistics, estimate, band pre-warp, and
// two fuse streams taking alternate frames.
constexpr int kPipeStreams = 5;

struct stitch_ctx {
  Geo g;
  int flags = 0;
  int window = 3;
  long long lambda_q = 50000;
  float max_flow = 0.0f;
  int halo = 1;
  int device = 0;
  int host_T = 0;                     // frames estimated (host mirror of the device index)
  int host_F = 0;                     // frames fused (selects the band pre-warp slot)
  size_t pw_slot_bytes = 0;
  std::string err;
  RawStats *raw = nullptr;            // kRawSlots slots
  ColorState *state = nullptr;
  TileDesc *tiles = nullptr;
  PwTile *pw_tiles = nullptr;
  void *pw = nullptr;                 // band pre-warp intermediate
  uint8_t *lut = nullptr;             // output tables of the colour slots (kColorSlots x kLutBytes)
  uint32_t *out_hist = nullptr;       // STITCH_BALANCE_OUTPUT: pre-balance histograms, frame F in slot F % 2
  unsigned int *win_fallback = nullptr;   // fuse tiles whose source window did not fit (counter)
  int stats_grid_x = 1;
  StatsParams sp{};
  EstimateParams ep{};
  FuseParams fp{};
  cudaStream_t cap_stream = nullptr;
  cudaStream_t net_stream = nullptr;  // learned contexts: the network beside the plain estimate
  cudaEvent_t net_ev[2] = {};         // fork (statistics done) and join (network done)
  cudaStream_t pipe[kPipeStreams] = {};   // statistics, estimate, band pre-warp and two fuse streams of a
                                          // recorded sequence
  cudaEvent_t pev[4][8] = {};         // per-stage completion events (stats, pre-warp, estimate, fuse) by t % 8
  std::vector<GraphEntry> graphs;
  bool prof = false;                  // record stage events (stitch_profile)
  std::vector<ProfPair> *prof_sink = nullptr;   // where new pairs go (a graph while capturing)
  std::vector<ProfPair> pending;      // pairs whose times the next stitch_profile_read sums
  std::vector<ProfPair> owned;        // per-call pairs, destroyed after they are read
  HostStage stage[2];                 // device staging of stitch_sequence_host, two frames in flight
  float4 *flow_pw = nullptr;          // stitch_estimate_flow: float32 pre-warped bands
  uint8_t *flow_Y = nullptr;          // its luminance pyramids
  int16_t *flow_d = nullptr;          // its chosen displacements (dx then dy)
  FlowParams flow_fl{};               // the latest stitch_estimate_flow's level sizes and offsets
  bool flow_ready = false;            // (for stitch_get_flow_luma)
  RefineState *refine_state = nullptr;  // stitch_refine_homographies: radix-selection state
  uint32_t *refine_hist = nullptr;      // and histograms (8 medians per pair)
  double *corr_buf = nullptr;         // stitch_pair_M_correspondence: block partials, then the totals
  cudaStream_t copy_in = nullptr;     // host-to-device copies of stitch_sequence_host
  cudaStream_t copy_out = nullptr;    // device-to-host copies of stitch_sequence_host
  int shape = 0;                      // fuse tile shape (index into kTileShapes)
  LearnedState *ls = nullptr;         // learned estimator state (STITCH_LEARNED contexts)
  stitch_mlp *mlp = nullptr;          // attached network (not owned)
};

namespace {

int set_err(stitch_ctx *ctx, int code, const std::string &msg) {
  if (ctx)
    ctx->err = msg;
  else
    g_last_error = msg;
  return code;
}

int cuda_err(stitch_ctx *ctx, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return set_err(ctx, e == cudaErrorMemoryAllocation ? STITCH_ENOMEM : STITCH_ECUDA, m);
}

size_t band_elems(const Geo &g, int p) {
  return (size_t)(g.band[p][1] - g.band[p][0]) * (size_t)(g.band[p][3] - g.band[p][2]);
}

// Profiling: record an event on `s` and return it (nullptr when off).
cudaEvent_t prof_mark(stitch_ctx *ctx, cudaStream_t s) {
  if (!ctx->prof) return nullptr;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  // Inside stream capture a plain record only forms a dependency; the external
  // flag makes it an event node that records (with a timestamp) on every replay.
  const unsigned flags = ctx->prof_sink ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (cudaEventRecordWithFlags(e, s, flags) != cudaSuccess) {
    cudaEventDestroy(e);
    return nullptr;
  }
  return e;
}

void prof_pair(stitch_ctx *ctx, cudaEvent_t a, cudaEvent_t b, int stage) {
  if (!a || !b) {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return;
  }
  ProfPair pp{a, b, stage};
  if (ctx->prof_sink) {
    ctx->prof_sink->push_back(pp);
  } else {
    ctx->pending.push_back(pp);
    ctx->owned.push_back(pp);
  }
}

// Statistics of frame T into slot T % kRawSlots (cleared by the estimate of frame T - 2).
int launch_stats_for(stitch_ctx *ctx, const uint8_t *const *frames, int T, cudaStream_t s) {
  StatsParams sp = ctx->sp;
  for (int k = 0; k < ctx->g.n; ++k) {
    sp.src[k] = frames[k];
    sp.vec_ok[k] = ((reinterpret_cast<uintptr_t>(frames[k]) & 15u) == 0 && ctx->g.pitch[k] % 16 == 0) ? 1 : 0;
  }
  sp.raw = ctx->raw + (T % kRawSlots);
  // Every timing pair owns its two events (they are destroyed pairwise).
  cudaEvent_t e0 = prof_mark(ctx, s);
  cudaError_t e = launch_stats(sp, ctx->stats_grid_x, s);
  if (e != cudaSuccess) return cuda_err(ctx, e, "stats launch");
  cudaEvent_t e1 = prof_mark(ctx, s);
  prof_pair(ctx, e0, e1, 0);
  return STITCH_OK;
}

int launch_estimate_for(stitch_ctx *ctx, cudaStream_t s) {
  cudaEvent_t e0 = prof_mark(ctx, s);
  cudaError_t e = cudaSuccess;
  if (ctx->mlp && ctx->ls && ctx->g.n > 1) {
    // Learned estimate of frame T: the features and the network read only
    // the statistics, so they run on their own stream beside the plain
    // estimate; the residual test and re-chain join both.
    LearnedParams lp{};
    lp.n_cams = ctx->g.n;
    lp.n_pairs = ctx->g.n - 1;
    lp.ref = ctx->g.ref;
    lp.window = ctx->window;
    lp.raw_slots = kRawSlots;
    lp.raw = ctx->raw;
    lp.state = ctx->state;
    lp.ls = ctx->ls;
    cudaStream_t n = ctx->net_stream;
    e = cudaEventRecord(ctx->net_ev[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(n, ctx->net_ev[0], 0);
    if (e == cudaSuccess) e = launch_learned_features(lp, n);
    if (e != cudaSuccess) return cuda_err(ctx, e, "learned features launch");
    const int rc = stitch_mlp_forward(ctx->mlp, reinterpret_cast<const uint16_t *>(&ctx->ls->feat[0][0]), lp.n_pairs,
                                      &ctx->ls->y[0][0], reinterpret_cast<stitch_stream_t>(n));
    if (rc != STITCH_OK) return set_err(ctx, rc, std::string("network forward: ") + g_last_error);
    e = cudaEventRecord(ctx->net_ev[1], n);
    if (e == cudaSuccess) e = launch_estimate(ctx->ep, s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "estimate launch");
    e = cudaStreamWaitEvent(s, ctx->net_ev[1], 0);
    if (e == cudaSuccess) e = launch_learned_select(lp, s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "learned select launch");
  } else {
    e = launch_estimate(ctx->ep, s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "estimate launch");
  }
  cudaEvent_t e1 = prof_mark(ctx, s);
  prof_pair(ctx, e0, e1, 1);
  return STITCH_OK;
}

FuseParams frame_params(stitch_ctx *ctx, const uint8_t *const *frames, const float *const *fij,
                        const float *const *fji, uint8_t *pano, int colour_T, int F) {
  FuseParams fp = ctx->fp;
  for (int k = 0; k < ctx->g.n; ++k) fp.src[k] = frames[k];
  for (int p = 0; p + 1 < ctx->g.n; ++p) {
    fp.flow_ij[p] = reinterpret_cast<const float2 *>(fij[p]);
    fp.flow_ji[p] = reinterpret_cast<const float2 *>(fji[p]);
  }
  fp.out = pano;
  const int slot = ((colour_T % kColorSlots) + kColorSlots) % kColorSlots;
  fp.color = &ctx->state->out[slot];
  fp.lut = ctx->lut + (size_t)slot * kLutBytes;
  fp.win_fallback = ctx->win_fallback;
  fp.out_hist = ctx->out_hist ? ctx->out_hist + (size_t)(F % 2) * 768 : nullptr;
  fp.flags |= kFlagPwOffset;
  fp.pw = static_cast<char *>(ctx->pw) + (size_t)(F % kPwSlots) * ctx->pw_slot_bytes;
  return fp;
}

// Band pre-warp (stage 3) and fuse (stage 2) of one frame.
int launch_prewarp_for(stitch_ctx *ctx, const FuseParams &fp, cudaStream_t s) {
  cudaEvent_t e0 = prof_mark(ctx, s);
  cudaError_t e = launch_prewarp(fp, s);
  if (e != cudaSuccess) return cuda_err(ctx, e, "band pre-warp launch");
  cudaEvent_t e1 = prof_mark(ctx, s);
  prof_pair(ctx, e0, e1, 3);
  return STITCH_OK;
}

int launch_fuse_for(stitch_ctx *ctx, const FuseParams &fp, cudaStream_t s) {
  cudaEvent_t e0 = prof_mark(ctx, s);
  cudaError_t e = launch_fuse(fp, ctx->shape, s);
  if (e != cudaSuccess) return cuda_err(ctx, e, "fuse launch");
  cudaEvent_t e1 = prof_mark(ctx, s);
  prof_pair(ctx, e0, e1, 2);
  return STITCH_OK;
}

int launch_estimate_color(stitch_ctx *ctx, const uint8_t *const *frames, cudaStream_t s) {
  int rc = launch_stats_for(ctx, frames, ctx->host_T, s);
  if (rc == STITCH_OK) rc = launch_estimate_for(ctx, s);
  if (rc == STITCH_OK) ctx->host_T += 1;
  return rc;
}

int launch_frame(stitch_ctx *ctx, const uint8_t *const *frames, const float *const *fij, const float *const *fji,
                 uint8_t *pano, cudaStream_t s) {
  // colour of the latest estimate, frame host_T - 1
  const FuseParams fp = frame_params(ctx, frames, fij, fji, pano, ctx->host_T - 1, ctx->host_F);
  int rc = launch_prewarp_for(ctx, fp, s);
  if (rc == STITCH_OK) rc = launch_fuse_for(ctx, fp, s);
  if (rc == STITCH_OK) ctx->host_F += 1;
  return rc;
}

bool check_ptrs(const void *const *p, int n) {
  if (!p) return false;
  for (int i = 0; i < n; ++i)
    if (!p[i]) return false;
  return true;
}

// Fuse tile pieces of one shape. A tile is cut at 16-column boundaries into
// pieces of one kind each: the chunks of the band rectangle's columns
// (kTileBand, when the tile's rows lie inside the band rectangle), the chunk
// holding a band edge and band columns outside the band rows (kTileBandPart),
// and own columns of one camera, kTileOwn when that camera covers every
// pixel of the piece with a margin (coverage is convex on the plane, so the
// corners decide; on the cylinder every border pixel is tested), else
// kTileOwnPart. The list holds the general pieces first (the partly covered
// own pieces, then the band-edge pieces), then the band pieces and the fully
// covered own pieces. Returns false (with a message) when a tile would touch two bands.
struct TileCounts {
  int n_band = 0, n_full = 0;
};

void set_counts(FuseParams &fp, const TileCounts &c) {
  fp.n_band = c.n_band;
  fp.n_full = c.n_full;
}

bool build_tiles(const Geo &g, int shape, std::vector<TileDesc> &tiles, TileCounts &cnt, std::string &err) {
  const int TW = kTileShapes[shape].w, TH = kTileShapes[shape].h;
  const int ntx = (g.pano_w + TW - 1) / TW, nty = (g.pano_h + TH - 1) / TH;
  if (ntx > 32767 || nty > 32767) {
    err = "panorama too large for the tile index";
    return false;
  }
  std::vector<TileDesc> gen, bpart, band, full;
  auto own_piece = [&](int k, int tx, int ty, int x0, int x1) {
    // columns [x0, x1) of tile (tx, ty), owned by camera k
    if (x0 >= x1) return;
    const int r0 = ty * TH, r1 = std::min(r0 + TH, g.pano_h) - 1;
    auto inside = [&](int x, int y) {
      double sx, sy, sw;
      pano_to_cam(g, k, x, y, sx, sy, sw);
      return sw > 0 && sx >= 0.01 && sx <= g.w[k] - 1.01 && sy >= 0.01 && sy <= g.h[k] - 1.01;
    };
    bool ok = x1 <= g.pano_w && r0 + TH <= g.pano_h;
    if (!g.cyl) {
      ok = ok && inside(x0, r0) && inside(x1 - 1, r0) && inside(x0, r1) && inside(x1 - 1, r1);
    } else {
      for (int x = x0; x < x1 && ok; ++x) ok = inside(x, r0) && inside(x, r1);
      for (int y = r0; y <= r1 && ok; ++y) ok = inside(x0, y) && inside(x1 - 1, y);
    }
    TileDesc t{};
    t.tx = (int16_t)tx;
    t.ty = (int16_t)ty;
    t.kind = (int8_t)(ok ? kTileOwn : kTileOwnPart);
    t.idx = (int8_t)k;
    t.c0 = (uint8_t)((x0 - tx * TW) / 16);
    t.c1 = (uint8_t)((x1 - tx * TW + 15) / 16);
    (ok ? full : gen).push_back(t);
  };
  auto band_piece = [&](int p, int kind, int tx, int ty, int x0, int x1) {
    if (x0 >= x1) return;
    TileDesc t{};
    t.tx = (int16_t)tx;
    t.ty = (int16_t)ty;
    t.kind = (int8_t)kind;
    t.idx = (int8_t)p;
    t.c0 = (uint8_t)((x0 - tx * TW) / 16);
    t.c1 = (uint8_t)((x1 - tx * TW + 15) / 16);
    (kind == kTileBand ? band : bpart).push_back(t);
  };
  for (int ty = 0; ty < nty; ++ty) {
    for (int tx = 0; tx < ntx; ++tx) {
      const int c0 = tx * TW, c1 = std::min(c0 + TW, g.pano_pitch);
      int hit = -1, nhit = 0;
      for (int p = 0; p + 1 < g.n; ++p)
        if (c0 < g.band[p][1] && c1 > g.band[p][0]) {
          hit = p;
          ++nhit;
        }
      if (nhit > 1) {
        err = "a camera's own columns are narrower than a fuse tile (" + std::to_string(TW) + " pixels)";
        return false;
      }
      if (hit < 0) {
        int k = 0;
        while (k < g.n - 1 && c0 >= g.own_hi[k]) ++k;
        own_piece(k, tx, ty, c0, c1);
        continue;
      }
      const int p = hit;
      const int bx0 = g.band[p][0], bx1 = g.band[p][1];
      const int a = bx0 & ~15, b = (bx0 + 15) & ~15;     // chunk holding the left band edge: [a, b)
      const int a2 = bx1 & ~15, b2 = (bx1 + 15) & ~15;   // chunk holding the right band edge: [a2, b2)
      // every row of the tile, also past a partial last tile row, inside the band rectangle
      const int r0 = ty * TH;
      const bool rows_in = r0 >= g.band[p][2] && r0 + TH <= g.band[p][3];
      auto clip0 = [&](int v) { return std::min(std::max(v, c0), c1); };
      own_piece(p, tx, ty, c0, clip0(a));
      own_piece(p + 1, tx, ty, clip0(b2), c1);
      if (b <= a2) {
        band_piece(p, kTileBandPart, tx, ty, clip0(a), clip0(b));
        band_piece(p, rows_in ? kTileBand : kTileBandPart, tx, ty, clip0(b), clip0(a2));
        band_piece(p, kTileBandPart, tx, ty, clip0(a2), clip0(b2));
      } else {
        band_piece(p, kTileBandPart, tx, ty, clip0(a), clip0(b2));
      }
    }
  }
  cnt.n_band = (int)band.size();
  cnt.n_full = (int)full.size();
  tiles = gen;
  tiles.insert(tiles.end(), bpart.begin(), bpart.end());
  tiles.insert(tiles.end(), band.begin(), band.end());
  tiles.insert(tiles.end(), full.begin(), full.end());
  return true;
}

// Pieces of the smallest shape (at least 32 x 16, at most five pieces per
// tile): room for any shape's list.
size_t max_tiles(const Geo &g) { return 5 * (size_t)((g.pano_w + 31) / 32) * (size_t)((g.pano_h + 15) / 16); }

// A tile shape replaces the default one only when it is faster by more than
// this factor.
constexpr float kTuneMargin = 0.95f;

// ---------------------------------------------------------------------------
// Autotuner results: the fastest fuse tile shape per (GPU, rig geometry,
// intermediate precision), kept for the process and, when STITCH_TUNE_CACHE
// names a file, in that file (one "key<TAB>shape" line per result; the last
// line of a key wins).
// ---------------------------------------------------------------------------
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_file_read = false;

// Cache key of a rig's tuned fuse tile shape: device, cameras, panorama,
// bands, intermediate precision, and whether the rig runs alone or inside a
// batched persistent launch (tuned separately).
std::string tune_key(const Geo &g, int flags, bool batched = false) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop{};
  std::string name = "unknown";
  int sms = 0;
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
    name = prop.name;
    sms = prop.multiProcessorCount;
  }
  for (char &c : name)
    if (c == '\t' || c == '\n') c = ' ';
  std::ostringstream k;
  k << name << "/" << sms << "sm|" << g.n;
  for (int i = 0; i < g.n; ++i) k << ":" << g.w[i] << "x" << g.h[i];
  k << "|" << g.pano_w << "x" << g.pano_h << "|";
  for (int p = 0; p + 1 < g.n; ++p) k << (g.band[p][1] - g.band[p][0]) << "x" << (g.band[p][3] - g.band[p][2]) << ",";
  k << "|fp16=" << ((flags & STITCH_FP16_INTERMEDIATE) ? 1 : 0);
  if (batched) k << "|batched";
  return k.str();
}

void tune_file_read_locked() {
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char *path = std::getenv("STITCH_TUNE_CACHE");
  if (!path || !*path) return;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t tab = line.rfind('\t');
    if (tab == std::string::npos) continue;
    const int shape = std::atoi(line.c_str() + tab + 1);
    if (shape >= 0 && shape < kNumTileShapes) g_tune[line.substr(0, tab)] = shape;
  }
}

int tuned_shape(const Geo &g, int flags, bool batched = false, int fallback = 0) {
  const std::string key = tune_key(g, flags, batched);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_file_read_locked();
  const auto it = g_tune.find(key);
  return it == g_tune.end() ? fallback : it->second;
}

void tune_record(const Geo &g, int flags, int shape, bool batched = false) {
  const std::string key = tune_key(g, flags, batched);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_file_read_locked();
  g_tune[key] = shape;
  const char *path = std::getenv("STITCH_TUNE_CACHE");
  if (path && *path) {
    std::ofstream f(path, std::ios::app);
    if (f) f << key << '\t' << shape << '\n';
  }
}

}  // namespace

extern "C" {

int stitch_geometry(const stitch_config *cfg, int *bands, int *rects) {
  Geo g;
  std::string err;
  const int rc = build_geometry(cfg, g, err);
  if (rc != STITCH_OK) return set_err(nullptr, rc, err);
  export_geometry(g, bands, rects);
  return STITCH_OK;
}

int stitch_init(const stitch_config *cfg, stitch_ctx **out) {
  if (!out) return set_err(nullptr, STITCH_EINVAL, "out is NULL");
  *out = nullptr;
  stitch_ctx *ctx = new (std::nothrow) stitch_ctx();
  if (!ctx) return set_err(nullptr, STITCH_ENOMEM, "host allocation failed");
  std::string err;
  int rc = build_geometry(cfg, ctx->g, err);
  if (rc != STITCH_OK) {
    delete ctx;
    return set_err(nullptr, rc, err);
  }
  const Geo &g = ctx->g;
  ctx->flags = cfg->flags;
  ctx->window = cfg->window;
  ctx->lambda_q = (long long)std::llround(cfg->lambda * 1e6);
  if (ctx->lambda_q <= 0 || ctx->lambda_q >= 500000) {
    delete ctx;
    return set_err(nullptr, STITCH_EINVAL, "lambda rounds to 0 or 0.5 in millionths");
  }
  ctx->max_flow = cfg->max_flow;
  ctx->halo = (int)std::ceil((double)cfg->max_flow) + 1;

  ctx->shape = tuned_shape(g, cfg->flags);
  std::vector<TileDesc> tiles;
  TileCounts tcnt;
  if (!build_tiles(g, ctx->shape, tiles, tcnt, err)) {
    if (ctx->shape != 0) {
      ctx->shape = 0;
      tiles.clear();
    }
    if (ctx->shape != 0 || !build_tiles(g, 0, tiles, tcnt, err)) {
      delete ctx;
      return set_err(nullptr, STITCH_EINVAL, err);
    }
  }

  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = estimate_setup();
  if (e == cudaSuccess) e = fuse_setup_attributes(0);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->raw, kRawSlots * sizeof(RawStats));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->lut, (size_t)kColorSlots * kLutBytes);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->win_fallback, sizeof(unsigned int));
  if (e == cudaSuccess && (cfg->flags & STITCH_BALANCE_OUTPUT)) {
    e = cudaMalloc(&ctx->out_hist, 2 * 768 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(ctx->out_hist, 0, 2 * 768 * sizeof(uint32_t));
  }
  if (e == cudaSuccess) e = cudaMemset(ctx->win_fallback, 0, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->state, sizeof(ColorState));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->tiles, max_tiles(g) * sizeof(TileDesc) + 16);
  if (e == cudaSuccess) e = cudaMemset(ctx->raw, 0, kRawSlots * sizeof(RawStats));
  if (e == cudaSuccess && (cfg->flags & STITCH_LEARNED)) {
    e = cudaMalloc(&ctx->ls, sizeof(LearnedState));
    if (e == cudaSuccess) e = cudaMemset(ctx->ls, 0, sizeof(LearnedState));
  }
  // Band pre-warp pieces and the intermediate (both cameras of every band).
  std::vector<PwTile> pw_tiles;
  size_t pw_elems = 0;
  size_t pw_off[kMaxPairs][2] = {};
  for (int p = 0; p + 1 < g.n; ++p) {
    const int x0 = g.band[p][0], x1 = g.band[p][1], y0 = g.band[p][2], y1 = g.band[p][3];
    for (int y = y0; y < y1; y += kTileH)
      for (int x = x0; x < x1; x += kTileW) pw_tiles.push_back(PwTile{p, x, y});
    const size_t area = (size_t)(x1 - x0) * (size_t)(y1 - y0);
    pw_off[p][0] = pw_elems;
    pw_off[p][1] = pw_elems + area;
    pw_elems += 2 * area;
  }
  const size_t pw_bytes = pw_elems * prewarp_elem_bytes(true);   // the frame path keeps halves
  if (e == cudaSuccess) e = cudaMalloc(&ctx->pw_tiles, pw_tiles.size() * sizeof(PwTile) + 16);
  ctx->pw_slot_bytes = (pw_bytes + 255) / 256 * 256;
  if (e == cudaSuccess) e = cudaMalloc(&ctx->pw, kPwSlots * ctx->pw_slot_bytes + 16);
  if (e == cudaSuccess && !pw_tiles.empty())
    e = cudaMemcpy(ctx->pw_tiles, pw_tiles.data(), pw_tiles.size() * sizeof(PwTile), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !tiles.empty())
    e = cudaMemcpy(ctx->tiles, tiles.data(), tiles.size() * sizeof(TileDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    ColorState *h = new ColorState();
    std::memset(h, 0, sizeof(ColorState));
    for (int p = 0; p < kMaxPairs; ++p)
      for (int k = 0; k < 9; ++k) h->M_pair[p][k] = (k % 4 == 0) ? 1.0 : 0.0;
    for (int c = 0; c < kMaxCams; ++c)
      for (int k = 0; k < 9; ++k) {
        h->M_cam[c][k] = (k % 4 == 0) ? 1.0 : 0.0;
        for (int s = 0; s < kColorSlots; ++s) h->out[s].M[c][k] = (k % 4 == 0) ? 1.0f : 0.0f;
      }
    for (int s = 0; s < kColorSlots; ++s)
      for (int c = 0; c < 3; ++c) h->out[s].curve[c].ident = 1.0f;
    e = cudaMemcpy(ctx->state, h, sizeof(ColorState), cudaMemcpyHostToDevice);
    delete h;
    // the identity curve's output table in every colour slot
    for (int sl = 0; sl < kColorSlots && e == cudaSuccess; ++sl)
      e = launch_curve_lut(&ctx->state->out[sl], cfg->flags, ctx->lut + (size_t)sl * kLutBytes, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
  for (int i = 0; i < kPipeStreams && e == cudaSuccess; ++i)
    e = cudaStreamCreateWithFlags(&ctx->pipe[i], cudaStreamNonBlocking);
  for (int a = 0; a < 4 && e == cudaSuccess; ++a)
    for (int b = 0; b < 8 && e == cudaSuccess; ++b) e = cudaEventCreateWithFlags(&ctx->pev[a][b], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->net_stream, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ctx->net_ev[k], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    const int code = cuda_err(nullptr, e, "stitch_init");
    stitch_destroy(ctx);
    return code;
  }

  // Stats launch geometry: about four blocks per SM over all camera rows.
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  long long rows = 0;
  int max_h = 0;
  for (int k = 0; k < g.n; ++k) {
    rows += g.h[k];
    max_h = std::max(max_h, g.h[k]);
  }
  // about two statistics blocks per SM: the per-block clearing and flushing
  // of the shared histograms is then a small share of the work
  const int rpb = (int)std::max(1ll, (rows + 2ll * sms - 1) / (2ll * sms));
  StatsParams &sp = ctx->sp;
  sp = StatsParams{};
  sp.n_cams = g.n;
  sp.rows_per_block = rpb;
  sp.raw = ctx->raw;
  for (int k = 0; k < g.n; ++k) {
    sp.w[k] = g.w[k];
    sp.h[k] = g.h[k];
    sp.pitch[k] = g.pitch[k];
    sp.n_roles[k] = 0;
  }
  for (int p = 0; p + 1 < g.n; ++p) {
    for (int side = 0; side < 2; ++side) {
      const int cam = side == 0 ? p : p + 1;
      RoleDev r{};
      r.rx0 = g.rect[p][side][0];
      r.rx1 = g.rect[p][side][1];
      r.ry0 = g.rect[p][side][2];
      r.ry1 = g.rect[p][side][3];
      r.pair = p;
      r.is_i = (g.pair_i[p] == cam) ? 1 : 0;
      sp.roles[cam][sp.n_roles[cam]++] = r;
    }
  }
  ctx->stats_grid_x = (max_h + rpb - 1) / rpb;

  EstimateParams &ep = ctx->ep;
  ep = EstimateParams{};
  ep.n_cams = g.n;
  ep.n_pairs = g.n - 1;
  ep.ref = g.ref;
  ep.window = ctx->window;
  ep.lambda_q = ctx->lambda_q;
  for (int p = 0; p + 1 < g.n; ++p) {
    ep.pair_i[p] = g.pair_i[p];
    ep.pair_j[p] = g.pair_j[p];
  }
  ep.raw = ctx->raw;
  ep.raw_slots = kRawSlots;
  ep.state = ctx->state;
  ep.flags = ctx->flags;
  ep.lut = ctx->lut;
  ep.out_hist = ctx->out_hist;

  FuseParams &fp = ctx->fp;
  fp = FuseParams{};
  fp.n_cams = g.n;
  fp.flags = ctx->flags;
  fp.pano_w = g.pano_w;
  fp.pano_h = g.pano_h;
  fp.pano_pitch = g.pano_pitch;
  fp.halo = ctx->halo;
  fp.max_flow = ctx->max_flow;
  fp.n_tiles = (int)tiles.size();
  set_counts(fp, tcnt);
  fp.tiles = ctx->tiles;
  fp.n_pw_tiles = (int)pw_tiles.size();
  fp.pw_tiles = ctx->pw_tiles;
  fp.pw = ctx->pw;
  for (int p = 0; p < kMaxPairs; ++p) {
    fp.pw_off[p][0] = pw_off[p][0];
    fp.pw_off[p][1] = pw_off[p][1];
  }
  for (int k = 0; k < g.n; ++k) {
    CamDev &c = fp.cam[k];
    if (!g.cyl) {
      double cx, cy, cw;
      proj(g.H[k], (g.w[k] - 1) * 0.5, (g.h[k] - 1) * 0.5, cx, cy, cw);
      c.ox = (int)std::lround(cx);
      c.oy = (int)std::lround(cy);
      // H^-1 . T(ox, oy): the kernel feeds (x - ox, y - oy, 1).
      double hs[9];
      for (int r = 0; r < 3; ++r) {
        hs[r * 3 + 0] = g.Hi[k][r * 3 + 0];
        hs[r * 3 + 1] = g.Hi[k][r * 3 + 1];
        hs[r * 3 + 2] = g.Hi[k][r * 3 + 0] * c.ox + g.Hi[k][r * 3 + 1] * c.oy + g.Hi[k][r * 3 + 2];
      }
      const double sc = 1.0 / hs[8];
      for (int e2 = 0; e2 < 9; ++e2) c.h[e2] = (float)(hs[e2] * sc);
      for (int e2 = 0; e2 < 9; ++e2) c.hm[e2] = (float)((hs[e2] - (e2 < 6 ? 0.5 * hs[6 + e2 % 3] : 0.0)) * sc);
      c.affine = (hs[6] == 0.0 && hs[7] == 0.0) ? 1 : 0;
      c.cyl = 0;
    } else {
      // The kernel feeds the ray (sin theta, h, cos theta) of panorama (x, y);
      // H^-1 is scaled by the norm of its last row (a positive factor keeps
      // the sign of w, which tells front from back).
      c.ox = c.oy = 0;
      const double *A = g.Hi[k];
      const double sc = 1.0 / std::sqrt(A[6] * A[6] + A[7] * A[7] + A[8] * A[8]);
      for (int e2 = 0; e2 < 9; ++e2) c.h[e2] = (float)(A[e2] * sc);
      for (int e2 = 0; e2 < 9; ++e2) c.hm[e2] = (float)((A[e2] - (e2 < 6 ? 0.5 * A[6 + e2 % 3] : 0.0)) * sc);
      c.affine = 0;
      c.cyl = 1;
      c.cyl_finv = (float)(1.0 / g.f);
      c.cyl_cx = (float)g.cx;
      c.cyl_cy = (float)g.cy;
    }
    c.w = g.w[k];
    c.h_px = g.h[k];
    c.pitch = g.pitch[k];
    c.wm1 = (float)(g.w[k] - 1);
    c.hm1 = (float)(g.h[k] - 1);
    c.own_lo = g.own_lo[k];
    c.own_hi = g.own_hi[k];
  }
  for (int p = 0; p + 1 < g.n; ++p) {
    BandDev &b = fp.band[p];
    b.x0 = g.band[p][0];
    b.x1 = g.band[p][1];
    b.y0 = g.band[p][2];
    b.y1 = g.band[p][3];
    b.inv_bw = (float)(1.0 / (double)(b.x1 - b.x0));
  }
  *out = ctx;
  return STITCH_OK;
}

int stitch_estimate_color(stitch_ctx *ctx, const uint8_t *const *frames_dev, stitch_stream_t stream) {
  NvtxRange nvtx_("stitch_estimate_color");
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  if (!check_ptrs(reinterpret_cast<const void *const *>(frames_dev), ctx->g.n))
    return set_err(ctx, STITCH_EINVAL, "frames_dev must hold n_cams non-NULL pointers");
  return launch_estimate_color(ctx, frames_dev, reinterpret_cast<cudaStream_t>(stream));
}

int stitch_frame(stitch_ctx *ctx, const uint8_t *const *frames_dev, const float *const *flow_ij_dev,
                 const float *const *flow_ji_dev, uint8_t *pano_dev, stitch_stream_t stream) {
  NvtxRange nvtx_("stitch_frame");
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  const int np = ctx->g.n - 1;
  if (!check_ptrs(reinterpret_cast<const void *const *>(frames_dev), ctx->g.n))
    return set_err(ctx, STITCH_EINVAL, "frames_dev must hold n_cams non-NULL pointers");
  if (!check_ptrs(reinterpret_cast<const void *const *>(flow_ij_dev), np) ||
      !check_ptrs(reinterpret_cast<const void *const *>(flow_ji_dev), np))
    return set_err(ctx, STITCH_EINVAL, "flow arrays must hold n_pairs non-NULL pointers");
  for (int p = 0; p < np; ++p)
    if ((reinterpret_cast<uintptr_t>(flow_ij_dev[p]) | reinterpret_cast<uintptr_t>(flow_ji_dev[p])) & 7u)
      return set_err(ctx, STITCH_EINVAL, "flow pointers must be 8-byte aligned (float2)");
  if (!pano_dev || (reinterpret_cast<uintptr_t>(pano_dev) & 15u))
    return set_err(ctx, STITCH_EINVAL, "pano_dev must be a non-NULL 16-byte aligned pointer");
  return launch_frame(ctx, frames_dev, flow_ij_dev, flow_ji_dev, pano_dev, reinterpret_cast<cudaStream_t>(stream));
}

int stitch_sequence(stitch_ctx *ctx, int n_frames, const uint8_t *const *frames_dev,
                    const float *const *flow_ij_dev, const float *const *flow_ji_dev,
                    uint8_t *const *pano_dev, stitch_stream_t stream) {
  NvtxRange nvtx_("stitch_sequence");
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  if (n_frames < 1) return set_err(ctx, STITCH_EINVAL, "n_frames must be >= 1");
  const int n = ctx->g.n, np = n - 1;
  if (!check_ptrs(reinterpret_cast<const void *const *>(frames_dev), n_frames * n) ||
      !check_ptrs(reinterpret_cast<const void *const *>(flow_ij_dev), n_frames * np) ||
      !check_ptrs(reinterpret_cast<const void *const *>(flow_ji_dev), n_frames * np) ||
      !check_ptrs(reinterpret_cast<const void *const *>(pano_dev), n_frames))
    return set_err(ctx, STITCH_EINVAL, "sequence pointer arrays must be complete and non-NULL");
  for (int t = 0; t < n_frames; ++t)
    if (reinterpret_cast<uintptr_t>(pano_dev[t]) & 15u)
      return set_err(ctx, STITCH_EINVAL, "pano_dev pointers must be 16-byte aligned");
  for (int i = 0; i < n_frames * np; ++i)
    if ((reinterpret_cast<uintptr_t>(flow_ij_dev[i]) | reinterpret_cast<uintptr_t>(flow_ji_dev[i])) & 7u)
      return set_err(ctx, STITCH_EINVAL, "flow pointers must be 8-byte aligned (float2)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<const void *> key;
  key.reserve((size_t)n_frames * (n + 2 * np + 1));
  for (int i = 0; i < n_frames * n; ++i) key.push_back(frames_dev[i]);
  for (int i = 0; i < n_frames * np; ++i) key.push_back(flow_ij_dev[i]);
  for (int i = 0; i < n_frames * np; ++i) key.push_back(flow_ji_dev[i]);
  for (int i = 0; i < n_frames; ++i) key.push_back(pano_dev[i]);
  // Slot rings repeat every lcm(kRawSlots, kColorSlots) estimates and every
  // kPwSlots fused frames: a recorded graph is valid for that phase only.
  const int parity = (ctx->host_T % 12) * kPwSlots + ctx->host_F % kPwSlots;
  GraphEntry *hit = nullptr;
  for (auto &ge : ctx->graphs)
    if (ge.n_frames == n_frames && ge.parity == parity && ge.prof == ctx->prof && ge.key == key) hit = &ge;
  if (!hit) {
    // Record the sequence on the library's own streams, then replay on `s`.
    // Frame t runs its statistics on pipe[0], its estimate on pipe[1], its
    // band pre-warp on pipe[4] and its fuse on pipe[2 + t % 2]; event edges
    // keep the order the slot rings need. So frame t+1's statistics and
    // pre-warp overlap frame t's estimate and fuse, and the fuse of two
    // consecutive frames (different colour and pre-warp slots) overlap too.
    const int T0 = ctx->host_T, F0 = ctx->host_F;
    cudaGraph_t graph = nullptr;
    GraphEntry ge;
    ge.prof = ctx->prof;
    cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_err(ctx, e, "graph capture begin");
    ctx->prof_sink = &ge.pairs;
    cudaStream_t sA = ctx->pipe[0], sB = ctx->pipe[1], sW = ctx->pipe[4];
    cudaStream_t sC2[2] = {ctx->pipe[2], ctx->pipe[3]};
    cudaEvent_t (&ev)[4][8] = ctx->pev;
    enum { kS = 0, kW = 1, kE = 2, kF = 3 };
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(cudaEventRecord(ev[kF][7], ctx->cap_stream));            // fork
    for (int i = 0; i < kPipeStreams; ++i) chk(cudaStreamWaitEvent(ctx->pipe[i], ev[kF][7], 0));
    int rc = STITCH_OK;
    for (int t = 0; t < n_frames && rc == STITCH_OK && e == cudaSuccess; ++t) {
      const uint8_t *const *fr = frames_dev + (size_t)t * n;
      const FuseParams fp = frame_params(ctx, fr, flow_ij_dev + (size_t)t * np, flow_ji_dev + (size_t)t * np,
                                         pano_dev[t], T0 + t, F0 + t);
      // statistics: slot (T0+t) % 3 was cleared by the estimate of frame t-2
      if (t >= 2) chk(cudaStreamWaitEvent(sA, ev[kE][(t - 2) % 8], 0));
      rc = launch_stats_for(ctx, fr, T0 + t, sA);
      chk(cudaEventRecord(ev[kS][t % 8], sA));
      // band pre-warp: its slot was last read by the fuse of frame t - kPwSlots
      if (t >= kPwSlots) chk(cudaStreamWaitEvent(sW, ev[kF][(t - kPwSlots) % 8], 0));
      if (rc == STITCH_OK) rc = launch_prewarp_for(ctx, fp, sW);
      chk(cudaEventRecord(ev[kW][t % 8], sW));
      // estimate: after this frame's statistics; its colour slot was last read by fuse t-4
      chk(cudaStreamWaitEvent(sB, ev[kS][t % 8], 0));
      if (t >= 4) chk(cudaStreamWaitEvent(sB, ev[kF][(t - 4) % 8], 0));
      // balance on the stitched image: the previous frame's panorama histogram
      if (ctx->out_hist && t >= 1) chk(cudaStreamWaitEvent(sB, ev[kF][(t - 1) % 8], 0));
      if (rc == STITCH_OK) rc = launch_estimate_for(ctx, sB);
      chk(cudaEventRecord(ev[kE][t % 8], sB));
      // fuse: after this frame's estimate and pre-warp
      cudaStream_t sC = sC2[t % 2];
      chk(cudaStreamWaitEvent(sC, ev[kE][t % 8], 0));
      chk(cudaStreamWaitEvent(sC, ev[kW][t % 8], 0));
      if (rc == STITCH_OK) rc = launch_fuse_for(ctx, fp, sC);
      chk(cudaEventRecord(ev[kF][t % 8], sC));
    }
    // join: every pipeline stream back into the capture stream
    for (int i = 0; i < kPipeStreams; ++i) {
      chk(cudaEventRecord(ev[i % 4][i], ctx->pipe[i]));
      chk(cudaStreamWaitEvent(ctx->cap_stream, ev[i % 4][i], 0));
    }
    if (e != cudaSuccess && rc == STITCH_OK) rc = cuda_err(ctx, e, "graph capture");
    e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    ctx->prof_sink = nullptr;
    ctx->host_T = T0;                 // the capture launched nothing
    ctx->host_F = F0;
    if (rc != STITCH_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      for (auto &pp : ge.pairs) {
        cudaEventDestroy(pp.a);
        cudaEventDestroy(pp.b);
      }
      return rc != STITCH_OK ? rc : cuda_err(ctx, e, "graph capture end");
    }
    ge.key = key;
    ge.n_frames = n_frames;
    ge.parity = parity;
    e = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_err(ctx, e, "graph instantiate");
    if (ctx->graphs.size() >= 8) {
      cudaDeviceSynchronize();
      GraphEntry &old = ctx->graphs.front();
      cudaGraphExecDestroy(old.exec);
      for (auto &pp : old.pairs) {
        cudaEventDestroy(pp.a);
        cudaEventDestroy(pp.b);
      }
      ctx->pending.clear();
      ctx->graphs.erase(ctx->graphs.begin());
    }
    ctx->graphs.push_back(std::move(ge));
    hit = &ctx->graphs.back();
  }
  cudaError_t e = cudaGraphLaunch(hit->exec, s);
  if (e != cudaSuccess) return cuda_err(ctx, e, "graph launch");
  if (hit->prof) ctx->pending.insert(ctx->pending.end(), hit->pairs.begin(), hit->pairs.end());
  ctx->host_T += n_frames;
  ctx->host_F += n_frames;
  return STITCH_OK;
}

int stitch_sequence_host(stitch_ctx *ctx, int n_frames, const uint8_t *const *frames_host,
                         const float *const *flow_ij_host, const float *const *flow_ji_host,
                         uint8_t *const *pano_host, stitch_stream_t stream) {
  NvtxRange nvtx_("stitch_sequence_host");
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  if (n_frames < 1) return set_err(ctx, STITCH_EINVAL, "n_frames must be >= 1");
  const Geo &g = ctx->g;
  const int n = g.n, np = n - 1;
  if (!check_ptrs(reinterpret_cast<const void *const *>(frames_host), n_frames * n) ||
      !check_ptrs(reinterpret_cast<const void *const *>(flow_ij_host), n_frames * np) ||
      !check_ptrs(reinterpret_cast<const void *const *>(flow_ji_host), n_frames * np) ||
      !check_ptrs(reinterpret_cast<const void *const *>(pano_host), n_frames))
    return set_err(ctx, STITCH_EINVAL, "sequence pointer arrays must be complete and non-NULL");
  const size_t pano_bytes = (size_t)3 * g.pano_pitch * g.pano_h;
  cudaError_t e = cudaSuccess;
  for (HostStage &hs : ctx->stage) {
    for (int k = 0; k < n && e == cudaSuccess; ++k)
      if (!hs.frames[k]) e = cudaMalloc(&hs.frames[k], (size_t)g.pitch[k] * g.h[k]);
    for (int p = 0; p < np && e == cudaSuccess; ++p) {
      if (!hs.fij[p]) e = cudaMalloc(&hs.fij[p], band_elems(g, p) * 8);
      if (e == cudaSuccess && !hs.fji[p]) e = cudaMalloc(&hs.fji[p], band_elems(g, p) * 8);
    }
    if (e == cudaSuccess && !hs.pano) e = cudaMalloc(&hs.pano, pano_bytes);
    for (cudaEvent_t *ev : {&hs.in_ready, &hs.computed, &hs.out_done})
      if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  }
  if (e == cudaSuccess && !ctx->copy_in) e = cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking);
  if (e == cudaSuccess && !ctx->copy_out) e = cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_err(ctx, e, "staging allocation");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaStream_t si = ctx->copy_in, so = ctx->copy_out;
  // Two frames in flight: the inputs of frame t + 1 copy in on `si` and the
  // panorama of frame t - 1 copies out on `so` while frame t computes on `s`.
  // A slot's inputs are rewritten only after the frame that read them has
  // computed, and its panorama only after the previous copy-out has finished.
  // On an error the three streams are drained before returning, so that no
  // copy of this call is still in flight at the next one.
  auto fail = [&](int rc) {
    cudaStreamSynchronize(si);
    cudaStreamSynchronize(s);
    cudaStreamSynchronize(so);
    return rc;
  };
  for (int t = 0; t < n_frames; ++t) {
    HostStage &hs = ctx->stage[t & 1];
    if (t >= 2) e = cudaStreamWaitEvent(si, hs.computed, 0);
    for (int k = 0; k < n && e == cudaSuccess; ++k)
      e = cudaMemcpyAsync(hs.frames[k], frames_host[(size_t)t * n + k], (size_t)g.pitch[k] * g.h[k],
                          cudaMemcpyHostToDevice, si);
    for (int p = 0; p < np && e == cudaSuccess; ++p) {
      e = cudaMemcpyAsync(hs.fij[p], flow_ij_host[(size_t)t * np + p], band_elems(g, p) * 8,
                          cudaMemcpyHostToDevice, si);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hs.fji[p], flow_ji_host[(size_t)t * np + p], band_elems(g, p) * 8,
                            cudaMemcpyHostToDevice, si);
    }
    if (e == cudaSuccess) e = cudaEventRecord(hs.in_ready, si);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, hs.in_ready, 0);
    if (e == cudaSuccess && t >= 2) e = cudaStreamWaitEvent(s, hs.out_done, 0);
    if (e != cudaSuccess) return fail(cuda_err(ctx, e, "host-to-device copy"));
    const uint8_t *fr[kMaxCams];
    const float *fi[kMaxPairs], *fj[kMaxPairs];
    for (int k = 0; k < n; ++k) fr[k] = hs.frames[k];
    for (int p = 0; p < np; ++p) {
      fi[p] = hs.fij[p];
      fj[p] = hs.fji[p];
    }
    int rc = launch_estimate_color(ctx, fr, s);
    if (rc == STITCH_OK) rc = launch_frame(ctx, fr, fi, fj, hs.pano, s);
    if (rc != STITCH_OK) return fail(rc);
    e = cudaEventRecord(hs.computed, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(so, hs.computed, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pano_host[t], hs.pano, pano_bytes, cudaMemcpyDeviceToHost, so);
    if (e == cudaSuccess) e = cudaEventRecord(hs.out_done, so);
    if (e != cudaSuccess) return fail(cuda_err(ctx, e, "device-to-host copy"));
  }
  // Join the copy-out stream back into `stream`.
  for (int q = 0; q < 2 && q < n_frames && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(s, ctx->stage[q].out_done, 0);
  if (e != cudaSuccess) return fail(cuda_err(ctx, e, "stream join"));
  return stitch_sync(ctx, stream);
}

int stitch_estimate_flow(stitch_ctx *ctx, const uint8_t *const *frames_dev, float *const *flow_ij_dev,
                         float *const *flow_ji_dev, stitch_stream_t stream) {
  NvtxRange nvtx_("stitch_estimate_flow");
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  const Geo &g = ctx->g;
  const int np = g.n - 1;
  if (np < 1) return set_err(ctx, STITCH_EINVAL, "flow needs at least two cameras");
  if (!check_ptrs(reinterpret_cast<const void *const *>(frames_dev), g.n) ||
      !check_ptrs(reinterpret_cast<const void *const *>(flow_ij_dev), np) ||
      !check_ptrs(reinterpret_cast<const void *const *>(flow_ji_dev), np))
    return set_err(ctx, STITCH_EINVAL, "frame and flow pointer arrays must be complete and non-NULL");
  for (int p = 0; p < np; ++p)
    if ((reinterpret_cast<uintptr_t>(flow_ij_dev[p]) | reinterpret_cast<uintptr_t>(flow_ji_dev[p])) & 7u)
      return set_err(ctx, STITCH_EINVAL, "flows must be 8-byte aligned");
  const int radius = std::max(1, (int)std::ceil((double)ctx->max_flow / (double)(1 << (kFlowLevels - 1))));
  if (radius > kFlowMaxRadius) return set_err(ctx, STITCH_EINVAL, "max_flow above 16 px is beyond the flow search");
  // Level sizes and buffer layout.
  FlowParams fl{};
  fl.n_pairs = np;
  // The full level's luminance comes first, laid out like the band pre-warp
  // (same offsets, one byte per element), so that the pre-warp writes it.
  size_t pw_elems = 0, y_bytes = 0, d_elems = 0;
  for (int p = 0; p < np; ++p) {
    const int w = g.band[p][1] - g.band[p][0], h = g.band[p][3] - g.band[p][2];
    fl.pw_off[p][0] = pw_elems;
    fl.pw_off[p][1] = pw_elems + (size_t)w * h;
    pw_elems += 2 * (size_t)w * h;
  }
  y_bytes = pw_elems;
  for (int p = 0; p < np; ++p) {
    int w = g.band[p][1] - g.band[p][0], h = g.band[p][3] - g.band[p][2];
    for (int l = 0; l < kFlowLevels; ++l) {
      if (l > 0) {
        w = (w + 1) / 2;
        h = (h + 1) / 2;
      }
      fl.lev[l].w[p] = w;
      fl.lev[l].h[p] = h;
      for (int k = 0; k < 2; ++k) {
        if (l == 0) {
          fl.lev[l].y_off[p][k] = fl.pw_off[p][k];
        } else {
          fl.lev[l].y_off[p][k] = y_bytes;
          y_bytes += (size_t)w * h;
        }
        fl.lev[l].d_off[p][k] = d_elems;
        d_elems += (size_t)w * h;
      }
    }
  }
  cudaError_t e = cudaSuccess;
  if (!ctx->flow_Y) e = cudaMalloc(&ctx->flow_Y, y_bytes + 16);
  if (e == cudaSuccess && !ctx->flow_d) e = cudaMalloc(&ctx->flow_d, 2 * d_elems * sizeof(int16_t) + 16);
  if (e != cudaSuccess) return cuda_err(ctx, e, "flow buffers");
  fl.Y = ctx->flow_Y;
  fl.dx = ctx->flow_d;
  fl.dy = ctx->flow_d + d_elems;
  for (int p = 0; p < np; ++p) {
    fl.out_ij[p] = reinterpret_cast<float2 *>(flow_ij_dev[p]);
    fl.out_ji[p] = reinterpret_cast<float2 *>(flow_ji_dev[p]);
  }
  // The float32 band pre-warp, written as the luminance pyramid, then the
  // matcher.
  const float *none[kMaxPairs] = {};
  FuseParams fp = frame_params(ctx, frames_dev, none, none, nullptr, ctx->host_T - 1, ctx->host_F);
  fp.flags &= ~(STITCH_FP16_INTERMEDIATE | kFlagPwOffset);
  fp.flags |= kFlagPwLuma;
  for (int p = 0; p < np; ++p) {
    fp.pw_off[p][0] = fl.pw_off[p][0];
    fp.pw_off[p][1] = fl.pw_off[p][1];
    for (int l = 1; l < kFlowLevels; ++l) {
      fp.lum_off[l - 1][p][0] = fl.lev[l].y_off[p][0];
      fp.lum_off[l - 1][p][1] = fl.lev[l].y_off[p][1];
      fp.lum_w[l - 1][p] = fl.lev[l].w[p];
    }
  }
  fp.pw = ctx->flow_Y;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  e = launch_prewarp(fp, s);
  if (e == cudaSuccess) e = launch_flow(fl, radius, s);
  if (e != cudaSuccess) return cuda_err(ctx, e, "flow launch");
  ctx->flow_fl = fl;
  ctx->flow_ready = true;
  return STITCH_OK;
}

int stitch_get_flow_luma(stitch_ctx *ctx, int pair, int side, int level, uint8_t *out_host, int *w, int *h) {
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  if (!ctx->flow_ready) return set_err(ctx, STITCH_EINVAL, "no flow has been estimated on this context");
  if (pair < 0 || pair >= ctx->flow_fl.n_pairs || side < 0 || side > 1 || level < 0 || level >= kFlowLevels)
    return set_err(ctx, STITCH_EINVAL, "pair, side or level out of range");
  const int lw = ctx->flow_fl.lev[level].w[pair], lh = ctx->flow_fl.lev[level].h[pair];
  if (w) *w = lw;
  if (h) *h = lh;
  if (!out_host) return STITCH_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(out_host, ctx->flow_Y + ctx->flow_fl.lev[level].y_off[pair][side], (size_t)lw * (size_t)lh,
                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(ctx, e, "flow luminance read");
  return STITCH_OK;
}

int stitch_pair_M_correspondence(stitch_ctx *ctx, const uint8_t *const *frames_dev, double *M_out) {
  NvtxRange nvtx_("stitch_pair_M_correspondence");
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  const Geo &g = ctx->g;
  const int np = g.n - 1;
  if (np < 1) return set_err(ctx, STITCH_EINVAL, "a correspondence fit needs at least two cameras");
  if (!M_out) return set_err(ctx, STITCH_EINVAL, "M_out is NULL");
  if (!check_ptrs(reinterpret_cast<const void *const *>(frames_dev), g.n))
    return set_err(ctx, STITCH_EINVAL, "frame pointer array must be complete and non-NULL");
  size_t pw_elems = 0;
  for (int p = 0; p < np; ++p) pw_elems += 2 * (size_t)(g.band[p][1] - g.band[p][0]) * (g.band[p][3] - g.band[p][2]);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && !ctx->flow_pw) e = cudaMalloc(&ctx->flow_pw, pw_elems * sizeof(float4) + 16);
  if (e != cudaSuccess) return cuda_err(ctx, e, "correspondence buffers");
  CorrParams cp{};
  cp.n_pairs = np;
  cp.pw = ctx->flow_pw;
  for (int p = 0; p < np; ++p) {
    const int left_is_i = g.pair_i[p] == p ? 1 : 0;
    cp.off_i[p] = ctx->fp.pw_off[p][left_is_i ? 0 : 1];
    cp.off_j[p] = ctx->fp.pw_off[p][left_is_i ? 1 : 0];
    cp.n[p] = (g.band[p][1] - g.band[p][0]) * (g.band[p][3] - g.band[p][2]);
  }
  const int blocks = 128;
  // one buffer of the context, allocated on the first call: block partials, then the totals
  if (e == cudaSuccess && !ctx->corr_buf) e = cudaMalloc(&ctx->corr_buf, (size_t)np * (blocks + 1) * kCorrSums * sizeof(double));
  cp.partial = ctx->corr_buf;
  cp.sums = ctx->corr_buf + (size_t)np * blocks * kCorrSums;
  // The float32 band pre-warp into the context's own buffer, then the sums.
  const float *none[kMaxPairs] = {};
  FuseParams fp = frame_params(ctx, frames_dev, none, none, nullptr, ctx->host_T - 1, ctx->host_F);
  fp.flags &= ~(STITCH_FP16_INTERMEDIATE | kFlagPwOffset);
  fp.pw = ctx->flow_pw;
  if (e == cudaSuccess) e = launch_prewarp(fp, nullptr);
  if (e == cudaSuccess) e = launch_corr(cp, blocks, nullptr);
  std::vector<double> sums((size_t)np * kCorrSums);
  if (e == cudaSuccess) e = cudaMemcpy(sums.data(), cp.sums, sums.size() * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(ctx, e, "correspondence fit");
  int rc = STITCH_OK;
  for (int p = 0; p < np; ++p) {
    const double *t = &sums[(size_t)p * kCorrSums];
    double A[3][4 + 3] = {{t[0], t[1], t[2]}, {t[1], t[3], t[4]}, {t[2], t[4], t[5]}};
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) A[r][3 + c] = t[6 + 3 * r + c];
    // Gaussian elimination with partial pivoting on [A | B].
    bool ok = true;
    for (int c = 0; c < 3 && ok; ++c) {
      int piv = c;
      for (int r = c + 1; r < 3; ++r)
        if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
      if (!(std::fabs(A[piv][c]) > 0.0)) {
        ok = false;
        break;
      }
      if (piv != c)
        for (int k = 0; k < 6; ++k) std::swap(A[c][k], A[piv][k]);
      for (int r = 0; r < 3; ++r) {
        if (r == c) continue;
        const double f = A[r][c] / A[c][c];
        for (int k = c; k < 6; ++k) A[r][k] -= f * A[c][k];
      }
    }
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) M_out[9 * p + 3 * r + c] = ok ? A[r][3 + c] / A[r][r] : (r == c ? 1.0 : 0.0);
    if (!ok) rc = set_err(ctx, STITCH_ESINGULAR, "a band has no colour variation; the identity was returned for it");
  }
  return rc;
}

int stitch_refine_homographies(stitch_ctx *ctx, const float *const *flow_ij_dev, const float *const *flow_ji_dev,
                               double *params_out, double *H_out) {
  NvtxRange nvtx_("stitch_refine_homographies");
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  const Geo &g = ctx->g;
  const int np = g.n - 1;
  if (np < 1) return set_err(ctx, STITCH_EINVAL, "refinement needs at least two cameras");
  if (g.cyl) return set_err(ctx, STITCH_EINVAL, "refinement is defined for planar panoramas only");
  if (!check_ptrs(reinterpret_cast<const void *const *>(flow_ij_dev), np) ||
      !check_ptrs(reinterpret_cast<const void *const *>(flow_ji_dev), np))
    return set_err(ctx, STITCH_EINVAL, "flow pointer arrays must be complete and non-NULL");
  for (int p = 0; p < np; ++p)
    if ((reinterpret_cast<uintptr_t>(flow_ij_dev[p]) | reinterpret_cast<uintptr_t>(flow_ji_dev[p])) & 7u)
      return set_err(ctx, STITCH_EINVAL, "flows must be 8-byte aligned");
  RefineParams rp{};
  rp.n_pairs = np;
  for (int p = 0; p < np; ++p) {
    rp.fij[p] = reinterpret_cast<const float2 *>(flow_ij_dev[p]);
    rp.fji[p] = reinterpret_cast<const float2 *>(flow_ji_dev[p]);
    rp.bw[p] = g.band[p][1] - g.band[p][0];
    rp.bh[p] = g.band[p][3] - g.band[p][2];
  }
  const int n_prob = 8 * np;
  cudaError_t e = cudaDeviceSynchronize();
  // buffers of the context, allocated on the first call (the geometry is fixed)
  if (e == cudaSuccess && !ctx->refine_state) e = cudaMalloc(&ctx->refine_state, n_prob * sizeof(RefineState));
  if (e == cudaSuccess && !ctx->refine_hist) e = cudaMalloc(&ctx->refine_hist, (size_t)n_prob * 256 * sizeof(uint32_t));
  rp.state = ctx->refine_state;
  rp.hist = ctx->refine_hist;
  if (e == cudaSuccess) e = cudaMemset(rp.state, 0, n_prob * sizeof(RefineState));
  if (e == cudaSuccess) e = cudaMemset(rp.hist, 0, (size_t)n_prob * 256 * sizeof(uint32_t));
  for (int shift = 24; shift >= 0 && e == cudaSuccess; shift -= 8) e = launch_refine_pass(rp, shift, nullptr);
  std::vector<RefineState> st(n_prob);
  if (e == cudaSuccess) e = cudaMemcpy(st.data(), rp.state, n_prob * sizeof(RefineState), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(ctx, e, "refinement");
  // The medians (0 where a statistic has no finite value).
  std::vector<double> med(n_prob, 0.0);
  for (int i = 0; i < n_prob; ++i) {
    if (st[i].bad) return set_err(ctx, STITCH_EINVAL, "the flows changed during the refinement");
    if (st[i].n == 0) continue;
    const uint32_t key = st[i].prefix;
    const uint32_t u = (key & 0x80000000u) ? (key & 0x7FFFFFFFu) : ~key;
    float v;
    std::memcpy(&v, &u, 4);
    med[i] = (double)v;
  }
  // Per pair: displacement d and growth g of the left content against the
  // right; the outer camera's correction (t, s) about the band centre; then
  // the corrections composed outward from the reference camera.
  auto mul = [](const double *A, const double *B, double *C) {
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) C[r * 3 + c] = A[r * 3] * B[c] + A[r * 3 + 1] * B[3 + c] + A[r * 3 + 2] * B[6 + c];
  };
  std::vector<std::array<double, 9>> A(np);
  for (int p = 0; p < np; ++p) {
    const double *a = &med[8 * p], *b = &med[8 * p + 4];
    const double dx = (a[0] - b[0]) / 2.0, dy = (a[1] - b[1]) / 2.0;
    const double gx = (a[2] - b[2]) / 2.0, gy = (a[3] - b[3]) / 2.0;
    const double sign = p < g.ref ? -1.0 : 1.0;
    const double tx = sign * dx, ty = sign * dy, sx = 1.0 + sign * gx, sy = 1.0 + sign * gy;
    const double cx = (g.band[p][0] + g.band[p][1] - 1) / 2.0, cy = (g.band[p][2] + g.band[p][3] - 1) / 2.0;
    if (params_out) {
      params_out[4 * p] = tx;
      params_out[4 * p + 1] = ty;
      params_out[4 * p + 2] = sx;
      params_out[4 * p + 3] = sy;
    }
    const double M[9] = {1.0, 0.0, tx, 0.0, 1.0, ty, 0.0, 0.0, 1.0};                      // Eq. 13, skew
    const double N[9] = {sx, 0.0, cx - sx * cx, 0.0, sy, cy - sy * cy, 0.0, 0.0, 1.0};      // scale about c
    mul(M, N, A[p].data());
  }
  std::vector<std::array<double, 9>> C(g.n);
  C[g.ref] = {1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0};
  for (int k = g.ref - 1; k >= 0; --k) mul(C[k + 1].data(), A[k].data(), C[k].data());
  for (int k = g.ref + 1; k < g.n; ++k) mul(C[k - 1].data(), A[k - 1].data(), C[k].data());
  if (H_out)
    for (int k = 0; k < g.n; ++k) mul(C[k].data(), g.H[k], H_out + 9 * k);
  return STITCH_OK;
}

int stitch_sync(stitch_ctx *ctx, stitch_stream_t stream) {
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_err(ctx, e, "stream synchronize");
  int word = 0;
  e = cudaMemcpy(&word, &ctx->state->cond_word, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(ctx, e, "condition read");
  if (word) {
    const int zero = 0;
    e = cudaMemcpy(&ctx->state->cond_word, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_err(ctx, e, "condition clear");
    if (word & 2) return set_err(ctx, STITCH_ETIMEOUT, "a bounded device wait expired");
    return set_err(ctx, STITCH_ESINGULAR, "a colour fit was ill-conditioned; the previous M was kept");
  }
  return STITCH_OK;
}

int stitch_get_color(stitch_ctx *ctx, double *M_out, float *curve_out, int *frame_idx) {
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_err(ctx, e, "device synchronize");
  ColorState *h = new ColorState();
  e = cudaMemcpy(h, ctx->state, sizeof(ColorState), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    delete h;
    return cuda_err(ctx, e, "state read");
  }
  if (M_out)
    for (int k = 0; k < ctx->g.n; ++k)
      for (int i = 0; i < 9; ++i) M_out[k * 9 + i] = h->M_cam[k][i];
  if (curve_out) {
    const Curve *cv = h->out[(h->T + kColorSlots - 1) % kColorSlots].curve;
    for (int c = 0; c < 3; ++c) std::memcpy(curve_out + c * STITCH_CURVE_FLOATS, &cv[c], sizeof(Curve));
  }
  if (frame_idx) *frame_idx = h->T;
  const int sing = h->singular_last;
  delete h;
  return sing ? set_err(ctx, STITCH_ESINGULAR, "a colour fit kept its previous M at the last estimate") : STITCH_OK;
}

int stitch_get_pair_M(stitch_ctx *ctx, double *M_out) {
  if (!ctx || !M_out) return set_err(ctx, STITCH_EINVAL, "ctx and M_out are required");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(M_out, ctx->state->M_pair, sizeof(double) * 9 * (ctx->g.n - 1), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(ctx, e, "pair M read");
  return STITCH_OK;
}

int stitch_get_frame_stats(stitch_ctx *ctx, uint32_t *pooled, uint32_t *Hi, uint32_t *Hj, uint32_t *Wv,
                           uint64_t *A, uint64_t *B) {
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_err(ctx, e, "device synchronize");
  int T = 0;
  e = cudaMemcpy(&T, &ctx->state->T, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(ctx, e, "state read");
  if (T < 1) return set_err(ctx, STITCH_EINVAL, "no frame has been estimated yet");
  const int np = ctx->g.n - 1;
  RawStats *h = new RawStats();
  e = cudaMemcpy(h, ctx->raw + ((T - 1) % kRawSlots), sizeof(RawStats), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    delete h;
    return cuda_err(ctx, e, "stats read");
  }
  if (pooled) std::memcpy(pooled, h->pooled, sizeof(h->pooled));
  if (Hi) std::memcpy(Hi, h->Hi, sizeof(uint32_t) * 768 * np);
  if (Hj) std::memcpy(Hj, h->Hj, sizeof(uint32_t) * 768 * np);
  if (Wv) std::memcpy(Wv, h->Wv, sizeof(uint32_t) * 1536 * np);
  delete h;
  if (A || B) {
    const int slot = (T - 1) % kMaxWindow;
    unsigned long long a[kMaxPairs][6], b[kMaxPairs][9];
    e = cudaMemcpy(a, ctx->state->A_ring[slot], sizeof(a), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(b, ctx->state->B_ring[slot], sizeof(b), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(ctx, e, "ring read");
    static const int sym[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
    for (int p = 0; p < np; ++p)
      for (int i = 0; i < 9; ++i) {
        if (A) A[p * 9 + i] = a[p][sym[i]];
        if (B) B[p * 9 + i] = b[p][i];
      }
  }
  return STITCH_OK;
}

int stitch_get_bands(stitch_ctx *ctx, int *bands, int *rects) {
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  export_geometry(ctx->g, bands, rects);
  return STITCH_OK;
}

struct StateHeader {
  uint32_t magic;
  int32_t n_cams, window, host_T;
  uint64_t bytes;
};

int stitch_save_state(stitch_ctx *ctx, void *buf, size_t *size) {
  if (!ctx || !size) return set_err(ctx, STITCH_EINVAL, "ctx and size are required");
  const size_t need = sizeof(StateHeader) + sizeof(ColorState) + (ctx->ls ? sizeof(LearnedState) : 0);
  if (!buf) {
    *size = need;
    return STITCH_OK;
  }
  if (*size < need) return set_err(ctx, STITCH_EINVAL, "buffer too small");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_err(ctx, e, "device synchronize");
  StateHeader hd{kStateMagic, ctx->g.n, ctx->window, ctx->host_T, sizeof(ColorState)};
  std::memcpy(buf, &hd, sizeof(hd));
  e = cudaMemcpy(static_cast<char *>(buf) + sizeof(hd), ctx->state, sizeof(ColorState), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && ctx->ls)
    e = cudaMemcpy(static_cast<char *>(buf) + sizeof(hd) + sizeof(ColorState), ctx->ls, sizeof(LearnedState),
                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(ctx, e, "state read");
  *size = need;
  return STITCH_OK;
}

int stitch_load_state(stitch_ctx *ctx, const void *buf, size_t size) {
  if (!ctx || !buf) return set_err(ctx, STITCH_EINVAL, "ctx and buf are required");
  if (size < sizeof(StateHeader) + sizeof(ColorState)) return set_err(ctx, STITCH_EINVAL, "state buffer too small");
  StateHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (hd.magic != kStateMagic || hd.bytes != sizeof(ColorState) || hd.n_cams != ctx->g.n || hd.window != ctx->window)
    return set_err(ctx, STITCH_EINVAL, "state was saved from a different configuration");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->state, static_cast<const char *>(buf) + sizeof(hd), sizeof(ColorState),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(ctx->raw, 0, kRawSlots * sizeof(RawStats));
  if (e == cudaSuccess && ctx->ls) {
    // A learned context restores its window of histograms when the buffer has it.
    if (size >= sizeof(StateHeader) + sizeof(ColorState) + sizeof(LearnedState))
      e = cudaMemcpy(ctx->ls, static_cast<const char *>(buf) + sizeof(hd) + sizeof(ColorState), sizeof(LearnedState),
                     cudaMemcpyHostToDevice);
    else
      e = cudaMemset(ctx->ls, 0, sizeof(LearnedState));
    // the learned features follow the restored frame index
    if (e == cudaSuccess) e = cudaMemcpy(&ctx->ls->frame, &ctx->state->T, sizeof(int), cudaMemcpyDeviceToDevice);
  }
  // no stitched image precedes the restored state
  if (e == cudaSuccess && ctx->out_hist) e = cudaMemset(ctx->out_hist, 0, 2 * 768 * sizeof(uint32_t));
  // the output tables follow the restored curves
  for (int sl = 0; sl < kColorSlots && e == cudaSuccess; ++sl)
    e = launch_curve_lut(&ctx->state->out[sl], ctx->flags, ctx->lut + (size_t)sl * kLutBytes, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_err(ctx, e, "state write");
  ctx->host_T = hd.host_T;
  return STITCH_OK;
}

int stitch_profile(stitch_ctx *ctx, int enable) {
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  ctx->prof = enable != 0;
  return STITCH_OK;
}

int stitch_profile_read(stitch_ctx *ctx, double *stage_ms, int *stage_count) {
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_err(ctx, e, "device synchronize");
  double ms[4] = {0.0, 0.0, 0.0, 0.0};
  int cnt[4] = {0, 0, 0, 0};
  for (const ProfPair &pp : ctx->pending) {
    float t = 0.0f;
    e = cudaEventElapsedTime(&t, pp.a, pp.b);
    if (e != cudaSuccess) return cuda_err(ctx, e, "event elapsed time");
    ms[pp.stage] += t;
    cnt[pp.stage] += 1;
  }
  ctx->pending.clear();
  for (auto &pp : ctx->owned) {
    cudaEventDestroy(pp.a);
    cudaEventDestroy(pp.b);
  }
  ctx->owned.clear();
  for (int i = 0; i < 4; ++i) {
    if (stage_ms) stage_ms[i] = ms[i];
    if (stage_count) stage_count[i] = cnt[i];
  }
  return STITCH_OK;
}

int stitch_attach_mlp(stitch_ctx *ctx, stitch_mlp *mlp) {
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  if (mlp && !ctx->ls) return set_err(ctx, STITCH_EINVAL, "the context was not created with STITCH_LEARNED");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_err(ctx, e, "device synchronize");
  ctx->mlp = mlp;
  // the learned features start at the next frame to be estimated
  if (mlp) e = cudaMemcpy(&ctx->ls->frame, &ctx->state->T, sizeof(int), cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) return cuda_err(ctx, e, "learned frame index");
  // Recorded sequences embed the launches of the estimate stage: record again.
  for (auto &ge : ctx->graphs) {
    if (ge.exec) cudaGraphExecDestroy(ge.exec);
    for (auto &pp : ge.pairs) {
      cudaEventDestroy(pp.a);
      cudaEventDestroy(pp.b);
    }
  }
  ctx->graphs.clear();
  return STITCH_OK;
}

int stitch_learned_stats(stitch_ctx *ctx, long long *n_learned, long long *n_fallback) {
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  long long a = 0, b = 0;
  if (ctx->ls) {
    cudaError_t e = cudaDeviceSynchronize();
    unsigned long long v[2] = {0ull, 0ull};
    if (e == cudaSuccess) e = cudaMemcpy(v, &ctx->ls->n_learned, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(ctx, e, "learned counters read");
    a = (long long)v[0];
    b = (long long)v[1];
  }
  if (n_learned) *n_learned = a;
  if (n_fallback) *n_fallback = b;
  return STITCH_OK;
}

int stitch_get_learned(stitch_ctx *ctx, double *M_hat, double *resid, int *used) {
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  if (!ctx->ls) return set_err(ctx, STITCH_EINVAL, "the context was not created with STITCH_LEARNED");
  const int np = ctx->g.n - 1;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && M_hat && np > 0) e = cudaMemcpy(M_hat, ctx->ls->M_hat, sizeof(double) * 9 * np, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && resid && np > 0) e = cudaMemcpy(resid, ctx->ls->resid, sizeof(double) * np, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && used && np > 0) e = cudaMemcpy(used, ctx->ls->used, sizeof(int) * np, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(ctx, e, "learned state read");
  return STITCH_OK;
}

int stitch_n_pairs(const stitch_ctx *ctx) { return ctx ? ctx->g.n - 1 : -1; }

int stitch_get_output_hist(stitch_ctx *ctx, uint32_t *hist_out) {
  if (!ctx || !hist_out) return set_err(ctx, STITCH_EINVAL, "ctx and hist_out are required");
  if (!ctx->out_hist) return set_err(ctx, STITCH_EINVAL, "the context was not created with STITCH_BALANCE_OUTPUT");
  const int F = ctx->host_F - 1;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(hist_out, ctx->out_hist + (size_t)(((F % 2) + 2) % 2) * 768, 768 * sizeof(uint32_t),
                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_err(ctx, e, "output histogram read");
  return STITCH_OK;
}

int stitch_window_fallbacks(stitch_ctx *ctx, unsigned long long *count, int reset) {
  if (!ctx || !count) return set_err(ctx, STITCH_EINVAL, "ctx and count are required");
  unsigned int v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, ctx->win_fallback, sizeof(v), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && reset) e = cudaMemset(ctx->win_fallback, 0, sizeof(unsigned int));
  if (e != cudaSuccess) return cuda_err(ctx, e, "window fallback counter");
  *count = v;
  return STITCH_OK;
}

int stitch_autotune(stitch_ctx *ctx, const uint8_t *const *frames_dev, const float *const *flow_ij_dev,
                    const float *const *flow_ji_dev, uint8_t *pano_dev, int reps, int *shape_out, float *ms_out) {
  NvtxRange nvtx_("stitch_autotune");
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  const int np = ctx->g.n - 1;
  if (reps < 1 || reps > 1000) return set_err(ctx, STITCH_EINVAL, "reps must be in 1..1000");
  if (!check_ptrs(reinterpret_cast<const void *const *>(frames_dev), ctx->g.n) ||
      !check_ptrs(reinterpret_cast<const void *const *>(flow_ij_dev), np) ||
      !check_ptrs(reinterpret_cast<const void *const *>(flow_ji_dev), np))
    return set_err(ctx, STITCH_EINVAL, "frame and flow arrays must be complete and non-NULL");
  for (int p = 0; p < np; ++p)
    if ((reinterpret_cast<uintptr_t>(flow_ij_dev[p]) | reinterpret_cast<uintptr_t>(flow_ji_dev[p])) & 7u)
      return set_err(ctx, STITCH_EINVAL, "flow pointers must be 8-byte aligned (float2)");
  if (!pano_dev || (reinterpret_cast<uintptr_t>(pano_dev) & 15u))
    return set_err(ctx, STITCH_EINVAL, "pano_dev must be a non-NULL 16-byte aligned pointer");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_err(ctx, e, "device synchronize");
  cudaStream_t s = ctx->cap_stream;
  FuseParams fp = frame_params(ctx, frames_dev, flow_ij_dev, flow_ji_dev, pano_dev, ctx->host_T - 1, ctx->host_F);
  e = launch_prewarp(fp, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms[kNumTileShapes];
  int best = -1;
  std::vector<TileDesc> bt;
  TileCounts tc;
  std::string err;
  for (int sh = 0; sh < kNumTileShapes && e == cudaSuccess; ++sh) {
    ms[sh] = -1.0f;
    bt.clear();
    if (!build_tiles(ctx->g, sh, bt, tc, err)) continue;
    e = cudaMemcpyAsync(ctx->tiles, bt.data(), bt.size() * sizeof(TileDesc), cudaMemcpyHostToDevice, s);
    fp.tiles = ctx->tiles;
    fp.n_tiles = (int)bt.size();
    set_counts(fp, tc);
    for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = launch_fuse(fp, sh, s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_fuse(fp, sh, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess) {
      ms[sh] = t / (float)reps;
      if (best < 0 || ms[sh] < ms[best]) best = sh;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess && best < 0) e = cudaErrorInvalidValue;
  // The default shape stays unless another is clearly faster: the shapes time
  // within a few per cent of each other when the fuse runs alone, and the
  // default overlaps best with the other stages of the frame pipeline.
  if (e == cudaSuccess && ms[0] > 0.0f && ms[best] > kTuneMargin * ms[0]) best = 0;
  // Keep the winner: its tile list goes back into the context.
  if (e == cudaSuccess) {
    bt.clear();
    build_tiles(ctx->g, best, bt, tc, err);
    e = cudaMemcpy(ctx->tiles, bt.data(), bt.size() * sizeof(TileDesc), cudaMemcpyHostToDevice);
    ctx->fp.n_tiles = (int)bt.size();
    set_counts(ctx->fp, tc);
    ctx->shape = best;
  }
  if (e != cudaSuccess) return cuda_err(ctx, e, "autotune");
  for (auto &ge : ctx->graphs) {
    if (ge.exec) cudaGraphExecDestroy(ge.exec);
    for (auto &pp : ge.pairs) {
      cudaEventDestroy(pp.a);
      cudaEventDestroy(pp.b);
    }
  }
  ctx->graphs.clear();
  tune_record(ctx->g, ctx->flags, best);
  if (shape_out) *shape_out = best;
  if (ms_out)
    for (int sh = 0; sh < kNumTileShapes; ++sh) ms_out[sh] = ms[sh];
  return STITCH_OK;
}

int stitch_set_tile_shape(stitch_ctx *ctx, int shape) {
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  if (shape < 0 || shape >= kNumTileShapes) return set_err(ctx, STITCH_EINVAL, "no such tile shape");
  std::vector<TileDesc> bt;
  TileCounts tc;
  std::string err;
  if (!build_tiles(ctx->g, shape, bt, tc, err)) return set_err(ctx, STITCH_EINVAL, err);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(ctx->tiles, bt.data(), bt.size() * sizeof(TileDesc), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_err(ctx, e, "tile list upload");
  ctx->fp.n_tiles = (int)bt.size();
  set_counts(ctx->fp, tc);
  ctx->shape = shape;
  for (auto &ge : ctx->graphs) {
    if (ge.exec) cudaGraphExecDestroy(ge.exec);
    for (auto &pp : ge.pairs) {
      cudaEventDestroy(pp.a);
      cudaEventDestroy(pp.b);
    }
  }
  ctx->graphs.clear();
  return STITCH_OK;
}

int stitch_tile_shape(const stitch_ctx *ctx, int *tile_w, int *tile_h) {
  if (!ctx) return set_err(nullptr, STITCH_EINVAL, "ctx is NULL");
  if (tile_w) *tile_w = kTileShapes[ctx->shape].w;
  if (tile_h) *tile_h = kTileShapes[ctx->shape].h;
  return ctx->shape;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched launch of several independent rigs.
// ---------------------------------------------------------------------------

struct BatchGraph {
  std::vector<const void *> key;
  int n_frames = 0;
  cudaGraphExec_t exec = nullptr;
  FuseParams *params = nullptr;       // n_frames x n_rigs parameter blocks
  int *counters = nullptr;            // three work counters per frame (partly covered [+ band], band, fully covered)
};

struct stitch_batch {
  std::vector<stitch_ctx *> ctx;
  std::vector<int> shapes;            // fuse tile shape of every rig
  int uniform = 0;                    // the common shape of all rigs, or -1 when they differ
  bool half = false;
  int cams = 0, pairs = 0;            // totals over the rigs
  std::vector<int> cam_off, pair_off;
  MultiItem *fuse_items = nullptr;    // partly covered pieces of every rig (and the band pieces when the
  int n_fuse_items = 0;               // rigs' tile shapes differ)
  MultiItem *band_items = nullptr;    // band pieces of every rig (rigs of one tile shape)
  int n_band_items = 0;
  int grid_band = 0;
  MultiItem *own_items = nullptr;     // fully covered own tiles of every rig
  int n_own_items = 0;
  int grid_own = 0;
  MultiItem *pw_items = nullptr;
  int n_pw_items = 0;
  int grid = 0;                       // persistent fuse blocks
  size_t mix_smem = 0, mix_own_smem = 0;   // mixed-shape kernels: shared memory for the rigs' shapes
  cudaStream_t cap = nullptr;
  cudaStream_t pipe[kPipeStreams] = {};   // statistics, estimate, band pre-warp, two fuse streams
  cudaEvent_t ev[4][8] = {};
  std::vector<BatchGraph> graphs;
  std::string err;
};

namespace {

int batch_err(stitch_batch *b, int code, const std::string &m) {
  if (b) b->err = m;
  g_last_error = m;
  return code;
}

void free_batch_graph(BatchGraph &g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  cudaFree(g.params);
  cudaFree(g.counters);
  g.exec = nullptr;
  g.params = nullptr;
  g.counters = nullptr;
}

// Work lists of the batch for one tile shape per rig: every rig's band and
// partly covered tiles (band tiles first, the costliest, so that the dynamic
// schedule ends evenly), its fully covered own tiles (the one-camera kernel),
// and its band pre-warp pieces.
int batch_items(stitch_batch *b, const std::vector<int> &shapes) {
  std::vector<MultiItem> band, part, full, pw;
  std::string err;
  for (int r = 0; r < (int)b->ctx.size(); ++r) {
    const int sh = shapes[r];
    if (sh < 0 || sh >= kNumTileShapes) return batch_err(b, STITCH_EINVAL, "tile shape out of range");
    std::vector<TileDesc> bt;
    TileCounts tc;
    if (!build_tiles(b->ctx[r]->g, sh, bt, tc, err)) return batch_err(b, STITCH_EINVAL, err);
    for (const TileDesc &t : bt)
      (t.kind == kTileOwn ? full : t.kind == kTileBand ? band : part).push_back(MultiItem{r, sh, t, PwTile{}});
    const Geo &g = b->ctx[r]->g;
    for (int p = 0; p + 1 < g.n; ++p)
      for (int y = g.band[p][2]; y < g.band[p][3]; y += kTileH)
        for (int x = g.band[p][0]; x < g.band[p][1]; x += kTileW)
          pw.push_back(MultiItem{r, 0, TileDesc{}, PwTile{p, x, y}});
  }
  int uniform = shapes.empty() ? 0 : shapes[0];
  for (int sh : shapes)
    if (sh != uniform) uniform = -1;
  // Rigs of one tile shape: the band pieces in their own persistent kernel
  // (as for a single rig). Otherwise they follow the partly covered pieces,
  // which go first (costliest per pixel) so that the dynamic schedule ends
  // evenly.
  if (uniform < 0) {
    part.insert(part.end(), band.begin(), band.end());
    band.clear();
  }
  cudaFree(b->fuse_items);
  cudaFree(b->band_items);
  cudaFree(b->own_items);
  cudaFree(b->pw_items);
  b->fuse_items = nullptr;
  b->band_items = nullptr;
  b->own_items = nullptr;
  b->pw_items = nullptr;
  cudaError_t e = cudaMalloc(&b->fuse_items, part.size() * sizeof(MultiItem) + 16);
  if (e == cudaSuccess) e = cudaMalloc(&b->band_items, band.size() * sizeof(MultiItem) + 16);
  if (e == cudaSuccess) e = cudaMalloc(&b->own_items, full.size() * sizeof(MultiItem) + 16);
  if (e == cudaSuccess) e = cudaMalloc(&b->pw_items, pw.size() * sizeof(MultiItem) + 16);
  if (e == cudaSuccess && !part.empty())
    e = cudaMemcpy(b->fuse_items, part.data(), part.size() * sizeof(MultiItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !band.empty())
    e = cudaMemcpy(b->band_items, band.data(), band.size() * sizeof(MultiItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !full.empty())
    e = cudaMemcpy(b->own_items, full.data(), full.size() * sizeof(MultiItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !pw.empty())
    e = cudaMemcpy(b->pw_items, pw.data(), pw.size() * sizeof(MultiItem), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return batch_err(b, STITCH_ECUDA, std::string("batch work lists: ") + cudaGetErrorString(e));
  b->n_fuse_items = (int)part.size();
  b->n_band_items = (int)band.size();
  b->n_own_items = (int)full.size();
  b->n_pw_items = (int)pw.size();
  int sms = 148, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->mix_smem = uniform < 0 ? fuse_mixed_smem(shapes.data(), (int)shapes.size(), 2) : 0;
  b->mix_own_smem = uniform < 0 ? fuse_mixed_smem(shapes.data(), (int)shapes.size(), 1) : 0;
  const int per_sm = std::max(1, fuse_multi_blocks_per_sm(b->half, uniform, b->mix_smem));
  b->grid = std::max(1, std::min(b->n_fuse_items, per_sm * sms));
  const int per_sm_band = uniform < 0 ? 1 : std::max(1, fuse_band_multi_blocks_per_sm(b->half, uniform));
  b->grid_band = std::max(1, std::min(b->n_band_items, per_sm_band * sms));
  const int per_sm_own = std::max(1, fuse_own_multi_blocks_per_sm(uniform, b->mix_own_smem));
  b->grid_own = std::max(1, std::min(b->n_own_items, per_sm_own * sms));
  b->shapes = shapes;
  b->uniform = uniform;
  for (auto &g : b->graphs) free_batch_graph(g);
  b->graphs.clear();
  return STITCH_OK;
}

bool batch_ptrs_ok(stitch_batch *b, int n_frames, const uint8_t *const *frames_dev, const float *const *fij,
                   const float *const *fji, uint8_t *const *pano_dev) {
  const int R = (int)b->ctx.size();
  if (!check_ptrs(reinterpret_cast<const void *const *>(frames_dev), n_frames * b->cams) ||
      !check_ptrs(reinterpret_cast<const void *const *>(pano_dev), n_frames * R))
    return false;
  if (b->pairs > 0 && (!check_ptrs(reinterpret_cast<const void *const *>(fij), n_frames * b->pairs) ||
                       !check_ptrs(reinterpret_cast<const void *const *>(fji), n_frames * b->pairs)))
    return false;
  for (int i = 0; i < n_frames * R; ++i)
    if (reinterpret_cast<uintptr_t>(pano_dev[i]) & 15u) return false;
  for (int i = 0; i < n_frames * b->pairs; ++i)
    if ((reinterpret_cast<uintptr_t>(fij[i]) | reinterpret_cast<uintptr_t>(fji[i])) & 7u) return false;
  return true;
}

}  // namespace

extern "C" {

int stitch_batch_create(stitch_ctx *const *ctxs, int n_ctx, stitch_batch **out) {
  for (int i = 0; ctxs && i < n_ctx; ++i)
    if (ctxs[i] && (ctxs[i]->flags & STITCH_BALANCE_OUTPUT))
      return batch_err(nullptr, STITCH_EINVAL, "a batch cannot hold a context with STITCH_BALANCE_OUTPUT");
  if (!out) return batch_err(nullptr, STITCH_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctxs || n_ctx < 1 || n_ctx > STITCH_BATCH_MAX_RIGS)
    return batch_err(nullptr, STITCH_EINVAL, "need 1..STITCH_BATCH_MAX_RIGS contexts");
  for (int i = 0; i < n_ctx; ++i) {
    if (!ctxs[i]) return batch_err(nullptr, STITCH_EINVAL, "a context is NULL");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return batch_err(nullptr, STITCH_EINVAL, "a context appears twice");
    if ((ctxs[i]->flags & STITCH_FP16_INTERMEDIATE) != (ctxs[0]->flags & STITCH_FP16_INTERMEDIATE))
      return batch_err(nullptr, STITCH_EINVAL, "all contexts must agree on STITCH_FP16_INTERMEDIATE");
    if (ctxs[i]->device != ctxs[0]->device) return batch_err(nullptr, STITCH_EINVAL, "contexts are on different GPUs");
  }
  stitch_batch *b = new (std::nothrow) stitch_batch();
  if (!b) return batch_err(nullptr, STITCH_ENOMEM, "host allocation failed");
  b->ctx.assign(ctxs, ctxs + n_ctx);
  b->half = (ctxs[0]->flags & STITCH_FP16_INTERMEDIATE) != 0;
  for (stitch_ctx *c : b->ctx) {
    b->cam_off.push_back(b->cams);
    b->pair_off.push_back(b->pairs);
    b->cams += c->g.n;
    b->pairs += c->g.n - 1;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (int i = 0; i < kPipeStreams && e == cudaSuccess; ++i)
    e = cudaStreamCreateWithFlags(&b->pipe[i], cudaStreamNonBlocking);
  for (int a = 0; a < 4 && e == cudaSuccess; ++a)
    for (int k = 0; k < 8 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&b->ev[a][k], cudaEventDisableTiming);
  // Each rig starts from its batched-launch shape in the tune cache, else the
  // shape its own context runs with.
  std::vector<int> sh(n_ctx, 0);
  for (int r = 0; r < n_ctx; ++r) sh[r] = tuned_shape(ctxs[r]->g, ctxs[r]->flags, true, ctxs[r]->shape);
  int rc = e == cudaSuccess ? batch_items(b, sh) : batch_err(b, STITCH_ECUDA, cudaGetErrorString(e));
  if (rc != STITCH_OK && e == cudaSuccess) rc = batch_items(b, std::vector<int>(n_ctx, 0));
  if (rc != STITCH_OK) {
    const std::string m = b->err;
    stitch_batch_destroy(b);
    return batch_err(nullptr, rc, m);
  }
  *out = b;
  return STITCH_OK;
}

int stitch_batch_sequence(stitch_batch *b, int n_frames, const uint8_t *const *frames_dev,
                          const float *const *flow_ij_dev, const float *const *flow_ji_dev, uint8_t *const *pano_dev,
                          stitch_stream_t stream) {
  NvtxRange nvtx_("stitch_batch_sequence");
  if (!b) return batch_err(nullptr, STITCH_EINVAL, "batch is NULL");
  if (n_frames < 1) return batch_err(b, STITCH_EINVAL, "n_frames must be >= 1");
  if (!batch_ptrs_ok(b, n_frames, frames_dev, flow_ij_dev, flow_ji_dev, pano_dev))
    return batch_err(b, STITCH_EINVAL,
                     "pointer arrays must be complete and non-NULL, panoramas 16-byte and flows 8-byte aligned");
  const int R = (int)b->ctx.size();
  if (R == 1) {
    // One rig: there is no cross-rig work to merge, so the frames run the
    // rig's own persistent kernels in its recorded sequence graph (the same
    // streams and slot rings), at the batch's tile shape.
    stitch_ctx *c = b->ctx[0];
    int rc = STITCH_OK;
    if (c->shape != b->shapes[0]) rc = stitch_set_tile_shape(c, b->shapes[0]);
    if (rc == STITCH_OK) rc = stitch_sequence(c, n_frames, frames_dev, flow_ij_dev, flow_ji_dev, pano_dev, stream);
    return rc == STITCH_OK ? STITCH_OK : batch_err(b, rc, "batch sequence: " + c->err);
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<const void *> key;
  for (int i = 0; i < n_frames * b->cams; ++i) key.push_back(frames_dev[i]);
  for (int i = 0; i < n_frames * b->pairs; ++i) key.push_back(flow_ij_dev[i]);
  for (int i = 0; i < n_frames * b->pairs; ++i) key.push_back(flow_ji_dev[i]);
  for (int i = 0; i < n_frames * R; ++i) key.push_back(pano_dev[i]);
  for (stitch_ctx *c : b->ctx) {   // each rig's slot phases and its network
    key.push_back(reinterpret_cast<const void *>((uintptr_t)((c->host_T % 12) * kPwSlots + c->host_F % kPwSlots)));
    key.push_back(c->mlp);
  }
  BatchGraph *hit = nullptr;
  for (auto &bg : b->graphs)
    if (bg.n_frames == n_frames && bg.key == key) hit = &bg;
  if (!hit) {
    BatchGraph bg;
    bg.key = key;
    bg.n_frames = n_frames;
    cudaError_t e = cudaMalloc(&bg.params, (size_t)n_frames * R * sizeof(FuseParams));
    if (e == cudaSuccess) e = cudaMalloc(&bg.counters, (size_t)n_frames * 3 * sizeof(int));
    std::vector<FuseParams> hp((size_t)n_frames * R);
    for (int t = 0; t < n_frames; ++t)
      for (int r = 0; r < R; ++r) {
        stitch_ctx *c = b->ctx[r];
        const int np = c->g.n - 1;
        const size_t fo = (size_t)t * b->cams + b->cam_off[r], po = (size_t)t * b->pairs + b->pair_off[r];
        hp[(size_t)t * R + r] = frame_params(c, frames_dev + fo, np ? flow_ij_dev + po : nullptr,
                                             np ? flow_ji_dev + po : nullptr, pano_dev[(size_t)t * R + r],
                                             c->host_T + t, c->host_F + t);
      }
    if (e == cudaSuccess)
      e = cudaMemcpy(bg.params, hp.data(), hp.size() * sizeof(FuseParams), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      free_batch_graph(bg);
      return batch_err(b, STITCH_ECUDA, std::string("batch parameters: ") + cudaGetErrorString(e));
    }
    // Same five-stream structure and slot-ring edges as stitch_sequence, with
    // every rig's statistics and estimate launched per rig and the band
    // pre-warp and fuse of all rigs in one launch each: frame t's statistics
    // on pipe[0], its estimate on pipe[1], its band pre-warp on pipe[4] and its
    // fuse on pipe[2 + t % 2], so consecutive frames' fuses overlap.
    std::vector<char> prof(R);
    for (int r = 0; r < R; ++r) {
      prof[r] = b->ctx[r]->prof;
      b->ctx[r]->prof = false;
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    cudaStream_t sA = b->pipe[0], sB = b->pipe[1], sW = b->pipe[4];
    cudaStream_t sC2[2] = {b->pipe[2], b->pipe[3]};
    auto &ev = b->ev;
    enum { kS = 0, kW = 1, kE = 2, kF = 3 };
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(cudaEventRecord(ev[kF][7], b->cap));
    for (int i = 0; i < kPipeStreams; ++i) chk(cudaStreamWaitEvent(b->pipe[i], ev[kF][7], 0));
    int rc = STITCH_OK;
    for (int t = 0; t < n_frames && rc == STITCH_OK && e == cudaSuccess; ++t) {
      // statistics: slot (T0+t) % 3 was cleared by the estimate of frame t-2
      if (t >= 2) chk(cudaStreamWaitEvent(sA, ev[kE][(t - 2) % 8], 0));
      for (int r = 0; r < R && rc == STITCH_OK; ++r)
        rc = launch_stats_for(b->ctx[r], frames_dev + (size_t)t * b->cams + b->cam_off[r], b->ctx[r]->host_T + t, sA);
      chk(cudaEventRecord(ev[kS][t % 8], sA));
      // band pre-warp: its slot was last read by the fuse of frame t - kPwSlots
      if (t >= kPwSlots) chk(cudaStreamWaitEvent(sW, ev[kF][(t - kPwSlots) % 8], 0));
      MultiParams mp{bg.params, t * R, b->n_pw_items, b->pw_items, nullptr};
      chk(launch_prewarp_multi(mp, b->half, sW));
      chk(cudaEventRecord(ev[kW][t % 8], sW));
      // estimate: after this frame's statistics; its colour slot was last read by fuse t-4
      chk(cudaStreamWaitEvent(sB, ev[kS][t % 8], 0));
      if (t >= 4) chk(cudaStreamWaitEvent(sB, ev[kF][(t - 4) % 8], 0));
      for (int r = 0; r < R && rc == STITCH_OK; ++r) rc = launch_estimate_for(b->ctx[r], sB);
      chk(cudaEventRecord(ev[kE][t % 8], sB));
      // fuse: after this frame's estimate and pre-warp
      cudaStream_t sC = sC2[t % 2];
      chk(cudaStreamWaitEvent(sC, ev[kE][t % 8], 0));
      chk(cudaStreamWaitEvent(sC, ev[kW][t % 8], 0));
      chk(cudaMemsetAsync(bg.counters + 3 * t, 0, 3 * sizeof(int), sC));
      MultiParams mf{bg.params, t * R, b->n_fuse_items, b->fuse_items, bg.counters + 3 * t};
      chk(launch_fuse_multi(mf, b->half, b->uniform, b->grid, sC, b->mix_smem));
      MultiParams mb{bg.params, t * R, b->n_band_items, b->band_items, bg.counters + 3 * t + 1};
      chk(launch_fuse_band_multi(mb, b->half, b->uniform, b->grid_band, sC));
      MultiParams mo{bg.params, t * R, b->n_own_items, b->own_items, bg.counters + 3 * t + 2};
      chk(launch_fuse_own_multi(mo, b->uniform, b->grid_own, sC, b->mix_own_smem));
      chk(cudaEventRecord(ev[kF][t % 8], sC));
    }
    // join: every pipeline stream back into the capture stream
    for (int i = 0; i < kPipeStreams; ++i) {
      chk(cudaEventRecord(ev[i % 4][i], b->pipe[i]));
      chk(cudaStreamWaitEvent(b->cap, ev[i % 4][i], 0));
    }
    const cudaError_t e_end = cudaStreamEndCapture(b->cap, &graph);
    for (int r = 0; r < R; ++r) b->ctx[r]->prof = prof[r] != 0;
    if (e == cudaSuccess) e = e_end;
    if (rc == STITCH_OK && e == cudaSuccess) e = cudaGraphInstantiate(&bg.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc != STITCH_OK || e != cudaSuccess) {
      free_batch_graph(bg);
      if (rc != STITCH_OK) return batch_err(b, rc, "batch capture: " + b->ctx[0]->err);
      return batch_err(b, STITCH_ECUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    }
    if (b->graphs.size() >= 4) {
      cudaDeviceSynchronize();
      free_batch_graph(b->graphs.front());
      b->graphs.erase(b->graphs.begin());
    }
    b->graphs.push_back(std::move(bg));
    hit = &b->graphs.back();
  }
  const cudaError_t e = cudaGraphLaunch(hit->exec, s);
  if (e != cudaSuccess) return batch_err(b, STITCH_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  for (stitch_ctx *c : b->ctx) {
    c->host_T += n_frames;
    c->host_F += n_frames;
  }
  return STITCH_OK;
}

int stitch_batch_autotune(stitch_batch *b, const uint8_t *const *frames_dev, const float *const *flow_ij_dev,
                          const float *const *flow_ji_dev, uint8_t *const *pano_dev, int reps, int *shapes_out,
                          float *ms_out) {
  NvtxRange nvtx_("stitch_batch_autotune");
  if (!b) return batch_err(nullptr, STITCH_EINVAL, "batch is NULL");
  if (reps < 1 || reps > 1000) return batch_err(b, STITCH_EINVAL, "reps must be in 1..1000");
  if (!batch_ptrs_ok(b, 1, frames_dev, flow_ij_dev, flow_ji_dev, pano_dev))
    return batch_err(b, STITCH_EINVAL, "pointer arrays must be complete, non-NULL and aligned");
  const int R = (int)b->ctx.size();
  if (R == 1) {
    // One rig runs its own kernels (stitch_batch_sequence): tune those.
    int shape = 0;
    float ms1[kNumTileShapes];
    int rc = stitch_autotune(b->ctx[0], frames_dev, flow_ij_dev, flow_ji_dev, pano_dev[0], reps, &shape, ms1);
    if (rc != STITCH_OK) return batch_err(b, rc, "batch autotune: " + b->ctx[0]->err);
    rc = batch_items(b, std::vector<int>{shape});
    if (rc != STITCH_OK) return rc;
    if (shapes_out) shapes_out[0] = shape;
    if (ms_out)
      for (int sh = 0; sh < kNumTileShapes; ++sh) ms_out[sh] = ms1[sh];
    return STITCH_OK;
  }
  cudaError_t e = cudaDeviceSynchronize();
  FuseParams *params = nullptr;
  int *counter = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&params, R * sizeof(FuseParams));
  if (e == cudaSuccess) e = cudaMalloc(&counter, 3 * sizeof(int));
  std::vector<FuseParams> hp(R);
  for (int r = 0; r < R; ++r) {
    stitch_ctx *c = b->ctx[r];
    const int np = c->g.n - 1;
    hp[r] = frame_params(c, frames_dev + b->cam_off[r], np ? flow_ij_dev + b->pair_off[r] : nullptr,
                         np ? flow_ji_dev + b->pair_off[r] : nullptr, pano_dev[r], c->host_T - 1, c->host_F);
  }
  if (e == cudaSuccess) e = cudaMemcpy(params, hp.data(), R * sizeof(FuseParams), cudaMemcpyHostToDevice);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // The band intermediates of the frame (they do not depend on the shapes).
  if (e == cudaSuccess) {
    MultiParams pw{params, 0, b->n_pw_items, b->pw_items, nullptr};
    e = launch_prewarp_multi(pw, b->half, b->cap);
  }
  // Both fuse launches of the frame with the current work lists, timed.
  auto timed = [&](float &ms) {
    MultiParams mf{params, 0, b->n_fuse_items, b->fuse_items, counter};
    MultiParams mb{params, 0, b->n_band_items, b->band_items, counter + 1};
    MultiParams mo{params, 0, b->n_own_items, b->own_items, counter + 2};
    auto both = [&]() {
      cudaError_t x = cudaMemsetAsync(counter, 0, 3 * sizeof(int), b->cap);
      if (x == cudaSuccess) x = launch_fuse_multi(mf, b->half, b->uniform, b->grid, b->cap, b->mix_smem);
      if (x == cudaSuccess) x = launch_fuse_band_multi(mb, b->half, b->uniform, b->grid_band, b->cap);
      if (x == cudaSuccess) x = launch_fuse_own_multi(mo, b->uniform, b->grid_own, b->cap, b->mix_own_smem);
      return x;
    };
    cudaError_t x = cudaSuccess;
    for (int w = 0; w < 2 && x == cudaSuccess; ++w) x = both();
    if (x == cudaSuccess) x = cudaEventRecord(e0, b->cap);
    for (int k = 0; k < reps && x == cudaSuccess; ++k) x = both();
    if (x == cudaSuccess) x = cudaEventRecord(e1, b->cap);
    if (x == cudaSuccess) x = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (x == cudaSuccess) x = cudaEventElapsedTime(&t, e0, e1);
    ms = t / (float)reps;
    return x;
  };
  // One rig at a time (coordinate descent): try every shape for rig r with the
  // other rigs at their current shapes, keep the fastest batch.
  std::vector<int> cur = b->shapes;
  std::vector<float> ms((size_t)R * kNumTileShapes, -1.0f);
  for (int r = 0; r < R && e == cudaSuccess; ++r) {
    int best = cur[r];
    float best_ms = -1.0f;
    for (int sh = 0; sh < kNumTileShapes && e == cudaSuccess; ++sh) {
      std::vector<int> trial = cur;
      trial[r] = sh;
      if (batch_items(b, trial) != STITCH_OK) continue;   // a tile would touch two bands
      float t = 0.0f;
      e = timed(t);
      if (e != cudaSuccess) break;
      ms[(size_t)r * kNumTileShapes + sh] = t;
      if (best_ms < 0.0f || t < best_ms) {
        best_ms = t;
        best = sh;
      }
    }
    // as for one rig: the default shape unless another is clearly faster
    const float t0 = ms[(size_t)r * kNumTileShapes];
    if (t0 > 0.0f && best_ms > kTuneMargin * t0) best = 0;
    cur[r] = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(params);
  cudaFree(counter);
  const int rc = batch_items(b, e == cudaSuccess ? cur : b->shapes);
  if (e != cudaSuccess) return batch_err(b, STITCH_ECUDA, std::string("batch autotune: ") + cudaGetErrorString(e));
  if (rc != STITCH_OK) return rc;
  for (int r = 0; r < R; ++r) tune_record(b->ctx[r]->g, b->ctx[r]->flags, cur[r], true);
  if (shapes_out)
    for (int r = 0; r < R; ++r) shapes_out[r] = cur[r];
  if (ms_out)
    for (size_t i = 0; i < ms.size(); ++i) ms_out[i] = ms[i];
  return STITCH_OK;
}

int stitch_batch_tile_shapes(const stitch_batch *b, int *shapes_out) {
  if (!b || !shapes_out) return batch_err(nullptr, STITCH_EINVAL, "batch and shapes_out are required");
  for (size_t r = 0; r < b->shapes.size(); ++r) shapes_out[r] = b->shapes[r];
  return (int)b->shapes.size();
}

void stitch_batch_destroy(stitch_batch *b) {
  if (!b) return;
  cudaDeviceSynchronize();
  for (auto &g : b->graphs) free_batch_graph(g);
  cudaFree(b->fuse_items);
  cudaFree(b->band_items);
  cudaFree(b->own_items);
  cudaFree(b->pw_items);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int i = 0; i < kPipeStreams; ++i)
    if (b->pipe[i]) cudaStreamDestroy(b->pipe[i]);
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 8; ++k)
      if (b->ev[a][k]) cudaEventDestroy(b->ev[a][k]);
  delete b;
}

const char *stitch_batch_last_error(const stitch_batch *b) { return b ? b->err.c_str() : g_last_error.c_str(); }

const char *stitch_last_error(const stitch_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_last_error.c_str();
}

void stitch_destroy(stitch_ctx *ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  for (auto &ge : ctx->graphs) {
    if (ge.exec) cudaGraphExecDestroy(ge.exec);
    for (auto &pp : ge.pairs) {
      cudaEventDestroy(pp.a);
      cudaEventDestroy(pp.b);
    }
  }
  for (auto &pp : ctx->owned) {
    cudaEventDestroy(pp.a);
    cudaEventDestroy(pp.b);
  }
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->net_stream) cudaStreamDestroy(ctx->net_stream);
  for (int k = 0; k < 2; ++k)
    if (ctx->net_ev[k]) cudaEventDestroy(ctx->net_ev[k]);
  for (int i = 0; i < kPipeStreams; ++i)
    if (ctx->pipe[i]) cudaStreamDestroy(ctx->pipe[i]);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 8; ++b)
      if (ctx->pev[a][b]) cudaEventDestroy(ctx->pev[a][b]);
  cudaFree(ctx->raw);
  cudaFree(ctx->state);
  cudaFree(ctx->ls);
  cudaFree(ctx->tiles);
  cudaFree(ctx->pw_tiles);
  cudaFree(ctx->pw);
  cudaFree(ctx->lut);
  cudaFree(ctx->win_fallback);
  cudaFree(ctx->out_hist);
  for (HostStage &hs : ctx->stage) {
    for (int k = 0; k < kMaxCams; ++k) cudaFree(hs.frames[k]);
    for (int p = 0; p < kMaxPairs; ++p) {
      cudaFree(hs.fij[p]);
      cudaFree(hs.fji[p]);
    }
    cudaFree(hs.pano);
    if (hs.in_ready) cudaEventDestroy(hs.in_ready);
    if (hs.computed) cudaEventDestroy(hs.computed);
    if (hs.out_done) cudaEventDestroy(hs.out_done);
  }
  cudaFree(ctx->flow_pw);
  cudaFree(ctx->flow_Y);
  cudaFree(ctx->flow_d);
  cudaFree(ctx->refine_state);
  cudaFree(ctx->refine_hist);
  cudaFree(ctx->corr_buf);
  if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
  if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
  delete ctx;
}

}  // extern "C"
