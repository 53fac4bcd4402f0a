// Internal device-side structures of the stitching library (not part of the
// public ABI). Layouts here are shared by the host code and the kernels.
#pragma once

#include <climits>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "../../include/stitch.h"

namespace stitch {

constexpr int kMaxCams = STITCH_MAX_CAMS;
constexpr int kMaxPairs = STITCH_MAX_PAIRS;
constexpr int kMaxWindow = STITCH_MAX_WINDOW;
constexpr int kSmoothFrames = 3;      // Eq. 6-7: current frame and its last two
constexpr int kTileW = 64;            // band pre-warp piece: 64 x 32 panorama pixels
constexpr int kTileH = 32;
constexpr int kFuseThreads = 256;
// Fuse tile shapes (panorama pixels) the autotuner chooses from; shape 0 is
// the default. Width is a multiple of 32 (a warp spans 32 columns), height a
// multiple of 16, and width x height a multiple of the 256 threads of a
// block: 2 (32 x 16) to 16 (128 x 32) pixels per thread.
struct TileShape {
  int w, h;
};
constexpr int kNumTileShapes = 6;
constexpr TileShape kTileShapes[kNumTileShapes] = {{64, 32}, {64, 16}, {32, 32}, {128, 16}, {32, 16}, {128, 32}};
constexpr int kStatsThreads = 256;
constexpr int kEstimateThreads = 256;
constexpr double kCondLimit = 1e12;
// Buffer rings that let successive frames overlap in a recorded sequence:
// statistics slots (stats of frame t+1 run beside the estimate of frame t),
// colour slots (the estimate of frame t+1 runs beside the fuse of frame t) and
// band pre-warp slots.
constexpr int kRawSlots = 3;
constexpr int kColorSlots = 4;
constexpr int kPwSlots = 2;
// Output table of the balance curve (Eq. 5) and the final rounding: per
// channel, entry n holds round_half_even(F(n / 16)) for the fused, clamped
// value n / 16, n = 0 .. 4080 (a sixteenth of a grey level per step).
constexpr int kLutEntries = 4096;
constexpr float kLutTop = 4080.0f;
constexpr int kLutBytes = 3 * kLutEntries;
// Internal fuse flag (above the public STITCH_* bits): the band pre-warp of a
// frame stores v - 128 (the fused path's offset form) instead of v.
constexpr int kFlagPwOffset = 1 << 20;
// Band pre-warp for the flow: write the integer luminance of the float32
// samples (one byte per band pixel and side, element offsets pw_off) instead
// of the samples themselves, and the next two levels of its pyramid
// (FuseParams::lum_off / lum_w).
constexpr int kFlagPwLuma = 1 << 21;

// Integer statistics of one frame, written by the stats kernel (K1) and read
// by the estimate kernel (K2). Frame T uses slot T % kRawSlots.
struct RawStats {
  uint32_t pooled[3][256];            // full-frame histogram of all cameras
  uint32_t Hi[kMaxPairs][3][256];     // overlap histogram, colour-source side i
  uint32_t Hj[kMaxPairs][3][256];     // overlap histogram, reference side j
  uint32_t Wv[kMaxPairs][6][256];     // value-weighted histograms of side i
  unsigned long long A[kMaxPairs][6]; // Gram sums (00,01,02,11,12,22) of side i
};

// Per-channel balance curve used by the fuse kernel (Eq. 5 reading).
struct Curve {
  float m1, m2, d1, d2, s, g1, g2, inv_m1, inv_bm, ident;
};

// What the fuse kernel reads: frame T's estimate is in slot T % kColorSlots.
struct ColorOut {
  float M[kMaxCams][9];               // row-vector convention, v' = v . M
  Curve curve[3];
};

// Temporal state of the colour estimate, owned by the estimate kernel.
struct ColorState {
  int T;                              // frames estimated so far
  int cond_word;                      // sticky device conditions (bit 0 singular, bit 1 timeout)
  int singular_last;                  // bitmask of pairs that kept their M at the last estimate
  int pad;
  unsigned long long A_ring[kMaxWindow][kMaxPairs][6];
  unsigned long long B_ring[kMaxWindow][kMaxPairs][9];
  int n_ring[kMaxWindow][kMaxPairs][2];
  int knots[kSmoothFrames][3][2];     // ring of per-frame (m1, m2) per channel
  double M_pair[kMaxPairs][9];
  double M_cam[kMaxCams][9];
  double knot_mean[3][2];
  ColorOut out[kColorSlots];
};

// One camera as the fuse kernel sees it. h maps (x - ox, y - oy, 1) of the
// panorama to the camera (float32, origin-shifted so that the numbers
// entering the products stay small).
struct CamDev {
  float h[9];
  float hm[9];                        // h with rows x and y less half of row w: maps to s - (1/2, 1/2)
  int ox, oy;
  int w, h_px, pitch;
  float wm1, hm1;
  int own_lo, own_hi;
  int affine;                         // h[6] == h[7] == 0: no perspective divide
  int cyl;                            // cylindrical panorama: h maps the ray of (x, y), see below
  float cyl_finv, cyl_cx, cyl_cy;     // theta = (x - cyl_cx) * cyl_finv, height = (y - cyl_cy) * cyl_finv
};

struct BandDev {
  int x0, x1, y0, y1;
  float inv_bw;
};

// One piece of a fuse tile: columns [16 c0, 16 c1) of the tile (tx, ty); the
// pieces of one tile write disjoint 16-byte column chunks, so different
// blocks can stitch them independently.
struct TileDesc {
  int16_t tx, ty;                     // tile origin / (tile width, tile height)
  int8_t kind;                        // kTileOwn, kTileBand, kTileOwnPart or kTileBandPart
  int8_t idx;                         // camera (own kinds) or pair (band kinds)
  uint8_t c0, c1;                     // column range in 16-pixel units within the tile
};
constexpr int kTileOwn = 0;           // own columns of camera idx, every pixel seen by it with a margin
constexpr int kTileBand = 1;          // inside the blend band rectangle of pair idx
constexpr int kTileOwnPart = 2;       // own columns of camera idx, partly covered
constexpr int kTileBandPart = 3;      // band columns of pair idx with other pixels (band edge chunk, rows
                                      // outside the band rectangle)

// One kTileW x kTileH piece of a band rectangle for the band pre-warp kernel.
struct PwTile {
  int pair;
  int x0, y0;                         // panorama origin of the piece
};

struct alignas(16) FuseParams {
  int n_cams;
  int flags;
  int pano_w, pano_h, pano_pitch;
  int halo;
  float max_flow;
  int n_tiles;
  int n_band;                         // tiles [n_tiles - n_full - n_band, n_tiles - n_full) are band tiles
  int n_full;                         // the last n_full tiles are fully covered own tiles
  const TileDesc *tiles;
  int n_pw_tiles;
  const PwTile *pw_tiles;
  void *pw;                           // pre-warped band intermediate (both cameras of every band)
  size_t pw_off[kMaxPairs][2];        // element offsets of band p, left / right camera
  const ColorOut *color;
  const uint8_t *lut;                 // the colour slot's output table (kLutBytes)
  unsigned int *win_fallback;         // tiles whose source window did not fit in shared memory (counter)
  uint32_t *out_hist;                 // STITCH_BALANCE_OUTPUT: this frame's pre-balance histogram [3][256], or null
  size_t lum_off[2][kMaxPairs][2];    // kFlagPwLuma: byte offsets (into pw) of pyramid levels 1 and 2, band p, side
  int lum_w[2][kMaxPairs];            // their widths
  CamDev cam[kMaxCams];
  BandDev band[kMaxPairs];
  const uint8_t *src[kMaxCams];
  const float2 *flow_ij[kMaxPairs];
  const float2 *flow_ji[kMaxPairs];
  uint8_t *out;
};

// One unit of a launch that covers several rigs (and frames): rig r's tile
// (or band pre-warp piece) with the parameters params[base + r].
struct MultiItem {
  int rig;
  int shape;                          // fuse items: the rig's tile shape (index into kTileShapes)
  TileDesc tile;                      // fuse items
  PwTile pw;                          // pre-warp items
};

struct MultiParams {
  const FuseParams *params;           // device array, indexed by base + rig
  int base;
  int n_items;
  const MultiItem *items;
  int *counter;                       // work counter of the persistent fuse (zero before the launch)
};

struct RoleDev {
  int rx0, rx1, ry0, ry1;
  int pair;
  int is_i;                           // 1: colour-source side (H, W and A), 0: reference side (H)
};

struct StatsParams {
  int n_cams;
  int rows_per_block;
  int vec_ok[kMaxCams];               // 16-byte aligned rows: vector loads allowed
  const uint8_t *src[kMaxCams];
  int w[kMaxCams], h[kMaxCams], pitch[kMaxCams];
  int n_roles[kMaxCams];
  RoleDev roles[kMaxCams][2];
  RawStats *raw;                      // the slot this frame accumulates into (cleared beforehand)
};

struct EstimateParams {
  int n_cams, n_pairs, ref, window;
  int flags;                          // STITCH_BALANCE_OFF selects the identity output table
  uint8_t *lut;                       // kColorSlots output tables (slot T % kColorSlots), or null
  uint32_t *out_hist;                 // STITCH_BALANCE_OUTPUT: 2 x [3][256], frame F in slot F % 2, or null
  long long lambda_q;                 // lambda in millionths
  int pair_i[kMaxPairs], pair_j[kMaxPairs];
  int raw_slots;                      // frame T reads slot T % raw_slots and clears slot (T - 1) % raw_slots
  RawStats *raw;
  ColorState *state;
};

// One batch of independent overlap pairs for the labeller of the learned
// estimator: pair p is two packed-RGB patches of pw x ph pixels, side i then
// side j, at pairs + p * 2 * pw * ph * 3.
struct PairParams {
  const uint8_t *pairs;
  int n, pw, ph;
  long long lambda_q;                 // lambda in millionths
  __nv_bfloat16 *feat;                // [n][1536]
  float *targ;                        // [n][12]
  double *M;                          // [n][9] or null
  int *flags;                         // [n] or null
};

// State of the learned estimator inside a context: the per-frame overlap
// histograms of the last kMaxWindow frames (the window-pooled features), the
// features and network output of the latest frame, and its decisions.
struct LearnedState {
  uint32_t H_ring[kMaxWindow][kMaxPairs][2][768];
  __nv_bfloat16 feat[kMaxPairs][STITCH_MLP_IN];
  float y[32][STITCH_MLP_OUT];        // network output, target units (rows >= n_pairs unused)
  double M_hat[kMaxPairs][9];
  double resid[kMaxPairs];
  int used[kMaxPairs];
  int frame;                          // the frame whose features are formed next (the colour state's T)
  unsigned long long n_learned, n_fallback;
};

struct LearnedParams {
  int n_cams, n_pairs, ref, window, raw_slots;
  const RawStats *raw;
  ColorState *state;
  LearnedState *ls;
};

// Homography refinement (k_refine.cu): radix-selection state of one median.
struct RefineState {
  uint32_t prefix, mask;              // key bits chosen so far
  uint32_t k;                         // rank still wanted among the keys that match them
  uint32_t n;                         // finite values
  uint32_t bad;                       // counts changed between passes
  uint32_t pad[3];
};

struct RefineParams {
  const float2 *fij[kMaxPairs];
  const float2 *fji[kMaxPairs];
  int bw[kMaxPairs], bh[kMaxPairs];
  int n_pairs;
  RefineState *state;                 // [n_pairs * 8], zeroed before the first pass
  uint32_t *hist;                     // [n_pairs * 8][256], zeroed before the first pass
};

// Band optical flow (k_flow.cu): a coarse-to-fine block matcher over the
// luminance of both cameras' pre-warped band images.
constexpr int kFlowLevels = 3;
constexpr int kFlowMaxRadius = 4;     // coarsest search radius: max_flow up to STITCH_MAX_FLOW = 16 px
static_assert(STITCH_MAX_FLOW <= (float)(kFlowMaxRadius << (kFlowLevels - 1)), "the coarsest search covers max_flow");
static_assert(kFlowLevels == 3, "the band pre-warp writes levels 1 and 2 of the luminance pyramid");
static_assert(kTileW % 4 == 0 && kTileH % 4 == 0,
              "pre-warp pieces start at multiples of 4 band pixels, so each builds whole 2 x 2 blocks of both levels");

struct FlowLevelDev {
  int w[kMaxPairs], h[kMaxPairs];     // level size of every band
  size_t y_off[kMaxPairs][2];         // luminance of the left / right camera (bytes into Y)
  size_t d_off[kMaxPairs][2];         // chosen displacements, direction 0 / 1 (elements into dx, dy)
};

struct FlowParams {
  int n_pairs;
  FlowLevelDev lev[kFlowLevels];
  size_t pw_off[kMaxPairs][2];        // full-level luminance of band p, left / right camera (offsets into Y)
  uint8_t *Y;
  int16_t *dx, *dy;
  float2 *out_ij[kMaxPairs], *out_ji[kMaxPairs];
};

// One-frame colour transfer from pixel correspondences (k_corr.cu).
constexpr int kCorrSums = 15;         // A = X^T X (6 distinct entries), B = X^T Y (9)
constexpr int kCorrMaxBlocks = 256;

struct CorrParams {
  int n_pairs;
  const float4 *pw;                   // float32 pre-warped bands
  size_t off_i[kMaxPairs], off_j[kMaxPairs];   // element offsets of the colour source / target band
  int n[kMaxPairs];                   // band pixels
  double *partial;                    // [n_pairs][blocks][kCorrSums]
  double *sums;                       // [n_pairs][kCorrSums]
};

// Launchers (defined in the kernel files).
cudaError_t launch_stats(const StatsParams &p, int grid_x, cudaStream_t s);
cudaError_t launch_estimate(const EstimateParams &p, cudaStream_t s);
// The output table of one colour slot from its curve (after a state load).
cudaError_t launch_curve_lut(const ColorOut *slot, int flags, uint8_t *lut, cudaStream_t s);
cudaError_t estimate_setup();
cudaError_t launch_prewarp(const FuseParams &p, cudaStream_t s);
cudaError_t launch_fuse(const FuseParams &p, int shape, cudaStream_t s);
cudaError_t launch_prewarp_multi(const MultiParams &m, bool half, cudaStream_t s);
// The persistent multi-rig fuse kernels: shape >= 0 when every rig uses that
// tile shape, -1 to run every item with its MultiItem::shape.
// mixed_smem: for shape -1, the dynamic shared memory of the mixed-shape
// kernels (fuse_mixed_smem over the batch's shapes; 0 = enough for any shape).
cudaError_t launch_fuse_multi(const MultiParams &m, bool half, int shape, int grid, cudaStream_t s,
                              size_t mixed_smem = 0);
int fuse_multi_blocks_per_sm(bool half, int shape, size_t mixed_smem = 0);
cudaError_t launch_fuse_own_multi(const MultiParams &m, int shape, int grid, cudaStream_t s, size_t mixed_smem = 0);
int fuse_own_multi_blocks_per_sm(int shape, size_t mixed_smem = 0);
// Shared memory a mixed-shape fuse kernel needs for tiles of the given shapes
// (windows = 2: band and partly covered pieces; 1: fully covered own tiles).
size_t fuse_mixed_smem(const int *shapes, int n, int windows);
cudaError_t launch_fuse_band_multi(const MultiParams &m, bool half, int shape, int grid, cudaStream_t s);
int fuse_band_multi_blocks_per_sm(bool half, int shape);
cudaError_t fuse_setup_attributes(int max_halo);
// The correspondence sums of every pair (blocks per pair, fixed-order totals).
cudaError_t launch_corr(const CorrParams &p, int blocks, cudaStream_t s);
// Every level of the band flow of every pair, both directions.
// The matcher levels of every pair (the band pre-warp under kFlagPwLuma has
// written every luminance level).
cudaError_t launch_flow(const FlowParams &p, int radius, cudaStream_t s);
// One radix pass (key bits [shift, shift + 8)) of every band-flow median.
cudaError_t launch_refine_pass(const RefineParams &p, int shift, cudaStream_t s);
size_t stats_smem_bytes();
size_t prewarp_elem_bytes(bool fp16);
cudaError_t launch_learned_features(const LearnedParams &p, cudaStream_t s);
cudaError_t launch_learned_select(const LearnedParams &p, cudaStream_t s);

}  // namespace stitch

#include <string>
namespace stitch {
int prepare_estimate_params(const stitch_config *cfg, StatsParams &sp, int &grid_x, EstimateParams &ep,
                            std::string &err);
void record_last_error(const std::string &msg);
}  // namespace stitch
