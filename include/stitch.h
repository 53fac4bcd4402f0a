/*
 * stitch.h -- C ABI of the B300 video-stitching hot path.
 *
 * Implements the per-frame data-parallel path of "GPU Accelerated Color
 * Correction and Frame Warping for Real-time Video Stitching" (arXiv
 * 2308.09209): inverse-homography pre-warp (section 3.1), optical-flow local
 * warping with bilinear sampling (section 3.2, Eq. 17-18), the spatio-temporal
 * 3D-M colour transfer (section 2.1, Eq. 1-4), the piecewise online colour
 * balance (section 2.2, Eq. 5-7) and weighted-mean fusion (Eq. 15-16), plus the
 * integer overlap statistics that estimate M.
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status (stitch_status). Argument errors are
 *    detected on the host before anything is launched. No C++ exception
 *    crosses this boundary.
 *  - Device pointers ("_dev") are CUDA device addresses owned by the caller;
 *    the library never frees them. Host pointers ("_host") are plain host
 *    memory (page-locked memory makes the copies asynchronous and faster).
 *  - Launches are asynchronous on the given stream (NULL = legacy default
 *    stream). Device-side conditions (a singular colour fit) are recorded in
 *    the context and reported by stitch_sync / stitch_get_color.
 *  - Camera frames are packed RGB uint8, row-major (HWC), row pitch in bytes
 *    >= 3 * width. The panorama is planar uint8: three planes (R, G, B), each
 *    pano_h rows of pano_pitch bytes, plane c starting at c * pano_pitch *
 *    pano_h. Bytes [pano_w, pano_pitch) of a row are not part of the image and
 *    may be overwritten with 0.
 *  - Pixel centres sit at integer coordinates. A camera homography maps a
 *    camera pixel (u, v, 1) to panorama coordinates.
 *  - Adjacent cameras k, k+1 form pair k. Each pair has a blend band: an
 *    integer rectangle [x0, x1) x [y0, y1) of panorama pixels covered by both
 *    cameras. Flow fields are per pair, float2 (dx, dy) per band pixel,
 *    row-major band_w x band_h, indexed by (x - x0, y - y0).
 */
#ifndef STITCH_H
#define STITCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *stitch_stream_t;

typedef enum {
  STITCH_OK = 0,
  STITCH_EINVAL = -1,     /* bad argument or geometry; nothing was launched */
  STITCH_ENOMEM = -2,     /* a device or host allocation failed */
  STITCH_ECUDA = -3,      /* a CUDA runtime call failed (message in stitch_last_error) */
  STITCH_ESINGULAR = -4,  /* a pair's colour fit was ill-conditioned: its previous M was kept */
  STITCH_ETIMEOUT = -5,   /* a bounded device-side wait expired */
  STITCH_EFALLBACK = 1    /* informational: the learned estimator fell back to the plain fit */
} stitch_status;

/* stitch_config.flags */
#define STITCH_BALANCE_OFF 1          /* skip the online balance (Eq. 5) */
#define STITCH_FP16_INTERMEDIATE 2    /* warped band tiles held in FP16; coordinates stay FP32 */
#define STITCH_FLOW_WEIGHTS_PRINTED 4 /* Eq. 17 exactly as printed (theta_i on flow_ij) */
#define STITCH_LEARNED 8              /* learned estimator for M (falls back to the plain fit) */
#define STITCH_BALANCE_OUTPUT 16      /* balance knots from the stitched image of the previous frame */

#define STITCH_MAX_CAMS 8
#define STITCH_MAX_PAIRS (STITCH_MAX_CAMS - 1)
#define STITCH_MAX_WINDOW 16
#define STITCH_MAX_FLOW 16.0f
#define STITCH_CURVE_FLOATS 10        /* per channel, see stitch_get_color */

typedef struct {
  int n_cams;               /* 2 .. STITCH_MAX_CAMS */
  const int *cam_w;         /* n_cams widths (>= 2) */
  const int *cam_h;         /* n_cams heights (>= 2) */
  const int *cam_pitch;     /* n_cams row pitches in bytes (>= 3 * w); NULL = 3 * w */
  const double *H;          /* n_cams x 9, row-major, inverted by the library in float64
                               (section 3.1). Planar: camera -> panorama homography.
                               Cylindrical: camera pixel (u, v, 1) -> viewing ray
                               (x right, y down, z forward) in the rig's frame,
                               e.g. R_k^T K_k^-1. */
  int pano_w, pano_h;       /* panorama size in pixels */
  int pano_pitch;           /* bytes per panorama row, >= pano_w, multiple of 16 */
  int projection;           /* STITCH_PROJ_PLANAR or STITCH_PROJ_CYLINDRICAL */
  int ref_cam;              /* colour reference camera; -1 = n_cams / 2 */
  int window;               /* 3D-M temporal window W in frames (Eq. 2-3; 3 in the paper), 1..16 */
  double lambda;            /* balance quantile (section 2.2; 0.05 in the paper), 0 < lambda < 0.5 */
  float max_flow;           /* flow components are clamped to +-max_flow pixels, 0..16 */
  int flags;                /* STITCH_* flags above */
  /* Cylindrical projection only: panorama pixel (x, y) is the ray at azimuth
   * theta = (x - cyl_cx) / cyl_focal and height (y - cyl_cy) / cyl_focal on
   * the unit cylinder, i.e. direction (sin theta, (y - cyl_cy) / cyl_focal,
   * cos theta). cyl_focal is in panorama pixels per radian. */
  double cyl_focal, cyl_cx, cyl_cy;
} stitch_config;

#define STITCH_PROJ_PLANAR 0
#define STITCH_PROJ_CYLINDRICAL 1

typedef struct stitch_ctx stitch_ctx;

/*
 * stitch_geometry -- the overlap geometry of a configuration, on the host only
 * (section 2.1 step 1: the overlap region follows from the homographies;
 * section 3.1). Needs no GPU and allocates no device memory.
 *   bands: out, (n_cams - 1) x 4 ints: x0, x1, y0, y1 of each pair's blend band.
 *   rects: out, (n_cams - 1) x 8 ints: the band's source rectangle in the left
 *          camera (x0, x1, y0, y1) then in the right camera, both half-open.
 *   Either output may be NULL. Returns STITCH_EINVAL (message in
 *   stitch_last_error(NULL)) for an invalid configuration.
 */
int stitch_geometry(const stitch_config *cfg, int *bands, int *rects);

/*
 * stitch_init -- validate cfg, compute the geometry in float64, allocate the
 * context's device state (statistics ring, colour state, tile lists) on the
 * current CUDA device. *out receives the new context; free it with
 * stitch_destroy. cfg and the arrays it points to may be freed afterwards.
 */
int stitch_init(const stitch_config *cfg, stitch_ctx **out);

/*
 * stitch_estimate_color -- colour statistics and estimate of the next frame T
 * (section 2.1 steps 2-4, Eq. 1-3; section 2.2 Eq. 6-7).
 *   frames_dev: n_cams device pointers to this frame's camera images.
 * Launches the statistics reduction (pooled full-frame histograms; per pair
 * the overlap histograms, value-weighted histograms and Gram sums) and the
 * single-block estimate (histogram specification, windowed M = A^-1 B in
 * float64, chaining to the reference camera, balance knots and curve).
 * Advances the frame index T by one.
 */
int stitch_estimate_color(stitch_ctx *ctx, const uint8_t *const *frames_dev, stitch_stream_t stream);

/*
 * stitch_frame -- fused pre-warp, local warping, colour transfer, balance and
 * blend of one frame into the panorama (section 3.1, Eq. 4-5, Eq. 15-18),
 * using the colour state of the latest stitch_estimate_color.
 *   frames_dev:  n_cams device pointers (the same images given to the estimate).
 *   flow_ij_dev: n_pairs device pointers, flow sampled for the LEFT camera of
 *                each pair (float2 per band pixel, 8-byte aligned).
 *   flow_ji_dev: n_pairs device pointers, flow for the RIGHT camera.
 *   pano_dev:    device pointer (16-byte aligned) to 3 * pano_pitch * pano_h
 *                bytes, written.
 */
int stitch_frame(stitch_ctx *ctx, const uint8_t *const *frames_dev, const float *const *flow_ij_dev,
                 const float *const *flow_ji_dev, uint8_t *pano_dev, stitch_stream_t stream);

/*
 * stitch_sequence -- n_frames consecutive frames (estimate + frame for each)
 * in one call. Arrays are frame-major: frames_dev[t * n_cams + k],
 * flow_*_dev[t * n_pairs + p], pano_dev[t]. The first call with a given set
 * of pointers records a CUDA graph of the whole sequence; later calls with
 * the same pointers replay it.
 */
int stitch_sequence(stitch_ctx *ctx, int n_frames, const uint8_t *const *frames_dev,
                    const float *const *flow_ij_dev, const float *const *flow_ji_dev,
                    uint8_t *const *pano_dev, stitch_stream_t stream);

/*
 * stitch_sequence_host -- as stitch_sequence, but every array is HOST memory:
 * the library copies each frame's images and flows to its own device staging
 * buffers (two frames' worth), runs the frame on `stream` and copies the
 * panorama back. The copies run on two library-owned streams so that the
 * inputs of frame t + 1 and the panorama of frame t - 1 move while frame t
 * computes; events order them against `stream`. Returns after all of it has
 * drained (on an error too). Host frames are read with the configured row
 * pitch; host flows are dense band_w x band_h float2. Page-locked host memory
 * is needed for the copies to overlap.
 */
int stitch_sequence_host(stitch_ctx *ctx, int n_frames, const uint8_t *const *frames_host,
                         const float *const *flow_ij_host, const float *const *flow_ji_host,
                         uint8_t *const *pano_host, stitch_stream_t stream);

/*
 * stitch_estimate_flow -- optical flow between the pre-warped images of every
 * pair over its blend band (section 3.2), in the layout stitch_frame takes:
 *   frames_dev:  n_cams device pointers (packed RGB, as for stitch_frame).
 *   flow_ij_dev: n_pairs device pointers (8-byte aligned, band_w x band_h
 *                float2), written: the left camera's pre-warped image sampled
 *                at q + flow_ij(q) matches the right camera's at q.
 *   flow_ji_dev: likewise, the right camera's image onto the left one's.
 * Method (the paper leaves it to a library routine): both cameras are
 * pre-warped over the band in float32 (the band pre-warp kernel, into the
 * context's own buffer), reduced to integer luminance round((R + 2G + B) / 4),
 * and matched coarse to fine over a 3-level 2 x 2 integer pyramid by the sum
 * of absolute differences over 7 x 7 windows (coordinates clamped into the
 * band): radius R = max(1, ceil(max_flow / 4)) at the coarsest level,
 * 2 d + [-1, 1]^2 below, ties to the smaller |d - start|^2, then d_y, then
 * d_x; a float32 parabola through the costs of the neighbours gives the
 * sub-pixel step (at most half a pixel). Asynchronous on `stream`; calls on
 * one context must be ordered by the caller. STITCH_EINVAL for fewer than two
 * cameras, bad pointers or max_flow above 32 px.
 */
int stitch_estimate_flow(stitch_ctx *ctx, const uint8_t *const *frames_dev, float *const *flow_ij_dev,
                         float *const *flow_ji_dev, stitch_stream_t stream);

/*
 * stitch_get_flow_luma -- one level of the integer luminance pyramid that the
 * latest stitch_estimate_flow on this context matched (paper section 3.2; the
 * pyramid is this library's flow, not printed in the paper): level `level`
 * (0 = full band resolution, then each level the 2 x 2 average of the one
 * below, 3 levels) of camera `pair + side` (side 0 = the left camera of the
 * pair, 1 = the right one) over the blend band of pair `pair`. *w and *h
 * (each optional) receive the level's size; out_host (caller-owned host
 * memory of w * h bytes, rows of w bytes; NULL to query the size only)
 * receives the image. A diagnostic: it lets a test separate the float32
 * pre-warp's rounding of the luminance from the integer matching that
 * follows. Synchronises the device. Returns STITCH_OK, STITCH_EINVAL (no flow
 * estimated yet, or an index out of range) or STITCH_ECUDA.
 */
int stitch_get_flow_luma(stitch_ctx *ctx, int pair, int side, int level, uint8_t *out_host, int *w, int *h);

/*
 * stitch_pair_M_correspondence -- the one-frame colour transfer from pixel
 * correspondences that the paper compares its 3D-M against (Tables 2-3, the
 * 2D-M method): for every pair, with colour source i and target j oriented
 * toward the reference camera, X and Y the two cameras' float32 pre-warped
 * samples over the pair's blend band (rows of RGB at the same panorama
 * positions), M = (X^T X)^-1 (X^T Y) with the sums in float64 (fixed-order
 * reduction) and the 3 x 3 solve on the host.
 *   frames_dev: n_cams device pointers (as for stitch_frame).
 *   M_out (host): n_pairs x 9 doubles, row-major, row-vector convention.
 * The context's colour state is not touched. Synchronous. STITCH_ESINGULAR
 * (identity written for that pair) when a band's X^T X is singular.
 */
int stitch_pair_M_correspondence(stitch_ctx *ctx, const uint8_t *const *frames_dev, double *M_out);

/*
 * stitch_refine_homographies -- revised camera homographies from one frame's
 * band flows (section 3.1, Eq. 13-14: the skew matrix M and the scale matrix
 * N, with the flow fields in place of SURF matches). Planar panoramas only.
 *   flow_ij_dev / flow_ji_dev: n_pairs device pointers laid out as for
 *       stitch_frame (band_w x band_h float2, 8-byte aligned); read only.
 *   params_out (optional, host): n_pairs x 4 doubles (t_x, t_y, s_x, s_y),
 *       the correction of the pair's camera farther from the reference:
 *       q -> c + s (q - c) + t in panorama pixels, c the band centre
 *       ((x0 + x1 - 1) / 2, (y0 + y1 - 1) / 2).
 *   H_out (optional, host): n_cams x 9 doubles, row-major camera -> panorama
 *       homographies C_k H_k, the corrections composed outward from the
 *       reference camera (C_ref = I, C_k = C_(k+1) A_k to its left and
 *       C_(k-1) A_(k-1) to its right); pass them to a new stitch_init.
 * Per pair the left camera's content sits displaced by d = (median flow_ij -
 * median flow_ji) / 2 against the right camera's and grows across the band by
 * g = (median forward difference of flow_ij - the same of flow_ji) / 2 (x
 * differences of x, y differences of y; float32 subtractions); the outer
 * camera gets (t, s) = (-d, 1 - g) on the left of the reference and (+d, 1 + g)
 * on its right. A median is the ((n - 1) / 2)-th smallest finite value, exact
 * (radix selection on the GPU); with none it is 0. The context itself is not
 * changed. Synchronous (waits for the device first). STITCH_EINVAL for a
 * cylindrical context, fewer than two cameras or bad pointers.
 */
int stitch_refine_homographies(stitch_ctx *ctx, const float *const *flow_ij_dev, const float *const *flow_ji_dev,
                               double *params_out, double *H_out);

/*
 * stitch_sync -- wait for `stream`, then report (and clear) the device-side
 * condition word: STITCH_ESINGULAR if a colour fit kept its previous M since
 * the last report, else STITCH_OK.
 */
int stitch_sync(stitch_ctx *ctx, stitch_stream_t stream);

/*
 * stitch_get_color -- current colour state (synchronises the device).
 *   M_out:     n_cams x 9 doubles, each camera's matrix chained to the
 *              reference (row-vector convention v' = v . M, Eq. 4). May be NULL.
 *   curve_out: 3 x STITCH_CURVE_FLOATS floats per channel: m1, m2 (smoothed
 *              knots, Eq. 6-7), d1, d2, s, g1, g2, 1/m1, 1/(255 - m2),
 *              identity flag (1.0f when m2 - m1 < 1). May be NULL.
 *   frame_idx: number of frames estimated so far. May be NULL.
 * Returns STITCH_ESINGULAR when the latest estimate kept a previous M.
 */
int stitch_get_color(stitch_ctx *ctx, double *M_out, float *curve_out, int *frame_idx);

/*
 * stitch_get_pair_M -- the latest per-pair transfer matrices M = A^-1 B
 * (n_pairs x 9 doubles, row-major, Eq. 1/Eq. 3), pair p mapping its
 * colour-source camera onto its neighbour toward the reference. Synchronises.
 */
int stitch_get_pair_M(stitch_ctx *ctx, double *M_out);

/*
 * stitch_get_frame_stats -- the integer statistics of the latest estimated
 * frame (synchronises the device). Any output may be NULL.
 *   pooled: 3 x 256 uint32, per-channel histogram of all camera frames.
 *   Hi, Hj: n_pairs x 3 x 256 uint32, overlap histograms of the colour-source
 *           camera i and of its reference neighbour j (section 2.1 step 2).
 *   Wv:     n_pairs x 6 x 256 uint32, value-weighted histograms of side i,
 *           W_cd[v] = sum of channel c over pixels whose channel d equals v,
 *           for (c, d) = (0,1), (0,2), (1,0), (1,2), (2,0), (2,1).
 *   A:      n_pairs x 9 uint64, this frame's I_i^T I_i (Eq. 3 term).
 *   B:      n_pairs x 9 uint64, this frame's I_i^T I_j with I_j the
 *           specified ("revised") image i (Eq. 3 term).
 */
int stitch_get_frame_stats(stitch_ctx *ctx, uint32_t *pooled, uint32_t *Hi, uint32_t *Hj, uint32_t *Wv,
                           uint64_t *A, uint64_t *B);

/* stitch_get_bands -- the context's geometry, same layout as stitch_geometry. */
int stitch_get_bands(stitch_ctx *ctx, int *bands, int *rects);

/*
 * stitch_save_state / stitch_load_state -- serialise the temporal state (frame
 * index, windowed statistics ring, knot ring, per-pair M, colour state) so a
 * stream can resume mid-sequence with identical output. save: if buf is NULL,
 * *size receives the byte count; else *size must be at least that and the
 * state is written (synchronises the device). load: buf/size from a context
 * with the same configuration.
 */
int stitch_save_state(stitch_ctx *ctx, void *buf, size_t *size);
int stitch_load_state(stitch_ctx *ctx, const void *buf, size_t size);

/*
 * stitch_profile / stitch_profile_read -- stage timing with CUDA events.
 * While enabled, every stage launch is bracketed by two events on its stream
 * (also inside graphs recorded by stitch_sequence, as event nodes). read
 * synchronises the device and returns, per stage (0 = statistics, 1 =
 * estimate, 2 = fused warp, 3 = band pre-warp; stage_ms and stage_count hold 4
 * entries each), the summed GPU milliseconds and the number of launches since
 * the last read, then forgets them. For a replayed graph, read after every
 * replay: its events hold the latest replay only. In a recorded sequence the
 * stages of successive frames overlap on separate streams, so the stage times
 * add up to more than the elapsed time.
 */
int stitch_profile(stitch_ctx *ctx, int enable);
int stitch_profile_read(stitch_ctx *ctx, double *stage_ms, int *stage_count);

/*
 * stitch_estimate_color_noalloc -- the colour estimate of ONE frame without
 * any device allocation. The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc, such as plugins whose host
 * application owns every device buffer, code that must not allocate while a
 * stream is being captured, or real-time threads that may not block in the
 * driver's allocator. It needs no context (stitch_init allocates; this does
 * not).
 *   cfg:           as for stitch_init, at most STITCH_NOALLOC_MAX_CAMS cameras
 *                  (larger rigs are rejected with STITCH_EINVAL). The fit uses
 *                  this frame only: it equals the first stitch_estimate_color of
 *                  a fresh context (window and knot mean over one frame).
 *   frames_dev:    n_cams device pointers to the frame's camera images.
 *   M_out_dev:     device buffer of n_cams x 9 doubles, written: each camera's
 *                  matrix chained to the reference (as stitch_get_color).
 *   curve_out_dev: device buffer of 3 x STITCH_CURVE_FLOATS floats, written (as
 *                  stitch_get_color).
 *   flags_out_dev: optional device int, written: bitmask of pairs whose fit was
 *                  ill-conditioned (those pairs get the identity).
 * Working memory is a fixed STITCH_NOALLOC_SCRATCH_BYTES array in the
 * library's device image, held by every GPU that loads the library until the
 * process exits, and shared by all calls on that GPU: calls whose work
 * overlaps on the GPU (other streams, other threads) race and corrupt each
 * other; serialise them. Each call clears the part that must start at zero.
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * Later calls on a stream that is not being captured look the address up
 * again (a cudaDeviceReset reloads the library's device image, possibly at
 * another address); a call during a capture uses the address found last, so
 * after a reset make one call outside any capture before capturing again.
 * Launches are asynchronous on `stream`; the call performs no cudaMalloc,
 * cudaFree or other allocation of device memory.
 */
#define STITCH_NOALLOC_MAX_CAMS 8
#define STITCH_NOALLOC_SCRATCH_BYTES 196608
int stitch_estimate_color_noalloc(const stitch_config *cfg, const uint8_t *const *frames_dev, double *M_out_dev,
                                  float *curve_out_dev, int *flags_out_dev, stitch_stream_t stream);

/*
 * Learned colour estimator. The paper estimates M only by the plain fit of
 * section 2.1 (Eq. 1-3); this part predicts it with a small network and keeps
 * the plain fit as its fallback and judge.
 *
 * Network: STITCH_MLP_IN -> 512 -> 512 -> 256 -> STITCH_MLP_OUT, bfloat16
 * weights and activations, float32 accumulation, ReLU after every layer but
 * the last. Input (features) per overlap pair: bfloat16, the three channel
 * histograms of side i then of side j, each bin scaled by 256 / pixel count
 * (so a flat histogram reads 1). Output (targets) per pair, float32:
 * M - I (9, row-major, row-vector convention of Eq. 4) then, per channel,
 * the span (m2 - m1) / 255 of the lambda-quantile knots (section 2.2) of the
 * pair's pooled histograms. The network works on targets normalised
 * per output, t_n = (t - mu) / sd (stitch_mlp_set_norm).
 *
 * Parameters (stitch_mlp_get_params / set_params): float32, layer by layer,
 * each layer W [out][in] row-major then b [out]; the last layer is stored
 * padded to 16 outputs (rows 12..15 are zero and stay zero).
 * stitch_mlp_n_params() gives the total count.
 */
#define STITCH_MLP_IN 1536
#define STITCH_MLP_OUT 12
typedef struct stitch_mlp stitch_mlp;

int stitch_mlp_n_params(void);

/* GEMM engines of the network's batched layers (training, and inference on
 * more than 16 rows; up to 16 rows use a small-batch mma.sync kernel):
 * tcgen05 (5th-generation tensor cores, accumulators in tensor memory; the
 * default) or mma.sync (warp-level tensor-core instructions). Both compute
 * in bfloat16 with float32 accumulation. */
#define STITCH_MLP_GEMM_MMA_SYNC 0
#define STITCH_MLP_GEMM_TCGEN05 1
int stitch_mlp_set_gemm(stitch_mlp *mlp, int engine);

/* Synchronise and report the network's device error word: STITCH_ETIMEOUT
 * if a bounded tensor-core wait ran out since the last report (the affected
 * outputs are not valid), else STITCH_OK. stitch_mlp_gradients and
 * stitch_mlp_get_params report it too. When the final drain of a GEMM's
 * MMAs ran out, the kernel keeps those MMAs' TMEM columns (freeing them could
 * hand a later block columns that are still being written): from then on
 * the condition is sticky -- every later call of this function returns
 * STITCH_ETIMEOUT, the tcgen05 GEMM kernel returns without work, and
 * stitch_mlp_forward / train_step / gradients refuse the tcgen05 engine
 * with STITCH_ETIMEOUT until the network is destroyed; the mma.sync engine
 * (stitch_mlp_set_gemm) stays usable. */
int stitch_mlp_status(stitch_mlp *mlp);

/* Failure detection without a device fault: writes `word` (0..3) into the
 * network's device error word as a timed-out kernel would (bit 0: a wait ran
 * out; bit 2 with bit 0 = 3: a drain ran out). The next stitch_mlp_status
 * reports it. For tests of the status handling; the paper has no counterpart.
 * Returns STITCH_OK, STITCH_EINVAL or STITCH_ECUDA. */
int stitch_mlp_inject_error(stitch_mlp *mlp, int word);

/* Diagnostic of the library's bounded device waits (failure detection
 * without a fault): one thread polls an mbarrier with the same bounded loop
 * the tensor-core GEMM uses, `limit` polls at most (1 .. 2^22). With
 * arrive = 0 nothing ever arrives, the wait gives up and the call returns
 * STITCH_ETIMEOUT with the device still usable; with arrive = 1 the arrival
 * comes first and the call returns STITCH_OK. Synchronous. */
int stitch_selftest_wait(int arrive, int limit);

/* Create a network with He-normal weights drawn from `seed` (a host
 * Mersenne-Twister stream) and buffers for batches up to max_batch (a
 * multiple of 32, at most 65536). Allocates device memory; synchronises. */
int stitch_mlp_create(int max_batch, unsigned long long seed, stitch_mlp **out);
void stitch_mlp_destroy(stitch_mlp *mlp);

/* Target normalisation: mu_host and sd_host hold STITCH_MLP_OUT floats
 * (sd > 0). Synchronous. Default: mu = 0, sd = 1. */
int stitch_mlp_set_norm(stitch_mlp *mlp, const float *mu_host, const float *sd_host);

/* Copy all parameters to / from a host buffer of stitch_mlp_n_params()
 * floats (layout above). Synchronous. */
int stitch_mlp_get_params(stitch_mlp *mlp, float *params_host);
int stitch_mlp_set_params(stitch_mlp *mlp, const float *params_host);

/* Inference: x_dev = batch x STITCH_MLP_IN bfloat16 (raw 16-bit patterns,
 * 16-byte aligned), y_dev = batch x STITCH_MLP_OUT float32 in target units
 * (de-normalised). 1 <= batch <= max_batch. Asynchronous on `stream`. */
int stitch_mlp_forward(stitch_mlp *mlp, const uint16_t *x_dev, int batch, float *y_dev, stitch_stream_t stream);

/* One training step: forward, mean squared error over the normalised
 * targets (t_dev: batch x STITCH_MLP_OUT float32, target units), backward,
 * Adam (beta 0.9 / 0.999, eps 1e-8, bias-corrected) on the float32 master
 * parameters, then the bfloat16 copies are refreshed. batch: a multiple of
 * 32 up to max_batch. loss_dev (optional): one float, the batch loss before
 * the update. Asynchronous on `stream`. */
int stitch_mlp_train_step(stitch_mlp *mlp, const uint16_t *x_dev, const float *t_dev, int batch, float lr,
                          float *loss_dev, stitch_stream_t stream);

/* Gradients of the batch loss with respect to every parameter (same layout
 * as the parameters), for checking the backward pass; no update. Synchronous
 * (legacy default stream). */
int stitch_mlp_gradients(stitch_mlp *mlp, const uint16_t *x_dev, const float *t_dev, int batch, float *grads_host,
                         float *loss_host);

/*
 * stitch_pairs_label -- plain estimate of many independent overlap pairs (the
 * training labeller): per pair the one-frame fit of section 2.1 (spec LUT,
 * Eq. 3 solved in float64; cond_1(A) > 1e12 or an empty side gives I and a
 * flag), the features above and the targets above.
 *   pairs_dev:    n_pairs x 2 x patch_h x patch_w x 3 bytes: per pair the side
 *                 i patch then the side j patch, packed RGB.
 *   lambda:       balance quantile, 0 < lambda < 0.5.
 *   features_dev: n_pairs x STITCH_MLP_IN bfloat16 (written).
 *   targets_dev:  n_pairs x STITCH_MLP_OUT float32 (written).
 *   M_dev, flags_dev: optional, n_pairs x 9 doubles and n_pairs ints.
 * Asynchronous on `stream`.
 */
int stitch_pairs_label(const uint8_t *pairs_dev, int n_pairs, int patch_w, int patch_h, double lambda,
                       uint16_t *features_dev, float *targets_dev, double *M_dev, int *flags_dev,
                       stitch_stream_t stream);

/*
 * stitch_attach_mlp -- give a context (created with STITCH_LEARNED) the
 * network it predicts M with; NULL detaches. The context does not own the
 * network: keep it alive while the context may use it. With a network
 * attached, each colour estimate also forms the window-pooled features of
 * every pair, runs the network and forms its residual: the relative excess of
 * Eq. 2's least-squares error over the window's plain fit M* = A^-1 B,
 * r = ||X (M_hat - M*)||^2 / ||X M*||^2 = tr(D^T A D) / tr(M*^T A M*) with
 * D = M_hat - M* and the window's exact A = X^T X; a pair whose plain fit
 * succeeded and whose r <= 1e-3 (transferred colours within about 3 % RMS of
 * the plain fit's) takes M_hat, any other pair keeps the plain fit. The balance
 * curve always comes from the plain estimate (its knots are exact integer
 * quantiles). Without a network a STITCH_LEARNED context behaves as a plain
 * one.
 */
int stitch_attach_mlp(stitch_ctx *ctx, stitch_mlp *mlp);

/* Counts since stitch_init: pair estimates that used the network's M, and
 * pair estimates that fell back to the plain fit. Synchronises the context's
 * work. */
int stitch_learned_stats(stitch_ctx *ctx, long long *n_learned, long long *n_fallback);

/* The latest learned estimate of every pair (n_pairs entries each, any may
 * be NULL): the network's M_hat (9 doubles, row-major), its residual r and
 * whether the pair took it (1) or kept the plain fit (0). STITCH_LEARNED
 * contexts only. Synchronises the context's work. */
int stitch_get_learned(stitch_ctx *ctx, double *M_hat, double *resid, int *used);

/*
 * Fuse tile shapes and their autotuner. The paper fixes no tiling; the fuse
 * kernel (pre-warped band remap, colour transfer, blend, balance) runs one
 * thread block per panorama tile, and the best tile shape depends on the
 * rig's resolution. Shapes: 0 = 64 x 32 (default), 1 = 64 x 16, 2 = 32 x 32,
 * 3 = 128 x 16 panorama pixels.
 *
 * stitch_autotune times the fuse of one frame (after the band pre-warp of
 * that frame) with every shape that fits the rig (a tile may touch at most
 * one blend band), `reps` launches each, keeps the fastest in the context
 * (shape 0 unless another is more than 5 % faster: the fuse timed alone is
 * only a proxy for the overlapped sequence of frames, so small differences
 * are not trusted) and
 * records it: for the rest of the process, and in the file named by the
 * environment variable STITCH_TUNE_CACHE when set, keyed by the GPU model,
 * the rig geometry and STITCH_FP16_INTERMEDIATE. stitch_init picks up a
 * recorded shape for the same key. Arguments as stitch_frame (the panorama is
 * written); the frame uses the latest colour estimate. ms_out (optional):
 * STITCH_TILE_SHAPES floats, the mean ms per fuse launch of each shape, -1
 * for a shape that does not fit. Synchronous.
 */
/* The shapes, by index (width x height in panorama pixels; 2 to 16 pixels
 * per thread of a 256-thread block): 64 x 32 (the default), 64 x 16, 32 x 32,
 * 128 x 16, 32 x 16, 128 x 32. */
#define STITCH_TILE_SHAPES 6
int stitch_autotune(stitch_ctx *ctx, const uint8_t *const *frames_dev, const float *const *flow_ij_dev,
                    const float *const *flow_ji_dev, uint8_t *pano_dev, int reps, int *shape_out, float *ms_out);

/* The context's fuse tile shape: returns its index (or -1 for NULL) and
 * writes the width and height in pixels (either pointer may be NULL). */
/* Set the fuse tile shape by hand (STITCH_EINVAL if it does not fit the rig).
 * Synchronises; recorded sequences are recorded again. */
int stitch_set_tile_shape(stitch_ctx *ctx, int shape);
int stitch_tile_shape(const stitch_ctx *ctx, int *tile_w, int *tile_h);

/*
 * Batched launch of several independent rigs (streams of uneven geometry).
 * A batch drives up to STITCH_BATCH_MAX_RIGS contexts together: every frame
 * runs each rig's statistics and estimate, then ONE band pre-warp launch and
 * two persistent fuse launches over the tiles of all rigs (band and partly
 * covered tiles, then the fully covered ones; blocks take tiles from a work
 * counter, band tiles first), recorded in a CUDA graph and
 * replayed like stitch_sequence. Every rig's tiles keep that rig's own tile
 * shape: at creation the shape recorded for the rig in a batched launch (see
 * stitch_batch_autotune), else the shape its context runs with. The paper
 * stitches one rig; this is the serving form. The contexts keep their own
 * state and may still be used alone between batch calls. All contexts must
 * share the device and the STITCH_FP16_INTERMEDIATE flag. The batch does not
 * own the contexts: destroy the batch first. A batch of one rig has no
 * cross-rig work to merge: its calls run that rig's own persistent kernels
 * (stitch_sequence at the batch's tile shape; stitch_autotune for
 * stitch_batch_autotune).
 */
#define STITCH_BATCH_MAX_RIGS 16
typedef struct stitch_batch stitch_batch;
int stitch_batch_create(stitch_ctx *const *ctxs, int n_ctx, stitch_batch **out);

/* n_frames frames of every rig. Pointer arrays are frame-major, then rig by
 * rig in the order given to stitch_batch_create: frames_dev[t * C + o_r + k]
 * with C the total camera count and o_r the cameras of the rigs before r;
 * flow_*_dev[t * P + q_r + p] likewise over pairs; pano_dev[t * R + r]. The
 * same checks and alignment rules as stitch_sequence apply. */
int stitch_batch_sequence(stitch_batch *b, int n_frames, const uint8_t *const *frames_dev,
                          const float *const *flow_ij_dev, const float *const *flow_ji_dev, uint8_t *const *pano_dev,
                          stitch_stream_t stream);

/* The batch's own tile-shape autotune over one frame of every rig (arrays as
 * stitch_batch_sequence with n_frames = 1; the panoramas are written),
 * one rig at a time: with the other rigs at their current shapes, both fuse
 * launches of the batch are timed (`reps` times each) with every shape that
 * fits rig r, and the fastest (with the same 5 % preference for shape 0) is
 * kept before the next rig. The chosen shapes
 * are recorded per rig like stitch_autotune's (process table and
 * STITCH_TUNE_CACHE), under a key marked as batched. shapes_out (optional):
 * one int per rig. ms_out (optional): n_rigs x STITCH_TILE_SHAPES floats,
 * ms_out[r * STITCH_TILE_SHAPES + s] = mean ms of the batch's fuse launches
 * with rig r at shape s, -1 where that shape does not fit. Synchronous. */
int stitch_batch_autotune(stitch_batch *b, const uint8_t *const *frames_dev, const float *const *flow_ij_dev,
                          const float *const *flow_ji_dev, uint8_t *const *pano_dev, int reps, int *shapes_out,
                          float *ms_out);
/* The batch's tile shape of every rig (n_rigs ints); returns n_rigs, or
 * STITCH_EINVAL for a NULL argument. */
int stitch_batch_tile_shapes(const stitch_batch *b, int *shapes_out);
void stitch_batch_destroy(stitch_batch *b);
const char *stitch_batch_last_error(const stitch_batch *b);

/*
 * Balance on the stitched image (STITCH_BALANCE_OUTPUT; section 2.2 balances
 * "the whole stitched image", Eq. 5-7): with this flag the knots m1, m2 of
 * frame T come from the histogram of the panorama stitched for frame T - 1,
 * before its balance, instead of the pooled histogram of frame T's camera
 * frames (a one-frame lag; frame 0 is not balanced). A pixel counts when a
 * camera covers it; its channel's bin is its fused, clamped value v on the
 * output table's grid of sixteenths, q = round_half_even(16 v), binned at
 * floor((q + 8) / 16). Eq. 6-7 average the knots of the frames that have a
 * stitched predecessor (at most the last three). stitch_estimate_color and
 * stitch_frame calls must alternate (estimate of T, frame of T, estimate of
 * T + 1, ...); recorded sequences add the edge from each frame's fuse to the
 * next frame's estimate. Not available in a batch (stitch_batch_create
 * rejects such contexts).
 *
 * stitch_get_output_hist -- that histogram of the latest stitched frame
 * (before the next stitch_estimate_color consumes it): hist_out (host,
 * required) receives 3 x 256 uint32 counts, channel-major. Synchronises.
 * Returns STITCH_OK, STITCH_EINVAL (no such flag, NULL argument) or
 * STITCH_ECUDA.
 */
int stitch_get_output_hist(stitch_ctx *ctx, uint32_t *hist_out);

/* Number of adjacent pairs (n_cams - 1), or -1 for a NULL context. */
int stitch_n_pairs(const stitch_ctx *ctx);

/*
 * stitch_window_fallbacks -- diagnostic counter of the fuse and band
 * pre-warp kernels (section 3.1's pre-warp reads each tile's source window
 * from shared memory): the number of tiles, over every launch on this context
 * since stitch_init or the last reset, whose source window did not fit the
 * kernel's staging capacity (about 1.5 x the tile width by the tile height
 * + 16 rows) and therefore sampled the frame with per-pixel global loads
 * instead. Tiles whose window the frame's edge clips to under 2 x 2 pixels,
 * or with a corner behind the camera, take the per-pixel path too but are
 * not counted: there the window is not too large, only degenerate. The
 * result is the same either way; only the speed differs.
 * *count (required) receives the counter; reset != 0 clears it afterwards.
 * Synchronises the device. Returns STITCH_OK, STITCH_EINVAL or STITCH_ECUDA.
 */
int stitch_window_fallbacks(stitch_ctx *ctx, unsigned long long *count, int reset);

/*
 * stitch_last_error -- message of the last failing call on ctx, or of the
 * last failing stitch_geometry / stitch_init when ctx is NULL. The string is
 * owned by the library and valid until the next call on the same context.
 */
const char *stitch_last_error(const stitch_ctx *ctx);

/* stitch_destroy -- free the context and its device state (synchronises). */
void stitch_destroy(stitch_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* STITCH_H */
