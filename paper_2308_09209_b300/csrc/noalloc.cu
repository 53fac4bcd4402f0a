// Single-frame colour estimate that allocates no device memory.
//
// Some callers cannot call cudaMalloc: plugins whose host application owns
// every device allocation (a fixed memory pool handed out by the host, or a
// budget enforced by a media framework), code running under a stream
// capture that forbids allocation, or real-time threads that must never
// block in the driver's allocator. stitch_estimate_color_noalloc serves them:
// it runs the same statistics and estimate kernels as stitch_estimate_color,
// but its working memory (one raw-statistics slot and one colour state) is
// a file-scope __device__ array of fixed size, which the CUDA module loader
// places on every GPU that loads this library; it stays there until the
// process exits. The caller passes the frames and the output buffers.
#include <mutex>
#include <string>

#include "stitch_internal.h"

namespace stitch {
namespace {

constexpr size_t kRawBytes = sizeof(RawStats);
constexpr size_t kScratchBytes = ((kRawBytes + sizeof(ColorState)) + 255) / 256 * 256;
static_assert(kScratchBytes <= STITCH_NOALLOC_SCRATCH_BYTES, "scratch larger than the advertised size");

// The scratch. In host code this name is only a stand-in for the device
// symbol, never a device address: host code passes the address obtained from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[STITCH_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// The colour state must start as "no frame seen, every M the identity".
__global__ void k_noalloc_reset(ColorState *S) {
  const int t = threadIdx.x;
  if (t < kMaxPairs * 9) S->M_pair[t / 9][t % 9] = (t % 9 % 4 == 0) ? 1.0 : 0.0;
  if (t < kMaxCams * 9) S->M_cam[t / 9][t % 9] = (t % 9 % 4 == 0) ? 1.0 : 0.0;
}

// Copy the estimate of the single frame (colour slot 0) to the caller.
__global__ void k_noalloc_out(const ColorState *S, int n_cams, double *M_out, float *curve_out, int *flags_out) {
  const int t = threadIdx.x;
  if (t < n_cams * 9) M_out[t] = S->M_cam[t / 9][t % 9];
  if (t < 3 * STITCH_CURVE_FLOATS) {
    const float *c = reinterpret_cast<const float *>(&S->out[0].curve[t / STITCH_CURVE_FLOATS]);
    curve_out[t] = c[t % STITCH_CURVE_FLOATS];
  }
  if (t == 0 && flags_out) *flags_out = S->singular_last;
}

int fail(int code, const char *msg) {
  record_last_error(msg);
  return code;
}

}  // namespace
}  // namespace stitch

using namespace stitch;

extern "C" int stitch_estimate_color_noalloc(const stitch_config *cfg, const uint8_t *const *frames_dev,
                                             double *M_out_dev, float *curve_out_dev, int *flags_out_dev,
                                             stitch_stream_t stream) {
  if (!cfg) return fail(STITCH_EINVAL, "config is NULL");
  if (cfg->n_cams > STITCH_NOALLOC_MAX_CAMS)
    return fail(STITCH_EINVAL, "n_cams exceeds the no-allocation scratch (at most 8 cameras)");
  if (!frames_dev || !M_out_dev || !curve_out_dev) return fail(STITCH_EINVAL, "frames and outputs are required");
  StatsParams sp;
  EstimateParams ep;
  int grid_x = 1;
  std::string err;
  int rc = prepare_estimate_params(cfg, sp, grid_x, ep, err);
  if (rc != STITCH_OK) return fail(rc, err.c_str());
  for (int k = 0; k < sp.n_cams; ++k)
    if (!frames_dev[k]) return fail(STITCH_EINVAL, "frames_dev must hold n_cams non-NULL pointers");

  // One-time set-up per device, with that device current.
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(STITCH_ECUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) return fail(STITCH_EINVAL, "device ordinal out of range");
  unsigned char *scratch = nullptr;
  {
    // The address is looked up on the device's first call, and again on any
    // call whose stream is not being captured: a cudaDeviceReset reloads the
    // library's device image, possibly at another address (the set-up is
    // then redone too). A capturing call uses the cached address.
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(reinterpret_cast<cudaStream_t>(stream), &cs) != cudaSuccess ||
                           cs != cudaStreamCaptureStatusNone;
    if (!g_scratch_addr[dev] || !capturing) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return fail(STITCH_ECUDA, "cudaGetSymbolAddress of the scratch failed");
      if (p != g_scratch_addr[dev]) {
        e = estimate_setup();
        if (e != cudaSuccess) return fail(STITCH_ECUDA, "estimate kernel set-up failed");
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
      }
    }
    scratch = g_scratch_addr[dev];
  }

  RawStats *raw = reinterpret_cast<RawStats *>(scratch);
  ColorState *state = reinterpret_cast<ColorState *>(scratch + kRawBytes);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // The previous call's contents are still there: clear the statistics slots
  // and the colour state (frame index 0, empty rings), then set every M to I.
  e = cudaMemsetAsync(scratch, 0, kRawBytes + sizeof(ColorState), s);
  if (e != cudaSuccess) return fail(STITCH_ECUDA, "clearing the scratch failed");
  k_noalloc_reset<<<1, 128, 0, s>>>(state);
  for (int k = 0; k < sp.n_cams; ++k) {
    sp.src[k] = frames_dev[k];
    sp.vec_ok[k] = ((reinterpret_cast<uintptr_t>(frames_dev[k]) & 15u) == 0 && sp.pitch[k] % 16 == 0) ? 1 : 0;
  }
  sp.raw = raw;
  ep.raw = raw;
  ep.raw_slots = 1;
  ep.state = state;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_stats(sp, grid_x, s);
  if (e == cudaSuccess) e = launch_estimate(ep, s);
  if (e == cudaSuccess) {
    k_noalloc_out<<<1, 128, 0, s>>>(state, sp.n_cams, M_out_dev, curve_out_dev, flags_out_dev);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return fail(STITCH_ECUDA, cudaGetErrorString(e));
  return STITCH_OK;
}
