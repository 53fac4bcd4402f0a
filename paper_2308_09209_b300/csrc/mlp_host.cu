// Host side of the learned colour estimator: the MLP object (float32 master
// weights, bfloat16 working copies and their transposes, Adam moments,
// activation buffers), its forward pass, one training step, gradient readback
// for checks, parameter I/O, and the batched pair labeller.
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "stitch_internal.h"

using bf16 = __nv_bfloat16;

namespace stitch {
cudaError_t launch_gemm_nt(const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K, const float *bias,
                           int mode, float *Cf, int ldc, bf16 *Yb, int ldy, bf16 *Yt, int ldt, cudaStream_t s);
cudaError_t launch_transpose_bf16(const bf16 *in, int rows, int cols, bf16 *out, cudaStream_t s);
cudaError_t launch_layer_small(const bf16 *X, int ldx, int batch, const bf16 *W, int N, int K, const float *bias,
                               int mode, float *Cf, int ldc, bf16 *Yb, int ldy, const float *mu, const float *sd,
                               int n_used, cudaStream_t s);
cudaError_t launch_mse(const float *y, int ldy, const float *t, int batch, int n_out, const float *mu, const float *sd,
                       bf16 *dz, bf16 *dzt, float *loss, cudaStream_t s);
cudaError_t launch_relu_bwd(const float *dx, const bf16 *y, int batch, int n, bf16 *dz, bf16 *dzt, cudaStream_t s);
cudaError_t launch_bias_grad(const bf16 *dzt, int batch, int n, float *db, cudaStream_t s);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int count, float lr, float b1, float b2, float eps,
                        float c1, float c2, cudaStream_t s);
cudaError_t launch_to_bf16(const float *w, int n_out, int n_in, bf16 *wb, bf16 *wt, cudaStream_t s);
cudaError_t launch_denorm(const float *y, int ldy, int batch, int n_out, const float *mu, const float *sd, float *out,
                          cudaStream_t s);
cudaError_t launch_pair_label(const PairParams &p, cudaStream_t s);
cudaError_t gemm_tc_setup();
cudaError_t launch_wait_selftest(int arrive, int limit, int *err, cudaStream_t s);
cudaError_t launch_gemm_tc(const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K, const float *bias,
                           int mode, float *Cf, int ldc, bf16 *Yb, int ldy, bf16 *Yt, int ldt, int *err,
                           cudaStream_t s);
void record_last_error(const std::string &msg);
}  // namespace stitch

using namespace stitch;

namespace {

constexpr int kLayers = 4;
constexpr int kIn[kLayers] = {STITCH_MLP_IN, 512, 512, 256};
constexpr int kOut[kLayers] = {512, 512, 256, 16};   // last layer padded from 12 to 16 outputs
constexpr int kOutUsed = STITCH_MLP_OUT;

size_t layer_params(int l) { return (size_t)kOut[l] * kIn[l] + kOut[l]; }

size_t total_params() {
  size_t n = 0;
  for (int l = 0; l < kLayers; ++l) n += layer_params(l);
  return n;
}

int fail(int code, const std::string &msg) {
  record_last_error(msg);
  return code;
}

}  // namespace

struct stitch_mlp {
  int max_batch = 0;
  long long step = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // float32 params, grads, Adam moments
  size_t off[kLayers] = {};                                      // parameter offset of each layer (W then b)
  bf16 *wb[kLayers] = {}, *wt[kLayers] = {};                     // bfloat16 W [out][in] and W^T [in][out]
  bf16 *xt = nullptr;                                            // X^T [1536][batch]
  bf16 *y[kLayers] = {}, *yt[kLayers] = {};                      // activations [batch][out], transposes
  float *yf = nullptr;                                           // last layer output, float32 [batch][16]
  float *dx = nullptr;                                           // float32 input gradient scratch
  bf16 *dz[kLayers] = {}, *dzt[kLayers] = {};
  float *norm = nullptr;                                         // mu[16], sd[16]
  float *loss = nullptr;
  int *err = nullptr;                                            // device error word (tensor-core waits)
  int gemm = STITCH_MLP_GEMM_TCGEN05;                            // GEMM engine of the large-batch layers
  bool tc_dead = false;                                          // a tensor-core drain timed out: engine refused
};

namespace {

void free_mlp(stitch_mlp *n) {
  cudaFree(n->p);
  cudaFree(n->g);
  cudaFree(n->m);
  cudaFree(n->v);
  cudaFree(n->xt);
  cudaFree(n->yf);
  cudaFree(n->dx);
  cudaFree(n->norm);
  cudaFree(n->loss);
  cudaFree(n->err);
  for (int l = 0; l < kLayers; ++l) {
    cudaFree(n->wb[l]);
    cudaFree(n->wt[l]);
    cudaFree(n->y[l]);
    cudaFree(n->yt[l]);
    cudaFree(n->dz[l]);
    cudaFree(n->dzt[l]);
  }
}

// C = A B^T with the network's GEMM engine (tcgen05 or mma.sync); same modes.
cudaError_t gemm(stitch_mlp *n, const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K, const float *bias,
                 int mode, float *Cf, int ldc, bf16 *Yb, int ldy, bf16 *Yt, int ldt, cudaStream_t s) {
  if (n->gemm == STITCH_MLP_GEMM_TCGEN05)
    return launch_gemm_tc(A, lda, B, ldb, M, N, K, bias, mode, Cf, ldc, Yb, ldy, Yt, ldt, n->err, s);
  return launch_gemm_nt(A, lda, B, ldb, M, N, K, bias, mode, Cf, ldc, Yb, ldy, Yt, ldt, s);
}

cudaError_t refresh_bf16(stitch_mlp *n, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < kLayers && e == cudaSuccess; ++l)
    e = launch_to_bf16(n->p + n->off[l], kOut[l], kIn[l], n->wb[l], n->wt[l], s);
  return e;
}

// Forward pass; the last layer's float32 output goes to n->yf (normalised
// units). Inference on at most 16 rows with y_out given writes the
// denormalised outputs [batch][12] to y_out directly instead (and sets
// *denormed).
cudaError_t forward(stitch_mlp *n, const bf16 *x, int batch, bool keep_xt, cudaStream_t s, float *y_out = nullptr,
                    bool *denormed = nullptr) {
  cudaError_t e = cudaSuccess;
  if (denormed) *denormed = false;
  if (keep_xt) e = launch_transpose_bf16(x, batch, kIn[0], n->xt, s);
  const bf16 *in = x;
  if (!keep_xt && batch <= 16) {
    // Inference on a few rows: the small-batch layer kernel (K split over warps).
    for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
      const float *bias = n->p + n->off[l] + (size_t)kOut[l] * kIn[l];
      if (l < kLayers - 1)
        e = launch_layer_small(in, kIn[l], batch, n->wb[l], kOut[l], kIn[l], bias, 1, nullptr, 0, n->y[l], kOut[l],
                               nullptr, nullptr, 0, s);
      else if (y_out)
        e = launch_layer_small(in, kIn[l], batch, n->wb[l], kOut[l], kIn[l], bias, 2, y_out, kOutUsed, nullptr, 0,
                               n->norm, n->norm + 16, kOutUsed, s);
      else
        e = launch_layer_small(in, kIn[l], batch, n->wb[l], kOut[l], kIn[l], bias, 0, n->yf, kOut[l], nullptr, 0,
                               nullptr, nullptr, 0, s);
      in = n->y[l];
    }
    if (e == cudaSuccess && y_out && denormed) *denormed = true;
    return e;
  }
  for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
    const float *bias = n->p + n->off[l] + (size_t)kOut[l] * kIn[l];
    if (l < kLayers - 1)
      e = gemm(n, in, kIn[l], n->wb[l], kIn[l], batch, kOut[l], kIn[l], bias, 1, nullptr, 0, n->y[l], kOut[l],
               keep_xt ? n->yt[l] : nullptr, batch, s);
    else
      e = gemm(n, in, kIn[l], n->wb[l], kIn[l], batch, kOut[l], kIn[l], bias, 0, n->yf, kOut[l], nullptr, 0, nullptr, 0,
               s);
    in = n->y[l];
  }
  return e;
}

// Backward pass after forward(keep_xt = true) and the loss gradient in dz[3]/dzt[3].
cudaError_t backward(stitch_mlp *n, const bf16 *x, int batch, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int l = kLayers - 1; l >= 0 && e == cudaSuccess; --l) {
    float *gW = n->g + n->off[l];
    float *gb = gW + (size_t)kOut[l] * kIn[l];
    const bf16 *inT = l == 0 ? n->xt : n->yt[l - 1];
    // dW[out][in] = sum_b dZ^T[out][b] X^T[in][b]
    e = gemm(n, n->dzt[l], batch, inT, batch, kOut[l], kIn[l], batch, nullptr, 0, gW, kIn[l], nullptr, 0, nullptr, 0, s);
    if (e == cudaSuccess) e = launch_bias_grad(n->dzt[l], batch, kOut[l], gb, s);
    if (e == cudaSuccess && l > 0) {
      // dX[b][in] = sum_o dZ[b][o] W^T[in][o]
      e = gemm(n, n->dz[l], kOut[l], n->wt[l], kOut[l], batch, kIn[l], kOut[l], nullptr, 0, n->dx, kIn[l], nullptr, 0,
               nullptr, 0, s);
      if (e == cudaSuccess) e = launch_relu_bwd(n->dx, n->y[l - 1], batch, kIn[l], n->dz[l - 1], n->dzt[l - 1], s);
    }
  }
  (void)x;
  return e;
}

}  // namespace

// Device error word of the network's tensor-core kernels: bit 0, a bounded
// wait ran out (cleared when reported); bit 2, a drain ran out and MMAs may
// still write their accumulators. Bit 2 is sticky on the device (the GEMM
// kernel returns at once) and here: the tcgen05 engine is refused until the
// network is destroyed (the mma.sync engine stays available).
static int take_err(stitch_mlp *n) {
  int h = 0;
  if (cudaMemcpy(&h, n->err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return STITCH_ECUDA;
  if (h & 2) n->tc_dead = true;
  if (h) {
    if (!(h & 2)) cudaMemset(n->err, 0, 4);
    record_last_error(n->tc_dead ? "a tensor-core drain timed out: the tcgen05 engine is refused on this network"
                                 : "a tensor-core wait timed out");
    return STITCH_ETIMEOUT;
  }
  return n->tc_dead ? STITCH_ETIMEOUT : STITCH_OK;
}

// The engine refuses tcgen05 work after a failed drain.
static bool engine_refused(const stitch_mlp *n) { return n->tc_dead && n->gemm == STITCH_MLP_GEMM_TCGEN05; }

extern "C" {

int stitch_mlp_n_params(void) { return (int)total_params(); }

int stitch_mlp_set_gemm(stitch_mlp *n, int engine) {
  if (!n || (engine != STITCH_MLP_GEMM_MMA_SYNC && engine != STITCH_MLP_GEMM_TCGEN05))
    return fail(STITCH_EINVAL, "mlp is NULL or unknown GEMM engine");
  n->gemm = engine;
  return STITCH_OK;
}

int stitch_mlp_inject_error(stitch_mlp *n, int word) {
  if (!n || word < 0 || word > 3) return fail(STITCH_EINVAL, "mlp is NULL or the word is not 0..3");
  const cudaError_t e = cudaMemcpy(n->err, &word, sizeof(int), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? STITCH_OK : fail(STITCH_ECUDA, cudaGetErrorString(e));
}

int stitch_mlp_status(stitch_mlp *n) {
  if (!n) return fail(STITCH_EINVAL, "mlp is NULL");
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(STITCH_ECUDA, cudaGetErrorString(e));
  return take_err(n);
}

int stitch_selftest_wait(int arrive, int limit) {
  if (limit < 1 || limit > (1 << 22)) return fail(STITCH_EINVAL, "limit must be in [1, 2^22]");
  int *err = nullptr;
  cudaError_t e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
  if (e == cudaSuccess) e = launch_wait_selftest(arrive ? 1 : 0, limit, err, nullptr);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(err);
  if (e != cudaSuccess) return fail(STITCH_ECUDA, cudaGetErrorString(e));
  return h ? fail(STITCH_ETIMEOUT, "the bounded wait gave up, as expected without an arrival") : STITCH_OK;
}

int stitch_mlp_create(int max_batch, unsigned long long seed, stitch_mlp **out) {
  if (!out) return fail(STITCH_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_batch < 32 || max_batch % 32 != 0 || max_batch > 65536)
    return fail(STITCH_EINVAL, "max_batch must be a multiple of 32 in [32, 65536]");
  stitch_mlp *n = new (std::nothrow) stitch_mlp();
  if (!n) return fail(STITCH_ENOMEM, "host allocation failed");
  n->max_batch = max_batch;
  size_t o = 0;
  for (int l = 0; l < kLayers; ++l) {
    n->off[l] = o;
    o += layer_params(l);
  }
  const size_t np = total_params();
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) e = cudaMemset(*ptr, 0, bytes);
  };
  alloc((void **)&n->p, np * 4);
  alloc((void **)&n->g, np * 4);
  alloc((void **)&n->m, np * 4);
  alloc((void **)&n->v, np * 4);
  alloc((void **)&n->xt, (size_t)kIn[0] * max_batch * 2);
  alloc((void **)&n->yf, (size_t)max_batch * 16 * 4);
  alloc((void **)&n->dx, (size_t)max_batch * 512 * 4);
  alloc((void **)&n->norm, 32 * 4);
  alloc((void **)&n->loss, 4);
  alloc((void **)&n->err, 4);
  if (e == cudaSuccess) e = gemm_tc_setup();
  for (int l = 0; l < kLayers; ++l) {
    alloc((void **)&n->wb[l], (size_t)kOut[l] * kIn[l] * 2);
    alloc((void **)&n->wt[l], (size_t)kOut[l] * kIn[l] * 2);
    alloc((void **)&n->y[l], (size_t)max_batch * kOut[l] * 2);
    alloc((void **)&n->yt[l], (size_t)max_batch * kOut[l] * 2);
    alloc((void **)&n->dz[l], (size_t)max_batch * kOut[l] * 2);
    alloc((void **)&n->dzt[l], (size_t)max_batch * kOut[l] * 2);
  }
  // He-normal weights, zero biases; the padding outputs of the last layer stay zero.
  if (e == cudaSuccess) {
    std::vector<float> h(np, 0.0f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < kLayers; ++l) {
      std::normal_distribution<float> nd(0.0f, std::sqrt(2.0f / (float)kIn[l]));
      const int rows = l == kLayers - 1 ? kOutUsed : kOut[l];
      for (int r = 0; r < rows; ++r)
        for (int k = 0; k < kIn[l]; ++k) h[n->off[l] + (size_t)r * kIn[l] + k] = nd(rng) * (l == kLayers - 1 ? 0.1f : 1.0f);
    }
    e = cudaMemcpy(n->p, h.data(), np * 4, cudaMemcpyHostToDevice);
    const float norm[32] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0,
                            1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
    if (e == cudaSuccess) e = cudaMemcpy(n->norm, norm, sizeof(norm), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = refresh_bf16(n, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_mlp(n);
    delete n;
    return fail(e == cudaErrorMemoryAllocation ? STITCH_ENOMEM : STITCH_ECUDA, cudaGetErrorString(e));
  }
  *out = n;
  return STITCH_OK;
}

void stitch_mlp_destroy(stitch_mlp *n) {
  if (!n) return;
  cudaDeviceSynchronize();
  free_mlp(n);
  delete n;
}

int stitch_mlp_set_norm(stitch_mlp *n, const float *mu, const float *sd) {
  if (!n || !mu || !sd) return fail(STITCH_EINVAL, "mlp, mu and sd are required");
  float h[32];
  for (int i = 0; i < 16; ++i) {
    h[i] = i < kOutUsed ? mu[i] : 0.0f;
    h[16 + i] = i < kOutUsed ? sd[i] : 1.0f;
    if (!(h[16 + i] > 0.0f)) return fail(STITCH_EINVAL, "sd must be positive");
  }
  const cudaError_t e = cudaMemcpy(n->norm, h, sizeof(h), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? STITCH_OK : fail(STITCH_ECUDA, cudaGetErrorString(e));
}

int stitch_mlp_get_params(stitch_mlp *n, float *host) {
  if (!n || !host) return fail(STITCH_EINVAL, "mlp and host buffer are required");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(host, n->p, total_params() * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(STITCH_ECUDA, cudaGetErrorString(e));
  return take_err(n);
}

int stitch_mlp_set_params(stitch_mlp *n, const float *host) {
  if (!n || !host) return fail(STITCH_EINVAL, "mlp and host buffer are required");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(n->p, host, total_params() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = refresh_bf16(n, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? STITCH_OK : fail(STITCH_ECUDA, cudaGetErrorString(e));
}

int stitch_mlp_forward(stitch_mlp *n, const uint16_t *x_dev, int batch, float *y_dev, stitch_stream_t stream) {
  if (!n || !x_dev || !y_dev) return fail(STITCH_EINVAL, "mlp, x and y are required");
  if (batch < 1 || batch > n->max_batch) return fail(STITCH_EINVAL, "batch out of range");
  if (reinterpret_cast<uintptr_t>(x_dev) & 15u) return fail(STITCH_EINVAL, "x must be 16-byte aligned");
  if (engine_refused(n)) return fail(STITCH_ETIMEOUT, "the tcgen05 engine is refused after a drain timed out");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  bool denormed = false;
  cudaError_t e = forward(n, reinterpret_cast<const bf16 *>(x_dev), batch, false, s, y_dev, &denormed);
  if (e == cudaSuccess && !denormed) e = launch_denorm(n->yf, 16, batch, kOutUsed, n->norm, n->norm + 16, y_dev, s);
  return e == cudaSuccess ? STITCH_OK : fail(STITCH_ECUDA, cudaGetErrorString(e));
}

// Forward, MSE on normalised targets, backward; gradients land in n->g.
static cudaError_t grads(stitch_mlp *n, const bf16 *x, const float *t, int batch, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(n->loss, 0, 4, s);
  if (e == cudaSuccess) e = forward(n, x, batch, true, s);
  if (e == cudaSuccess)
    e = launch_mse(n->yf, 16, t, batch, kOutUsed, n->norm, n->norm + 16, n->dz[kLayers - 1], n->dzt[kLayers - 1],
                   n->loss, s);
  if (e == cudaSuccess) e = backward(n, x, batch, s);
  return e;
}

int stitch_mlp_train_step(stitch_mlp *n, const uint16_t *x_dev, const float *t_dev, int batch, float lr,
                          float *loss_dev, stitch_stream_t stream) {
  if (!n || !x_dev || !t_dev) return fail(STITCH_EINVAL, "mlp, x and targets are required");
  if (batch < 32 || batch % 32 != 0 || batch > n->max_batch)
    return fail(STITCH_EINVAL, "batch must be a multiple of 32 up to max_batch");
  if (engine_refused(n)) return fail(STITCH_ETIMEOUT, "the tcgen05 engine is refused after a drain timed out");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = grads(n, reinterpret_cast<const bf16 *>(x_dev), t_dev, batch, s);
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)n->step), c2 = 1.0f - std::pow(b2, (float)n->step);
  if (e == cudaSuccess) e = launch_adam(n->p, n->g, n->m, n->v, (int)total_params(), lr, b1, b2, 1e-8f, c1, c2, s);
  if (e == cudaSuccess) e = refresh_bf16(n, s);
  if (e == cudaSuccess && loss_dev) e = cudaMemcpyAsync(loss_dev, n->loss, 4, cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? STITCH_OK : fail(STITCH_ECUDA, cudaGetErrorString(e));
}

int stitch_mlp_gradients(stitch_mlp *n, const uint16_t *x_dev, const float *t_dev, int batch, float *grads_host,
                         float *loss_host) {
  if (!n || !x_dev || !t_dev || !grads_host) return fail(STITCH_EINVAL, "mlp, x, targets and output are required");
  if (batch < 32 || batch % 32 != 0 || batch > n->max_batch)
    return fail(STITCH_EINVAL, "batch must be a multiple of 32 up to max_batch");
  if (engine_refused(n)) return fail(STITCH_ETIMEOUT, "the tcgen05 engine is refused after a drain timed out");
  cudaError_t e = grads(n, reinterpret_cast<const bf16 *>(x_dev), t_dev, batch, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(grads_host, n->g, total_params() * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && loss_host) e = cudaMemcpy(loss_host, n->loss, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(STITCH_ECUDA, cudaGetErrorString(e));
  return take_err(n);
}

int stitch_pairs_label(const uint8_t *pairs_dev, int n_pairs, int patch_w, int patch_h, double lambda,
                       uint16_t *features_dev, float *targets_dev, double *M_dev, int *flags_dev,
                       stitch_stream_t stream) {
  if (!pairs_dev || !features_dev || !targets_dev) return fail(STITCH_EINVAL, "pairs, features and targets are required");
  if (n_pairs < 0 || patch_w < 1 || patch_h < 1 || (long long)patch_w * patch_h > (1ll << 24))
    return fail(STITCH_EINVAL, "bad pair count or patch size");
  const long long lq = std::llround(lambda * 1e6);
  if (lq <= 0 || lq >= 500000) return fail(STITCH_EINVAL, "lambda must be in (0, 0.5)");
  PairParams p{};
  p.pairs = pairs_dev;
  p.n = n_pairs;
  p.pw = patch_w;
  p.ph = patch_h;
  p.lambda_q = lq;
  p.feat = reinterpret_cast<bf16 *>(features_dev);
  p.targ = targets_dev;
  p.M = M_dev;
  p.flags = flags_dev;
  const cudaError_t e = launch_pair_label(p, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? STITCH_OK : fail(STITCH_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"
