// One-frame colour transfer from pixel correspondences: the 2D-M method the
// paper compares its 3D-M against (Tables 2-3). For a pair with colour source
// i and target j, the corresponding pixels are the two cameras' float32
// pre-warped samples at the same panorama position over the blend band; the
// kernels form A = X^T X (six distinct entries) and B = X^T Y (nine) in
// float64, X and Y the band's samples of i and j as rows of RGB.
//
// k_corr_partial: per block a strided share of the band's pixels, each
//   thread's fifteen sums reduced over the block in a fixed tree order.
// k_corr_final:   per pair, the blocks' partial sums added in block order,
//   so the result does not depend on scheduling.
#include "stitch_internal.h"

namespace stitch {

namespace {

constexpr int kCorrThreads = 256;

__global__ void __launch_bounds__(kCorrThreads) k_corr_partial(const CorrParams P) {
  const int pair = blockIdx.y;
  const float4 *X = P.pw + P.off_i[pair];
  const float4 *Y = P.pw + P.off_j[pair];
  const int n = P.n[pair];
  double s[kCorrSums];
#pragma unroll
  for (int k = 0; k < kCorrSums; ++k) s[k] = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float4 a = __ldg(X + e), b = __ldg(Y + e);
    const double x[3] = {a.x, a.y, a.z}, y[3] = {b.x, b.y, b.z};
    // A: (0,0) (0,1) (0,2) (1,1) (1,2) (2,2); B: row-major (c, d) = x_c y_d
    s[0] += x[0] * x[0];
    s[1] += x[0] * x[1];
    s[2] += x[0] * x[2];
    s[3] += x[1] * x[1];
    s[4] += x[1] * x[2];
    s[5] += x[2] * x[2];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) s[6 + 3 * c + d] += x[c] * y[d];
  }
  __shared__ double red[kCorrThreads];
  double *out = P.partial + ((size_t)pair * gridDim.x + blockIdx.x) * kCorrSums;
  for (int k = 0; k < kCorrSums; ++k) {
    red[threadIdx.x] = s[k];
    __syncthreads();
    for (int h = kCorrThreads / 2; h > 0; h >>= 1) {
      if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = red[0];
    __syncthreads();
  }
}

__global__ void k_corr_final(const CorrParams P, int blocks) {
  const int pair = blockIdx.x, k = threadIdx.x;
  if (k >= kCorrSums) return;
  double t = 0.0;
  for (int b = 0; b < blocks; ++b) t += P.partial[((size_t)pair * blocks + b) * kCorrSums + k];
  P.sums[pair * kCorrSums + k] = t;
}

}  // namespace

cudaError_t launch_corr(const CorrParams &p, int blocks, cudaStream_t s) {
  if (p.n_pairs <= 0) return cudaSuccess;
  if (blocks < 1 || blocks > kCorrMaxBlocks) return cudaErrorInvalidValue;
  k_corr_partial<<<dim3(blocks, p.n_pairs), kCorrThreads, 0, s>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_corr_final<<<p.n_pairs, 32, 0, s>>>(p, blocks);
  return cudaGetLastError();
}

}  // namespace stitch
