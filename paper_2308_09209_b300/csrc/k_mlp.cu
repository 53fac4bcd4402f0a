// Kernels of the learned colour estimator: a 1536 -> 512 -> 512 -> 256 -> 12
// MLP in bfloat16 with float32 accumulation and ReLU (none after the last
// layer), trained with its own forward and backward kernels.
//
// All products are one "NT" GEMM, C[m][n] = sum_k A[m][k] B[n][k], with both
// operands K-contiguous bfloat16 and float32 accumulation on the tensor cores
// (mma.sync m16n8k16, fragments loaded with ldmatrix from padded shared-memory
// tiles). Forward: Y = act(X W^T + b) with W stored [out][in]. Backward: the
// weight gradient dW = dZ^T X and the input gradient dX = dZ W, both in NT
// form by keeping transposed copies (X^T, Y^T, dZ^T, W^T).
#include <cuda_bf16.h>

#include "stitch_internal.h"

namespace stitch {

namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 64, BN = 64, BK = 32, LDS_K = BK + 8;   // padded rows: conflict-free ldmatrix
constexpr int kGemmThreads = 128;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Load a BM x BK (or BN x BK) tile of a K-contiguous matrix into shared
// memory, zero outside [0, rows) x [0, K). K is a multiple of 8.
__device__ __forceinline__ void load_tile(bf16 (*s)[LDS_K], const bf16 *__restrict__ g, int ld, int row0, int rows,
                                          int k0, int K) {
  // 64 rows x 4 chunks of 8 elements = 256 chunks, 2 per thread
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int c = threadIdx.x + it * kGemmThreads;
    const int r = c >> 2, q = c & 3;
    const int gr = row0 + r, gk = k0 + 8 * q;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gr < rows && gk < K) v = *reinterpret_cast<const uint4 *>(g + (size_t)gr * ld + gk);
    *reinterpret_cast<uint4 *>(&s[r][8 * q]) = v;
  }
}

}  // namespace

// mode 0: C (float32) = acc (+ bias[n] if bias) ; mode 1: Yb (bfloat16) = relu(acc + bias[n]), optionally Yt[n][m]
__global__ void __launch_bounds__(kGemmThreads) k_gemm_nt(const bf16 *__restrict__ A, int lda, const bf16 *__restrict__ B,
                                                          int ldb, int M, int N, int K, const float *__restrict__ bias,
                                                          int mode, float *Cf, int ldc, bf16 *Yb, int ldy, bf16 *Yt,
                                                          int ldt) {
  __shared__ __align__(16) bf16 As[BM][LDS_K];
  __shared__ __align__(16) bf16 Bs[BN][LDS_K];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = warp >> 1, wn = warp & 1;      // 2 x 2 warps, 32 x 32 each
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;

  for (int k0 = 0; k0 < K; k0 += BK) {
    load_tile(As, A, lda, m0, M, k0, K);
    load_tile(Bs, B, ldb, n0, N, k0, K);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int row = wm * 32 + i * 16 + (lane & 7) + 8 * ((lane >> 3) & 1);
        const int col = kk + 8 * (lane >> 4);
        ldmatrix_x4(smem_u32(&As[row][col]), af[i][0], af[i][1], af[i][2], af[i][3]);
      }
      uint32_t bfr[4][2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int row = wn * 32 + j * 16 + (lane & 7) + 8 * (lane >> 4);
        const int col = kk + 8 * ((lane >> 3) & 1);
        uint32_t r0, r1, r2, r3;
        ldmatrix_x4(smem_u32(&Bs[row][col]), r0, r1, r2, r3);
        bfr[2 * j][0] = r0;
        bfr[2 * j][1] = r1;
        bfr[2 * j + 1][0] = r2;
        bfr[2 * j + 1][1] = r3;
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j][0], bfr[j][1]);
    }
    __syncthreads();
  }
  // epilogue
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm * 32 + i * 16 + g + 8 * (q >> 1);
        const int n = n0 + wn * 32 + j * 8 + 2 * t + (q & 1);
        if (m >= M || n >= N) continue;
        float v = acc[i][j][q] + (bias ? bias[n] : 0.0f);
        if (mode == 0) {
          Cf[(size_t)m * ldc + n] = v;
        } else {
          v = fmaxf(v, 0.0f);
          const bf16 h = __float2bfloat16_rn(v);
          Yb[(size_t)m * ldy + n] = h;
          if (Yt) Yt[(size_t)n * ldt + m] = h;
        }
      }
}

// One layer for a small batch (at most 16 rows, e.g. the pairs of one rig at
// inference): Y = act(X W^T + b). Block b owns output columns [8 b, 8 b + 8);
// its sixteen warps split K into sixteen ranges and each runs one m16n8k16
// tile (rows >= batch read as zero) with fragments loaded straight from
// global memory (X is a few KB and stays in L1; each k-step reads one 32-byte
// sector of eight W rows). With at most six k-steps per warp, all of a
// block's weight loads are in flight at once: the layer costs about one
// memory latency. The sixteen partial tiles are summed in a fixed order in
// shared memory, so results do not depend on scheduling.
constexpr int kSmallWarps = 16;
constexpr int kSmallThreads = 32 * kSmallWarps;

__global__ void __launch_bounds__(kSmallThreads) k_layer_small(const bf16 *__restrict__ X, int ldx, int batch,
                                                                 const bf16 *__restrict__ W, int N, int K,
                                                                 const float *__restrict__ bias, int mode, float *Cf,
                                                                 int ldc, bf16 *Yb, int ldy,
                                                                 const float *__restrict__ mu,
                                                                 const float *__restrict__ sd, int n_used) {
  __shared__ float part[kSmallWarps][16][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int n0 = blockIdx.x * 8;
  const int ksteps = K / 16, per = (ksteps + kSmallWarps - 1) / kSmallWarps;
  const int k_lo = warp * per, k_hi = min(ksteps, k_lo + per);
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const bool r0 = g < batch, r1 = g + 8 < batch;
  const bool nok = n0 + g < N;
  const uint32_t *xa = reinterpret_cast<const uint32_t *>(X + (size_t)g * ldx);
  const uint32_t *xb = reinterpret_cast<const uint32_t *>(X + (size_t)(g + 8) * ldx);
  const uint32_t *wr = reinterpret_cast<const uint32_t *>(W + (size_t)(n0 + g) * K);
#pragma unroll 6
  for (int ks = k_lo; ks < k_hi; ++ks) {
    const int c = (ks * 16) / 2 + t;            // 32-bit word of columns 2t, 2t+1 of this k-step
    uint32_t a[4];
    a[0] = r0 ? __ldg(xa + c) : 0u;
    a[1] = r1 ? __ldg(xb + c) : 0u;
    a[2] = r0 ? __ldg(xa + c + 4) : 0u;
    a[3] = r1 ? __ldg(xb + c + 4) : 0u;
    const uint32_t b0 = nok ? __ldg(wr + c) : 0u;
    const uint32_t b1 = nok ? __ldg(wr + c + 4) : 0u;
    mma_bf16(acc, a, b0, b1);
  }
  // accumulator layout of m16n8: (row g, cols 2t, 2t+1) and (row g+8, same cols)
  part[warp][g][2 * t] = acc[0];
  part[warp][g][2 * t + 1] = acc[1];
  part[warp][g + 8][2 * t] = acc[2];
  part[warp][g + 8][2 * t + 1] = acc[3];
  __syncthreads();
  const int m = threadIdx.x >> 3, n = threadIdx.x & 7;   // the first 128 threads: 16 rows x 8 columns
  if (threadIdx.x < 128 && m < batch && n0 + n < N) {
    float v = part[0][m][n];
#pragma unroll
    for (int w = 1; w < kSmallWarps; ++w) v += part[w][m][n];
    if (bias) v += bias[n0 + n];
    if (mode == 0) {
      Cf[(size_t)m * ldc + n0 + n] = v;
    } else if (mode == 2) {
      // denormalised output of the last layer: v sd + mu, columns below n_used
      if (n0 + n < n_used) Cf[(size_t)m * ldc + n0 + n] = fmaf(v, sd[n0 + n], mu[n0 + n]);
    } else {
      Yb[(size_t)m * ldy + n0 + n] = __float2bfloat16_rn(fmaxf(v, 0.0f));
    }
  }
}

// Transpose a [rows][cols] bfloat16 matrix into [cols][rows].
__global__ void k_transpose_bf16(const bf16 *__restrict__ in, int rows, int cols, bf16 *__restrict__ out) {
  __shared__ bf16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = in[(size_t)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(size_t)c * rows + r] = tile[threadIdx.x][i];
  }
}

// Loss on the first n_out of ldy outputs: normalised targets t_norm = (t - mu) / sd,
// mean squared error over batch x n_out; dY = 2 (y - t_norm) / (batch n_out) in
// bfloat16 (both layouts), zero for the padding outputs. Loss partial sums go
// to loss[0] (float, accumulated with atomics).
__global__ void k_mse(const float *__restrict__ y, int ldy, const float *__restrict__ t, int batch, int n_out,
                      const float *__restrict__ mu, const float *__restrict__ sd, bf16 *dz, bf16 *dzt, float *loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (i < batch * ldy) {
    const int b = i / ldy, n = i % ldy;
    float d = 0.0f;
    if (n < n_out) {
      const float tn = (t[(size_t)b * n_out + n] - mu[n]) / sd[n];
      d = y[(size_t)b * ldy + n] - tn;
      l = d * d;
    }
    const bf16 gz = __float2bfloat16_rn(2.0f * d / (float)(batch * n_out));
    dz[(size_t)b * ldy + n] = gz;
    dzt[(size_t)n * batch + b] = gz;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, l / (float)(batch * n_out));
}

// dZ = dX * (Y > 0) in bfloat16, both layouts ([batch][n] and [n][batch]).
__global__ void k_relu_bwd(const float *__restrict__ dx, const bf16 *__restrict__ y, int batch, int n, bf16 *dz,
                           bf16 *dzt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch * n) return;
  const int b = i / n, c = i % n;
  const float v = __bfloat162float(y[i]) > 0.0f ? dx[i] : 0.0f;
  const bf16 h = __float2bfloat16_rn(v);
  dz[i] = h;
  dzt[(size_t)c * batch + b] = h;
}

// Bias gradient: db[n] = sum_b dZ[b][n] (from the transposed copy, one warp per n).
__global__ void k_bias_grad(const bf16 *__restrict__ dzt, int batch, int n, float *db) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= n) return;
  float s = 0.0f;
  for (int b = lane; b < batch; b += 32) s += __bfloat162float(dzt[(size_t)w * batch + b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) db[w] = s;
}

// Adam on float32 master parameters; refreshes the bfloat16 copy of weights
// (and its transpose) when wb is given. Parameters of a layer: W [n_out][n_in]
// then b [n_out] in one contiguous block.
__global__ void k_adam(float *p, const float *__restrict__ g, float *m, float *v, int count, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_to_bf16(const float *__restrict__ w, int n_out, int n_in, bf16 *wb, bf16 *wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_out * n_in) return;
  const int o = i / n_in, k = i % n_in;
  const bf16 h = __float2bfloat16_rn(w[i]);
  wb[i] = h;
  wt[(size_t)k * n_out + o] = h;
}

// y_out[b][n] = y_norm[b][n] * sd[n] + mu[n] for the first n_out outputs.
__global__ void k_denorm(const float *__restrict__ y, int ldy, int batch, int n_out, const float *__restrict__ mu,
                         const float *__restrict__ sd, float *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch * n_out) return;
  const int b = i / n_out, n = i % n_out;
  out[i] = fmaf(y[(size_t)b * ldy + n], sd[n], mu[n]);
}

cudaError_t launch_gemm_nt(const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K, const float *bias,
                           int mode, float *Cf, int ldc, bf16 *Yb, int ldy, bf16 *Yt, int ldt, cudaStream_t s) {
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  k_gemm_nt<<<grid, kGemmThreads, 0, s>>>(A, lda, B, ldb, M, N, K, bias, mode, Cf, ldc, Yb, ldy, Yt, ldt);
  return cudaGetLastError();
}

cudaError_t launch_layer_small(const bf16 *X, int ldx, int batch, const bf16 *W, int N, int K, const float *bias,
                               int mode, float *Cf, int ldc, bf16 *Yb, int ldy, const float *mu, const float *sd,
                               int n_used, cudaStream_t s) {
  if (batch < 1 || batch > 16 || K % 16 != 0) return cudaErrorInvalidValue;
  if (mode == 2 && (!mu || !sd)) return cudaErrorInvalidValue;
  k_layer_small<<<(N + 7) / 8, kSmallThreads, 0, s>>>(X, ldx, batch, W, N, K, bias, mode, Cf, ldc, Yb, ldy, mu, sd,
                                                       n_used);
  return cudaGetLastError();
}

cudaError_t launch_transpose_bf16(const bf16 *in, int rows, int cols, bf16 *out, cudaStream_t s) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  k_transpose_bf16<<<grid, dim3(32, 8), 0, s>>>(in, rows, cols, out);
  return cudaGetLastError();
}

cudaError_t launch_mse(const float *y, int ldy, const float *t, int batch, int n_out, const float *mu, const float *sd,
                       bf16 *dz, bf16 *dzt, float *loss, cudaStream_t s) {
  const int n = batch * ldy;
  k_mse<<<(n + 255) / 256, 256, 0, s>>>(y, ldy, t, batch, n_out, mu, sd, dz, dzt, loss);
  return cudaGetLastError();
}

cudaError_t launch_relu_bwd(const float *dx, const bf16 *y, int batch, int n, bf16 *dz, bf16 *dzt, cudaStream_t s) {
  k_relu_bwd<<<(batch * n + 255) / 256, 256, 0, s>>>(dx, y, batch, n, dz, dzt);
  return cudaGetLastError();
}

cudaError_t launch_bias_grad(const bf16 *dzt, int batch, int n, float *db, cudaStream_t s) {
  k_bias_grad<<<(n * 32 + 255) / 256, 256, 0, s>>>(dzt, batch, n, db);
  return cudaGetLastError();
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, int count, float lr, float b1, float b2, float eps,
                        float c1, float c2, cudaStream_t s) {
  k_adam<<<(count + 255) / 256, 256, 0, s>>>(p, g, m, v, count, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float *w, int n_out, int n_in, bf16 *wb, bf16 *wt, cudaStream_t s) {
  k_to_bf16<<<(n_out * n_in + 255) / 256, 256, 0, s>>>(w, n_out, n_in, wb, wt);
  return cudaGetLastError();
}

cudaError_t launch_denorm(const float *y, int ldy, int batch, int n_out, const float *mu, const float *sd, float *out,
                          cudaStream_t s) {
  k_denorm<<<(batch * n_out + 255) / 256, 256, 0, s>>>(y, ldy, batch, n_out, mu, sd, out);
  return cudaGetLastError();
}

}  // namespace stitch
