// The learned estimator's GEMMs on the 5th-generation tensor cores:
// C[m][n] = sum_k A[m][k] B[n][k] (both operands K-contiguous bfloat16),
// float32 accumulation in tensor memory.
//
// One CTA (128 threads) owns a 128 x 32 tile of C. K advances 64 at a time
// through a ring of kStages shared-memory stages: all threads copy a stage
// (A: 128 x 64, B: 32 x 64) from global memory with cp.async into the
// canonical K-major layout without swizzle (8-row x 16-byte core matrices;
// core matrices adjacent along K are 128 bytes apart, 8-row groups 1024 bytes
// apart), one thread issues four tcgen05.mma (M = 128, N = 32, K = 16 each)
// into the tile's 32 tensor-memory columns and commits them to the stage's
// mbarrier. Copies run kAhead tiles ahead of the MMAs, and a stage is only
// refilled once the MMAs that read it (kStages - kAhead tiles earlier) are
// done, so neither the copy latency nor the MMA latency is waited on in
// step. The epilogue reads the
// accumulators with tcgen05.ld (warp w owns rows 32w..32w+31) and applies
// the same modes as k_gemm_nt: float32 out (+bias), or ReLU(acc + bias) to
// bfloat16 (and optionally its transpose).
//
// Every mbarrier wait is bounded; a wait that runs out sets *err, drains
// (again bounded) and frees the tensor memory before the CTA returns.
#include <cuda_bf16.h>

#include "stitch_internal.h"

namespace stitch {

namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 128, BN = 32, BK = 64;
constexpr int kThreads = 128;
constexpr int kTileA = BM * BK * 2;            // 16 KB
constexpr int kTileB = BN * BK * 2;            // 4 KB
constexpr int kStage = kTileA + kTileB;        // 20 KB
constexpr uint32_t kTmemCols = 32;             // BN float32 accumulators per row
constexpr uint32_t kLBO = 128, kSBO = 1024;    // core-matrix strides (bytes): along K, along M / N
constexpr int kWaitLimit = 1 << 22;
constexpr int kStages = 4;
constexpr int kAhead = 2;   // tiles copied ahead of the MMAs; a stage is refilled kStages - kAhead tiles after its MMAs
constexpr size_t kSmemBytes = kStages * kStage + 64 + 1024;   // stages, barriers, alignment slack

// Instruction descriptor, kind::f16: float32 accumulate (bits 4-5 = 1), A and
// B bfloat16 (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4),
// version 1 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((kLBO >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((kSBO >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit = kWaitLimit) {
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Chunk c of a tile (8 bfloat16 = one core-matrix row): row c / 8, K group c % 8.
__device__ __forceinline__ uint32_t chunk_off(int row, int j) {
  return (uint32_t)((row >> 3) * kSBO + j * kLBO + (row & 7) * 16);
}

// Asynchronous 16-byte copy global -> shared; a chunk outside the matrix is
// zero-filled (source size 0, the source address then only needs to be valid).
__device__ __forceinline__ void copy_chunk(uint32_t dst, const bf16 *__restrict__ g, int ld, int row, int rows, int k,
                                           int K) {
  const bool in = row < rows && k < K;
  const bf16 *src = in ? g + (size_t)row * ld + k : g;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0) : "memory");
}

}  // namespace

// Diagnostic of the bounded waits: thread 0 initialises an mbarrier that
// expects one arrival and polls for its phase with the same bounded loop the
// GEMM uses. Without the arrival the poll gives up after `limit` tries and
// the kernel records that in *err, as k_gemm_tc does for a stalled pipeline;
// with it the wait succeeds at once. Nothing else waits, so it cannot stall.
__global__ void k_wait_selftest(int arrive, int limit, int *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = su32(&bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
  if (arrive) {
    uint64_t state;
    asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(state) : "r"(b) : "memory");
    (void)state;
  }
  if (!mbar_wait(b, 0u, limit)) atomicExch(err, 1);
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(b) : "memory");
}

__global__ void __launch_bounds__(kThreads) k_gemm_tc(const bf16 *__restrict__ A, int lda, const bf16 *__restrict__ B,
                                                      int ldb, int M, int N, int K, const float *__restrict__ bias,
                                                      int mode, float *Cf, int ldc, bf16 *Yb, int ldy, bf16 *Yt, int ldt,
                                                      int *err) {
  extern __shared__ uint8_t dsm[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
  uint64_t *bar = reinterpret_cast<uint64_t *>(base + kStages * kStage);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + kStages);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int nk = (K + BK - 1) / BK;
  // An earlier launch gave up on draining its MMAs (error bit 2) and kept its
  // TMEM columns: no tensor-core work on this device from then on.
  if (*reinterpret_cast<volatile int *>(err) & 2) return;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&bar[i])), "r"(1u));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  // Copy tile kt into its stage: A 8 chunks, B 2 chunks per thread.
  auto fetch = [&](int kt) {
    const uint32_t sa = su32(base + (kt % kStages) * kStage), sb = sa + kTileA;
    const int k0 = kt * BK;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = tid + i * kThreads, row = c >> 3, j = c & 7;
      copy_chunk(sa + chunk_off(row, j), A, lda, m0 + row, M, k0 + 8 * j, K);
    }
#pragma unroll
    for (int i = 0; i < BN * 8 / kThreads; ++i) {
      const int c = tid + i * kThreads, row = c >> 3, j = c & 7;
      copy_chunk(sb + chunk_off(row, j), B, ldb, n0 + row, N, k0 + 8 * j, K);
    }
  };
  for (int t = 0; t < kAhead; ++t) {
    if (t < nk) fetch(t);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  bool bad = false;
  int last = -1;   // the last tile whose MMAs were committed
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt % kStages;
    // this thread's copies of tile kt are done (kAhead - 1 younger groups may still fly)
    asm volatile("cp.async.wait_group %0;" ::"n"(kAhead - 1) : "memory");
    // make the copies visible to the tensor core (async proxy), then to the issuing thread
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = su32(base + s * kStage), sb = sa + kTileA;
#pragma unroll
      for (int q = 0; q < BK / 16; ++q) {
        const uint64_t ad = smem_desc(sa + (uint32_t)q * 2 * kLBO);
        const uint64_t bd = smem_desc(sb + (uint32_t)q * 2 * kLBO);
        const uint32_t acc = (kt > 0 || q > 0) ? 1u : 0u;
        asm volatile(
            "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&bar[s]))
                   : "memory");
    }
    last = kt;
    // copy tile kt + kAhead into the stage that tile kt + kAhead - kStages read, once its MMAs are done
    const int nt = kt + kAhead;
    if (nt < nk) {
      if (nt >= kStages) {
        const int pt = nt - kStages;
        const bool ok = mbar_wait(su32(&bar[pt % kStages]), (uint32_t)((pt / kStages) & 1));
        if (__syncthreads_or(!ok)) {
          bad = true;
          break;
        }
      }
      fetch(nt);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");

  // The last commit covers every MMA issued before it (after a timeout this
  // is the drain of the MMAs still in flight).
  bool drained = true;
  if (last >= 0) {
    const bool done = mbar_wait(su32(&bar[last % kStages]), (uint32_t)((last / kStages) & 1));
    drained = !__syncthreads_or(!done);
    if (!drained) bad = true;
  }
  if (bad) {
    // bit 0: a wait timed out (this launch's outputs are not valid); bit 2:
    // the MMAs may still be running, so their TMEM columns stay allocated
    if (tid == 0) atomicOr(err, drained ? 1 : 3);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int m = m0 + 32 * warp + lane;
#pragma unroll
    for (int cc = 0; cc < BN / 16; ++cc) {
      uint32_t r[16];
      const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(cc * 16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + cc * 16 + j;
          if (n >= N) continue;
          float v = __uint_as_float(r[j]) + (bias ? bias[n] : 0.0f);
          if (mode == 0) {
            Cf[(size_t)m * ldc + n] = v;
          } else {
            const bf16 h = __float2bfloat16_rn(fmaxf(v, 0.0f));
            Yb[(size_t)m * ldy + n] = h;
            if (Yt) Yt[(size_t)n * ldt + m] = h;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // Free the columns only when no MMA can still write them (a few columns
  // kept after a failed drain are lost until the process ends, which is what
  // bit 2 tells the host).
  if (warp == 0 && drained)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

cudaError_t launch_wait_selftest(int arrive, int limit, int *err, cudaStream_t s) {
  if (limit < 1 || limit > kWaitLimit) return cudaErrorInvalidValue;
  k_wait_selftest<<<1, 32, 0, s>>>(arrive, limit, err);
  return cudaGetLastError();
}

cudaError_t gemm_tc_setup() {
  return cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

cudaError_t launch_gemm_tc(const bf16 *A, int lda, const bf16 *B, int ldb, int M, int N, int K, const float *bias,
                           int mode, float *Cf, int ldc, bf16 *Yb, int ldy, bf16 *Yt, int ldt, int *err,
                           cudaStream_t s) {
  if (M < 1 || N < 1 || K < 1 || K % 8 != 0 || lda % 8 != 0 || ldb % 8 != 0) return cudaErrorInvalidValue;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  k_gemm_tc<<<grid, kThreads, kSmemBytes, s>>>(A, lda, B, ldb, M, N, K, bias, mode, Cf, ldc, Yb, ldy, Yt, ldt, err);
  return cudaGetLastError();
}

}  // namespace stitch
