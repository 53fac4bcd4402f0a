// Learned estimate of the pair matrices inside the per-frame pipeline.
// k_learned_features and the network run beside the plain estimate (K2) of
// frame T, on the statistics alone; k_learned_select runs after both, when K2
// has stored the window's exact Eq. 3 terms and the plain M of every pair and
// advanced the frame index.
//
// k_learned_features: per pair, keep frame T's overlap histograms in a ring,
// pool them over the window {T-W+1..T} and write the network's features
// (each side's histograms scaled by 256 / count, bfloat16).
// The network then runs on these features (k_mlp.cu).
// k_learned_select: per pair, M_hat = I + the network's first nine outputs and
// its residual: how much M_hat raises Eq. 2's least-squares error over the
// plain fit M* = A^-1 B of the window, relative to the energy of the fitted
// colours, r = ||X (M_hat - M*)||^2 / ||X M*||^2 = tr(D^T A D) / tr(M*^T A M*)
// with D = M_hat - M* and A = X^T X the window's summed Gram matrix (float64;
// the cross term vanishes at the optimum). A pair whose plain fit succeeded
// and whose r <= 1e-3 takes M_hat (its transferred colours within about 3 %
// RMS of the plain fit's); any other pair keeps the plain result. The chosen
// matrices are chained to the reference camera again and replace frame T's
// colour output.
#include "estimate_common.cuh"
#include "stitch_internal.h"

namespace stitch {

namespace {

using namespace est;

constexpr double kResidLimit = 1e-3;

// One block per (pair, side, channel), one thread per bin: the float64
// divisions spread over 6 blocks per pair instead of one (FP64 throughput is
// low on this part). Each block also pools its side's channel 0 for the pixel
// count.
__global__ void __launch_bounds__(256) k_learned_features(const LearnedParams P) {
  const int p = blockIdx.x;
  const int side = blockIdx.y / 3, ch = blockIdx.y % 3;
  const int v = threadIdx.x;
  LearnedState *L = P.ls;
  // the frame being estimated: this kernel runs beside the plain estimate,
  // which advances the colour state's T, so the index comes from the learned
  // state (k_learned_select moves it on after both)
  const int frame = L->frame;
  const int slot = frame % kMaxWindow;
  const RawStats *raw = P.raw + (frame % P.raw_slots);
  const int nw = min(frame + 1, P.window);
  const uint32_t *cur = side == 0 ? &raw->Hi[p][0][0] : &raw->Hj[p][0][0];
  __shared__ unsigned long long part[8];
  // window sums of bin v of this channel and of channel 0 (the count)
  const int i = ch * 256 + v;
  const uint32_t h = cur[i], h0 = cur[v];
  L->H_ring[slot][p][side][i] = h;
  uint32_t s = h, s0 = h0;
  for (int k = 1; k < nw; ++k) {
    const int sl = (frame - k) % kMaxWindow;
    s += L->H_ring[sl][p][side][i];
    s0 += L->H_ring[sl][p][side][v];
  }
  const unsigned long long w = warp_sum((unsigned long long)s0);
  if ((v & 31) == 0) part[v >> 5] = w;
  __syncthreads();
  unsigned long long c = 0ull;
#pragma unroll
  for (int q = 0; q < 8; ++q) c += part[q];
  // (H * 256) / n in float64, then float32, then bfloat16 (both round to nearest even)
  const double f = c ? ((double)s * 256.0) / (double)c : 0.0;
  L->feat[p][side * 768 + i] = __float2bfloat16_rn(__double2float_rn(f));
}

__global__ void __launch_bounds__(256) k_learned_select(const LearnedParams P) {
  ColorState *S = P.state;
  LearnedState *L = P.ls;
  const int frame = S->T - 1;
  const int np = P.n_pairs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double M_pair[kMaxPairs][9];
  __shared__ double M_cam[kMaxCams][9];
  __shared__ int n_used;
  if (threadIdx.x == 0) n_used = 0;
  __syncthreads();
  if (warp < np) {
    const int p = warp;
    const int e = lane < 9 ? lane : 0;
    const int r = e / 3, c = e % 3;
    static const int sym[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
    const int nw = min(frame + 1, P.window);
    unsigned long long As = 0ull;
    for (int i = 0; i < nw; ++i) {
      const int sl = (frame - i) % kMaxWindow;
      As += S->A_ring[sl][p][sym[e]];
    }
    const double a = (double)As;
    const double mh = (double)L->y[p][e] + (r == c ? 1.0 : 0.0);
    const double ms = S->M_pair[p][e];              // the plain fit of this window
    const double d = mh - ms;
    // (A D)(r, c) and (A M*)(r, c) = sum_k A(r, k) (.)(k, c)
    double ad = 0.0, am = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double ark = __shfl_sync(0xffffffffu, a, r * 3 + k);
      ad += ark * __shfl_sync(0xffffffffu, d, k * 3 + c);
      am += ark * __shfl_sync(0xffffffffu, ms, k * 3 + c);
    }
    double num = lane < 9 ? d * ad : 0.0;           // tr(D^T A D)
    double den = lane < 9 ? ms * am : 0.0;          // tr(M*^T A M*)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      num += __shfl_down_sync(0xffffffffu, num, o);
      den += __shfl_down_sync(0xffffffffu, den, o);
    }
    num = __shfl_sync(0xffffffffu, num, 0);
    den = __shfl_sync(0xffffffffu, den, 0);
    const double res = den > 0.0 ? num / den : INFINITY;
    const bool plain_ok = ((S->singular_last >> p) & 1) == 0;
    const bool use = plain_ok && isfinite(mh) && res <= kResidLimit;   // NaN fails both tests
    const bool all_finite = __all_sync(0xffffffffu, lane >= 9 || isfinite(mh));
    const bool take = use && all_finite;
    if (lane < 9) {
      L->M_hat[p][lane] = mh;
      M_pair[p][lane] = take ? mh : S->M_pair[p][lane];
    }
    if (lane == 0) {
      L->resid[p] = res;
      L->used[p] = take ? 1 : 0;
      if (take) atomicAdd(&n_used, 1);
    }
  }
  __syncthreads();
  if (warp == 0) {
    warp_chain(M_pair, M_cam, P.n_cams, P.ref);
    ColorOut &o = S->out[frame % kColorSlots];
    for (int i = lane; i < P.n_cams * 9; i += 32) {
      S->M_cam[i / 9][i % 9] = M_cam[i / 9][i % 9];
      o.M[i / 9][i % 9] = (float)M_cam[i / 9][i % 9];
    }
    for (int i = lane; i < np * 9; i += 32) S->M_pair[i / 9][i % 9] = M_pair[i / 9][i % 9];
    if (lane == 0) {
      L->n_learned += (unsigned long long)n_used;
      L->n_fallback += (unsigned long long)(np - n_used);
      L->frame = S->T;                // the next frame's features
    }
  }
}

}  // namespace

cudaError_t launch_learned_features(const LearnedParams &p, cudaStream_t s) {
  if (p.n_pairs <= 0) return cudaSuccess;
  k_learned_features<<<dim3(p.n_pairs, 6), 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_learned_select(const LearnedParams &p, cudaStream_t s) {
  if (p.n_pairs <= 0) return cudaSuccess;
  k_learned_select<<<1, 256, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace stitch
