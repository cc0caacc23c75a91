// Shared device-side definitions of the GB300 sketched flexible Golub-Kahan solver.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "sfl.h"

namespace sfl {

constexpr int kThreads = 256;          // threads per CTA of the streaming kernels
constexpr int kWarps = kThreads / 32;
constexpr int kMaxWindow = 8;          // largest orthogonalization window ell
constexpr int kRing = kMaxWindow + 2;  // ring slots: w needs ell+2, p needs ell+1
constexpr int kMaxS = 2048;            // largest sketch size s
constexpr int kMaxIt = 1024;           // largest maxit
constexpr int kMaxZeta = 16;           // nonzeros per sketch column
constexpr int kGroup = 32;             // CTAs per first-level reduction group
constexpr int kMaxGroups = 64;         // upper bound on first-level groups
constexpr int kRedExtra = 2 * kRing + 4;  // scalar slots in a reduction besides the sketch

// Internal stop codes beyond sfl_stop.
constexpr int kStopNonfinite = 100;

enum Method : int { kSFLSQR = 0, kSFLSMR = 1 };

// Device-resident state of one solve.  Vectors of the partially orthogonal
// bases are stored unnormalised (w~, p~) with their scales sig = 1/||.|| so
// that no kernel has to rescale a vector after its norm is known.
struct SolveState {
  uint64_t seed;    // sketch seed of this solve
  int k;            // completed steps
  int stop;         // sfl_stop (0 while running) or kStopNonfinite
  int lucky;        // ||w|| vanished at the current step
  int hist_pending; // x_k waits to be written to the history
  double beta0;     // ||b||
  double tol;       // eta * noise_norm / ||b||
  double stop_den;  // denominator of the stop ratio
  double eta, noise_norm, irw_eps;
  double R11;       // first diagonal entry of the small QR
  double relres;    // stop ratio of the last step
  double znorm_raw2, wnorm_raw2;  // squared norms before orthogonalization
  double alpha, betak;
  double sig_w[kRing], sig_p[kRing];            // scales by ring slot
  double gram_w[kRing][kRing], gram_p[kRing][kRing];  // <v_i, v_j> of unit vectors, by slot
  double cz[kMaxWindow + 2];   // MGS coefficients of z against the p window
  double hw[kMaxWindow + 2];   // MGS coefficients of w against the w window (column of H)
};

// Scratch of the two-level deterministic grid reduction.
struct RedScratch {
  double *part;        // [grid][stride]
  double *gpart;       // [kMaxGroups][stride]
  unsigned int *cnt;   // [kMaxGroups + 1], zero between launches
  int stride;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order two-level reduction of `cnt` per-CTA values (smem `vals`, valid
// in every thread).  Every CTA stores its values; the last CTA of each group of
// kGroup CTAs sums its group in CTA order; the last group finisher sums the
// group sums in group order into `out` (smem) and returns true.  The order of
// every sum is fixed, so the result is bitwise reproducible.  No CTA waits on
// another: the last arrivals are found with atomic tickets.
__device__ __forceinline__ bool grid_reduce(const double *vals, int cnt, const RedScratch &sc, double *out,
                                            int *s_flag) {
  const int G = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
  const int g = bid / kGroup;
  const int gsize = min(kGroup, G - g * kGroup);
  const int NG = (G + kGroup - 1) / kGroup;
  for (int i = tid; i < cnt; i += blockDim.x) sc.part[(size_t)bid * sc.stride + i] = vals[i];
  __threadfence();
  __syncthreads();
  if (tid == 0) *s_flag = (atomicAdd(&sc.cnt[g], 1u) == (unsigned)(gsize - 1));
  __syncthreads();
  if (!*s_flag) return false;
  __threadfence();
  for (int i = tid; i < cnt; i += blockDim.x) {
    double acc = 0.0;
    for (int b = g * kGroup; b < g * kGroup + gsize; ++b) acc += __ldcg(&sc.part[(size_t)b * sc.stride + i]);
    sc.gpart[(size_t)g * sc.stride + i] = acc;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    sc.cnt[g] = 0u;
    *s_flag = (atomicAdd(&sc.cnt[kMaxGroups], 1u) == (unsigned)(NG - 1));
  }
  __syncthreads();
  if (!*s_flag) return false;
  __threadfence();
  for (int i = tid; i < cnt; i += blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < NG; ++q) acc += __ldcg(&sc.gpart[(size_t)q * sc.stride + i]);
    out[i] = acc;
  }
  if (tid == 0) sc.cnt[kMaxGroups] = 0u;
  __syncthreads();
  return true;
}

// Sum of per-warp values held in lane 0 of each warp (smem scratch wtmp[kWarps]),
// fixed order; result valid in all threads after the call.
__device__ __forceinline__ double cta_sum(double v, double *wtmp) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) wtmp[warp] = v;
  __syncthreads();
  double acc = 0.0;
  for (int w = 0; w < kWarps; ++w) acc += wtmp[w];
  __syncthreads();
  return acc;
}

template <typename T> __device__ __forceinline__ double to_d(T v) { return (double)v; }
template <> __device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// Ring slot of basis vector j (1-based).
__device__ __forceinline__ int ring_slot(int j, int R) { return j % R; }

}  // namespace sfl
