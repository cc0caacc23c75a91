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

// kFLSQR: full orthogonalization with the exact projected problem min || beta e_1 - H y ||
// (no sketch), solved by the small least-squares kernel in its sFLSMR form with identity columns.
enum Method : int { kSFLSQR = 0, kSFLSMR = 1, kFLSQR = 2 };

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
  double rinv_cmax; // largest column norm of R^{-1} so far (R11 * it bounds kappa(R) from below)
  double relres;    // stop ratio of the last step
  double znorm_raw2, wnorm_raw2;  // squared norms before orthogonalization
  double alpha, betak;
  double sig_w[kRing], sig_p[kRing];            // scales by ring slot
  double gram_w[kRing][kRing], gram_p[kRing][kRing];  // <v_i, v_j> by slot: unit w and p (z_j when orth_z)
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

// Partial-sum buffers hold up to kPartStride quantities for up to kPartCap
// producer CTAs, quantity-major: part[q * kPartCap + cta], so that a warp
// reading one quantity over consecutive CTAs makes coalesced loads.
constexpr int kPartStride = 16;
constexpr int kPartCap = kGroup * kMaxGroups;   // largest grid of any step kernel

// Copy the device solve state into shared memory (one coalesced pass).
__device__ __forceinline__ void stage_state(const SolveState *st, SolveState *sst) {
  static_assert(sizeof(SolveState) % sizeof(double) == 0, "state must be a whole number of doubles");
  const double *src = reinterpret_cast<const double *>(st);
  double *dst = reinterpret_cast<double *>(sst);
  for (int i = threadIdx.x; i < (int)(sizeof(SolveState) / sizeof(double)); i += blockDim.x) dst[i] = __ldcg(src + i);
  __syncthreads();
}

// Sum over the 8 warp values w[0..7] as a balanced tree (3 dependent adds).
__device__ __forceinline__ double tree8(const double *w) {
  return ((w[0] + w[1]) + (w[2] + w[3])) + ((w[4] + w[5]) + (w[6] + w[7]));
}

// FP64 on this GPU issues one warp-instruction per ~79 cycles per SM
// sub-partition, whatever the number of active lanes, and a dependent FP64
// add takes 64 cycles.  The reductions below therefore use few, full-warp
// FP64 instructions and short dependency chains; their order is fixed, so
// results are bitwise reproducible.

// Totals of NQ <= kPartStride quantities over the per-CTA records of a
// producer kernel with G CTAs (part[q * kPartCap + b]).  Every CTA of the
// consumer computes the same values: warp q (and q + kWarps) sums quantity q.
// Each lane issues all its loads at once (kRedLoads records, one L2 round
// trip for G <= 32 * kRedLoads), adds them as a fixed tree, then the lanes
// fold with a butterfly.  out: smem [kPartStride].  All threads call.
constexpr int kRedLoads = 16;

template <int NQ>
__device__ __forceinline__ void reduce_partials_n(const double *part, int G, double *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = warp; q < NQ; q += kWarps) {
    double v[kRedLoads];
#pragma unroll
    for (int t = 0; t < kRedLoads; ++t) {
      const int b = lane + 32 * t;
      v[t] = b < G ? __ldcg(part + (size_t)q * kPartCap + b) : 0.0;
    }
#pragma unroll
    for (int w = kRedLoads / 2; w >= 1; w >>= 1)
#pragma unroll
      for (int t = 0; t < w; ++t) v[t] += v[t + w];
    double a = v[0];
    for (int b = lane + 32 * kRedLoads; b < G; b += 32) a += __ldcg(part + (size_t)q * kPartCap + b);
    a = warp_sum(a);
    if (lane == 0) out[q] = a;
  }
  __syncthreads();
}

__device__ __forceinline__ void reduce_partials(const double *part, int G, int nq, double *wsum, double *out) {
  (void)wsum;
  switch (nq) {
    case 1: reduce_partials_n<1>(part, G, out); break;
    case 2: reduce_partials_n<2>(part, G, out); break;
    case 3: reduce_partials_n<3>(part, G, out); break;
    case 4: reduce_partials_n<4>(part, G, out); break;
    case 5: reduce_partials_n<5>(part, G, out); break;
    case 6: reduce_partials_n<6>(part, G, out); break;
    case 7: reduce_partials_n<7>(part, G, out); break;
    case 8: reduce_partials_n<8>(part, G, out); break;
    case 9: reduce_partials_n<9>(part, G, out); break;
    default: reduce_partials_n<10>(part, G, out); break;
  }
}

// Per-CTA totals of NQ per-thread values, written to this CTA's record of a
// partial-sum buffer.  Threads park their values in shared memory (no FP64
// work); warp q adds the 8 values of its lanes as a tree and folds the lanes
// with a butterfly.  scr: smem [NQ * kThreads].  All threads call.
template <int NQ>
__device__ __forceinline__ void store_partials(const double (&v)[NQ], double *scr, double *part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) scr[q * kThreads + threadIdx.x] = v[q];
  __syncthreads();
  for (int q = warp; q < NQ; q += kWarps) {
    const double *s = scr + q * kThreads + lane;
    const double a = ((s[0] + s[32]) + (s[64] + s[96])) + ((s[128] + s[160]) + (s[192] + s[224]));
    const double t = warp_sum(a);
    if (lane == 0) part[(size_t)q * kPartCap + blockIdx.x] = t;
  }
}
static_assert(kThreads == 256, "store_partials adds 8 values per lane");

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

// Bytes of dynamic shared memory this launch received.
__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
  uint32_t v;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
  return v;
}

// Ring slot of basis vector j (1-based).
__device__ __forceinline__ int ring_slot(int j, int R) { return j % R; }

// Programmatic dependent launch.  griddep_wait blocks until the grid this one
// depends on has completed and its writes are visible (it returns at once for
// a launch without that dependency); griddep_launch_dependents lets the next
// kernel of the stream start launching its CTAs, which then wait in their own
// griddep_wait.  Every step kernel calls both before touching shared state.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

}  // namespace sfl
