// Kernels of one sketched flexible Golub-Kahan step (Algorithms 1 and 2).
//
// Per step k the solver runs, on one stream, captured in a CUDA graph:
//   zorth   p~_k = z - sum_j c_j p_j (MGS coefficients c_j), z~_k = tau_k(p~_k)
//   fwd     w = A z_k (CSR SpMV) + window dots <w_j, w> + sketch S_m w
//   worth   w~_{k+1} = w - sum_j h_j w_j, ||w~_{k+1}||  (column k of H)
//   bwd     z = A^T w_{k+1} (CSR of A^T, or B) + dots <p_j, z> (+ S_n z, sFLSMR)
//   ls      append one column to the FP64 QR of the sketched problem, update
//           y_k and the stop ratio, set the graph's loop condition
// Every reduction is fixed-order, so results are bitwise reproducible.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace sfl {

// ---------------------------------------------------------------- sketch table

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the first output of a
// generator whose state is `state`.
__device__ __forceinline__ uint64_t splitmix64_first(uint64_t state) {
  uint64_t z = state + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Column c of the sparse-sign sketch (Section 2.7): draws t = 0, 1, ... with
// h = splitmix64_first(seed ^ (c*2^32 + t)), row floor(h*s/2^64), sign from
// bit 0; duplicates rejected until zeta distinct rows.  Packed entry: row in
// bits 0..14, bit 15 set for a negative sign.  `zs` entries per column
// (zs >= zeta; unused entries are 0xFFFF).  Optional unpacked export.
// The seed is `seed` or, when seed_src is given, *seed_src (plus seed_add).
static __global__ void sketch_table_kernel(uint64_t seed, const uint64_t *seed_src, uint64_t seed_add, int s, int zeta,
                                    int64_t ncols, int zs, uint16_t *tab, int32_t *rows_out, int32_t *signs_out,
                                    int *err) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  if (seed_src) seed = *seed_src;
  seed += seed_add;
  int rows[kMaxZeta];
  int cnt = 0;
  for (uint32_t t = 0; cnt < zeta && t < 1000000u; ++t) {
    const uint64_t h = splitmix64_first(seed ^ (((uint64_t)c << 32) + t));
    const int r = (int)__umul64hi(h, (uint64_t)s);
    bool dup = false;
    for (int q = 0; q < cnt; ++q) dup |= (rows[q] == r);
    if (dup) continue;
    rows[cnt] = r;
    const int neg = (int)(h & 1ull);
    if (tab) tab[c * zs + cnt] = (uint16_t)(r | (neg << 15));
    if (rows_out) { rows_out[c * zeta + cnt] = r; signs_out[c * zeta + cnt] = neg ? -1 : 1; }
    ++cnt;
  }
  if (cnt < zeta) { atomicExch(err, 1); return; }
  if (tab) for (int q = cnt; q < zs; ++q) tab[c * zs + q] = 0xFFFFu;
}

// ---------------------------------------------------------------- fused SpMV

enum SpmvMode : int {
  kModeApply = 0,    // plain y = A x
  kModeInitB = 1,    // row value = b_i: ||b||^2, S_m b, w~_1 = b
  kModeInitBwd = 2,  // z = A^T w_1, ||z||^2, (sFLSMR) S_n z
  kModeFwd = 3,      // w = A z_k, window dots with w_j, ||w||^2, S_m w
  kModeBwd = 4,      // z = A^T w_{k+1}, window dots with p_j, ||z||^2, (sFLSMR) S_n z
  kModeSketch = 5    // row value = b_i: sk_out = S b only
};

template <typename VT, typename XT>
struct SpmvParams {
  const int32_t *rowptr;    // padded CSR (rows start at multiples of the load width)
  const int32_t *col;
  const VT *val;
  int64_t rows;
  int mode;
  int method;
  int stop_rule;
  int ell;
  int s;
  int zeta;
  int zs;
  int maxit;
  const XT *x;              // kModeApply: input vector
  const double *b;          // kModeInitB
  XT *y;                    // output (kModeApply / kModeInitB: explicit)
  SolveState *st;
  XT *wring; int64_t wstride; int RW;   // ring of w~ (m-vectors)
  XT *pring; int64_t pstride; int RP;   // ring of p~ (n-vectors)
  XT *Z; int64_t zstride;               // z~_j columns
  const double *sigZ;
  XT *wraw;                             // w = A z_k
  XT *zraw;                             // z = A^T w
  const uint16_t *tab;                  // sketch table of the output space (or null)
  double *SAZ;     // sFLSQR: LS columns S_m A z_k;  sFLSMR: m-side stop columns
  double *SAtW;    // sFLSMR: S_n A^T w_j columns (s x (maxit+1))
  double *Hband;   // sFLSMR: columns of H, (ell+2) entries per column
  double *rhs;     // LS right-hand side
  double *e;       // LS residual vector
  double *sbm;     // sFLSMR residual rule: S_m b
  double *sk_out;  // kModeSketch output
  RedScratch red;
};

// Loads of P consecutive stored entries (P*4 bytes of indices, P*sizeof(VT) of values).
template <typename VT, int P> struct Chunk;
template <> struct Chunk<double, 4> {
  int c[4]; double v[4];
  __device__ __forceinline__ void load(const int32_t *col, const double *val, int off) {
    const int4 ci = __ldcs(reinterpret_cast<const int4 *>(col + off));
    const double2 a = __ldcs(reinterpret_cast<const double2 *>(val + off));
    const double2 b = __ldcs(reinterpret_cast<const double2 *>(val + off + 2));
    c[0] = ci.x; c[1] = ci.y; c[2] = ci.z; c[3] = ci.w;
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};
template <> struct Chunk<float, 4> {
  int c[4]; float v[4];
  __device__ __forceinline__ void load(const int32_t *col, const float *val, int off) {
    const int4 ci = __ldcs(reinterpret_cast<const int4 *>(col + off));
    const float4 a = __ldcs(reinterpret_cast<const float4 *>(val + off));
    c[0] = ci.x; c[1] = ci.y; c[2] = ci.z; c[3] = ci.w;
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
};
template <> struct Chunk<__nv_bfloat16, 8> {
  int c[8]; float v[8];
  __device__ __forceinline__ void load(const int32_t *col, const __nv_bfloat16 *val, int off) {
    const int4 c0 = __ldcs(reinterpret_cast<const int4 *>(col + off));
    const int4 c1 = __ldcs(reinterpret_cast<const int4 *>(col + off + 4));
    const uint4 raw = __ldcs(reinterpret_cast<const uint4 *>(val + off));
    c[0] = c0.x; c[1] = c0.y; c[2] = c0.z; c[3] = c0.w;
    c[4] = c1.x; c[5] = c1.y; c[6] = c1.z; c[7] = c1.w;
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[2 * q] = __uint_as_float(w[q] << 16);
      v[2 * q + 1] = __uint_as_float(w[q] & 0xFFFF0000u);
    }
  }
};

template <typename VT> struct LoadWidth { static constexpr int P = 4; };
template <> struct LoadWidth<__nv_bfloat16> { static constexpr int P = 8; };

template <typename XT> struct AccT { using T = XT; };

// Finisher of the fused SpMV: runs in the single CTA holding the final sums.
//   tot[0] = ||y||^2, tot[1..nd] = window dots, tot[1+nd ..] = unscaled sketch.
template <typename VT, typename XT>
__device__ void spmv_finish(const SpmvParams<VT, XT> &p, int k, int lo, int nd, const double *tot, double *wtmp) {
  SolveState *st = p.st;
  const int tid = threadIdx.x;
  const double isz = 1.0 / sqrt((double)p.zeta);
  const double *sk = tot + 1 + nd;
  if (p.mode == kModeSketch) {
    for (int i = tid; i < p.s; i += blockDim.x) p.sk_out[i] = sk[i] * isz;
  } else if (p.mode == kModeInitB) {
    double *dst = (p.method == kSFLSQR) ? p.rhs : p.sbm;
    double ss = 0.0;
    for (int i = tid; i < p.s; i += blockDim.x) {
      const double v = sk[i] * isz;
      dst[i] = v;
      if (p.method == kSFLSQR) p.e[i] = v;
      ss += v * v;
    }
    ss = cta_sum(ss, wtmp);
    if (tid == 0) {
      const double beta = sqrt(tot[0]);
      st->beta0 = beta;
      st->sig_w[ring_slot(1, p.RW)] = 1.0 / beta;
      st->tol = (st->noise_norm > 0.0) ? st->eta * st->noise_norm / beta : 0.0;
      if (p.method == kSFLSQR || p.stop_rule == SFL_STOP_RULE_RESIDUAL) st->stop_den = sqrt(ss);
      if (!(beta > 0.0)) st->stop = SFL_STOP_BREAKDOWN;
      if (!isfinite(tot[0]) || !isfinite(ss)) st->stop = kStopNonfinite;
    }
  } else if (p.mode == kModeInitBwd) {
    if (p.method == kSFLSMR) {
      double ss = 0.0;
      const double beta = st->beta0;
      for (int i = tid; i < p.s; i += blockDim.x) {
        const double v = sk[i] * isz;
        p.SAtW[i] = v;
        p.rhs[i] = beta * v;
        p.e[i] = beta * v;
        ss += (beta * v) * (beta * v);
      }
      ss = cta_sum(ss, wtmp);
      if (tid == 0 && p.stop_rule == SFL_STOP_RULE_NORMAL) st->stop_den = sqrt(ss);
    }
    if (tid == 0) st->znorm_raw2 = tot[0];
  } else if (p.mode == kModeFwd) {
    double *col = p.SAZ + (size_t)(k - 1) * p.s;
    for (int i = tid; i < p.s; i += blockDim.x) col[i] = sk[i] * isz;
    if (tid == 0) {
      st->wnorm_raw2 = tot[0];
      // MGS coefficients through the window Gram matrix:
      // h_j = <w_j, w> - sum_{i<j} h_i <w_j, w_i>
      double h[kMaxWindow + 2];
      for (int a = 0; a < nd; ++a) {
        const int ja = lo + a;
        double v = tot[1 + a] * st->sig_w[ring_slot(ja, p.RW)];
        for (int c = 0; c < a; ++c) v -= h[c] * st->gram_w[ring_slot(ja, p.RW)][ring_slot(lo + c, p.RW)];
        h[a] = v;
        st->hw[a] = v;
      }
      if (p.method == kSFLSMR) {
        double *hb = p.Hband + (size_t)(k - 1) * (p.ell + 2);
        for (int q = 0; q < p.ell + 2; ++q) hb[q] = 0.0;
        for (int a = 0; a < nd; ++a) hb[(lo + a) - k + p.ell] = h[a];
      }
    }
  } else if (p.mode == kModeBwd) {
    if (p.method == kSFLSMR) {
      double *col = p.SAtW + (size_t)k * p.s;
      for (int i = tid; i < p.s; i += blockDim.x) col[i] = sk[i] * isz;
    }
    if (tid == 0) {
      st->znorm_raw2 = tot[0];
      double c[kMaxWindow + 2];
      for (int a = 0; a < nd; ++a) {
        const int ja = lo + a;
        double v = tot[1 + a] * st->sig_p[ring_slot(ja, p.RP)];
        for (int q = 0; q < a; ++q) v -= c[q] * st->gram_p[ring_slot(ja, p.RP)][ring_slot(lo + q, p.RP)];
        c[a] = v;
        st->cz[a] = v;
      }
    }
  }
}

// Row sum of one row for a group of LPR lanes (lane gl of the group), P
// entries per lane per load, four loads in flight per lane.
template <typename VT, typename XT, int LPR>
__device__ __forceinline__ typename AccT<XT>::T row_dot(const SpmvParams<VT, XT> &p, const XT *__restrict__ x,
                                                       int beg, int end, int gl) {
  constexpr int P = LoadWidth<VT>::P;
  constexpr int STR = LPR * P;
  using ACC = typename AccT<XT>::T;
  ACC s0 = (ACC)0, s1 = (ACC)0;
  int off = beg + gl * P;
#pragma unroll 1
  for (; off + 3 * STR < end; off += 4 * STR) {
    Chunk<VT, P> c0, c1, c2, c3;
    c0.load(p.col, p.val, off);
    c1.load(p.col, p.val, off + STR);
    c2.load(p.col, p.val, off + 2 * STR);
    c3.load(p.col, p.val, off + 3 * STR);
#pragma unroll
    for (int q = 0; q < P; ++q) {
      s0 += (ACC)c0.v[q] * (ACC)__ldg(x + c0.c[q]);
      s1 += (ACC)c1.v[q] * (ACC)__ldg(x + c1.c[q]);
      s0 += (ACC)c2.v[q] * (ACC)__ldg(x + c2.c[q]);
      s1 += (ACC)c3.v[q] * (ACC)__ldg(x + c3.c[q]);
    }
  }
#pragma unroll 1
  for (; off < end; off += STR) {
    Chunk<VT, P> c0;
    c0.load(p.col, p.val, off);
#pragma unroll
    for (int q = 0; q < P; ++q) s0 += (ACC)c0.v[q] * (ACC)__ldg(x + c0.c[q]);
  }
  return s0 + s1;
}

// A warp processes groups of G = 32/LPR consecutive rows (LPR lanes per row);
// lane 0 of each row's lanes then owns the row for the epilogue: output
// write, window dots, and the sparse-sign sketch accumulated into a
// warp-private shared-memory s-vector in a fixed order (groups in grid-stride
// order, rows in index order).  LPR = 1 is the vector pass (no matrix).
template <typename VT, typename XT, int LPR, bool MAT>
__global__ void __launch_bounds__(kThreads) spmv_fused_kernel(SpmvParams<VT, XT> p) {
  constexpr int G = 32 / LPR;
  using ACC = typename AccT<XT>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SolveState *st = p.st;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // ---- resolve the step's operands from the device state
  int k = 0, lo = 1, nd = 0;
  const XT *x = p.x;
  XT *y = p.y;
  const XT *win = nullptr; int64_t wst = 0; int R = 1;
  double xscale = 1.0;
  bool sketch = false, reduce = true;
  if (p.mode == kModeApply) {
    reduce = false;
  } else if (p.mode == kModeSketch) {
    sketch = true;
  } else {
    if (st->stop) return;
    k = st->k + 1;
    if (p.mode == kModeInitB) {
      y = p.wring + (size_t)ring_slot(1, p.RW) * p.wstride;
      sketch = true;
    } else if (p.mode == kModeInitBwd) {
      x = p.wring + (size_t)ring_slot(1, p.RW) * p.wstride;
      xscale = st->sig_w[ring_slot(1, p.RW)];
      y = p.zraw;
      sketch = (p.method == kSFLSMR);
    } else if (p.mode == kModeFwd) {
      x = p.Z + (size_t)(k - 1) * p.zstride;
      xscale = p.sigZ[k - 1];
      y = p.wraw;
      lo = max(1, k - p.ell); nd = k - lo + 1;
      win = p.wring; wst = p.wstride; R = p.RW;
      sketch = true;
    } else {  // kModeBwd
      if (st->lucky) return;
      x = p.wring + (size_t)ring_slot(k + 1, p.RW) * p.wstride;
      xscale = st->sig_w[ring_slot(k + 1, p.RW)];
      y = p.zraw;
      lo = max(1, k + 1 - p.ell); nd = k - lo + 1;
      win = p.pring; wst = p.pstride; R = p.RP;
      sketch = (p.method == kSFLSMR);
    }
  }
  XT *skacc = reinterpret_cast<XT *>(smem_raw);            // [kWarps][s] when sketching
  double *vals = reinterpret_cast<double *>(smem_raw + (sketch ? sizeof(XT) * kWarps * p.s : 0));
  const int nvals = 1 + nd + (sketch ? p.s : 0);
  double *wtmp = vals + nvals;                             // [kWarps * (kMaxWindow + 3)]
  __shared__ int s_flag;

  if (sketch) {
    for (int i = tid; i < kWarps * p.s; i += blockDim.x) skacc[i] = (XT)0;
    __syncthreads();
  }
  XT *myacc = skacc + warp * p.s;

  double dacc[kMaxWindow + 2];
#pragma unroll
  for (int a = 0; a < kMaxWindow + 2; ++a) dacc[a] = 0.0;
  double nacc = 0.0;
  const ACC sc = (ACC)xscale;

  const int64_t ngrp = (p.rows + G - 1) / G;
  const int gl = lane % LPR, grp = lane / LPR;
  const int64_t gstride = (int64_t)gridDim.x * kWarps;
  int64_t rb = (int64_t)blockIdx.x * kWarps + warp;
  int nbeg = 0, nend = 0;
  if (MAT && rb < ngrp) {
    const int64_t r = rb * G + grp;
    if (r < p.rows) { nbeg = p.rowptr[r]; nend = p.rowptr[r + 1]; }
  }
  for (; rb < ngrp; rb += gstride) {
    const int64_t row = rb * G + grp;
    const bool valid = row < p.rows;
    ACC yv = (ACC)0;
    if (MAT) {
      const int beg = nbeg, end = nend;
      const int64_t rn = (rb + gstride) * G + grp;     // prefetch the next group's row bounds
      if (rb + gstride < ngrp && rn < p.rows) { nbeg = p.rowptr[rn]; nend = p.rowptr[rn + 1]; }
      else { nbeg = 0; nend = 0; }
      ACC sum = row_dot<VT, XT, LPR>(p, x, beg, end, gl);
#pragma unroll
      for (int o = LPR / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      yv = sum * sc;
    } else {
      if (valid) yv = (ACC)p.b[row];
    }
    // ---- epilogue: lane gl == 0 of each group owns its row
    if (gl == 0 && valid) {
      if (y) y[row] = (XT)yv;
      if (reduce) {
        const double yd = (double)yv;
        nacc += yd * yd;
#pragma unroll
        for (int a = 0; a < kMaxWindow + 2; ++a)
          if (a < nd) dacc[a] += (double)win[(size_t)ring_slot(lo + a, R) * wst + row] * yd;
      }
    }
    if (sketch) {
      uint4 tw0 = make_uint4(0, 0, 0, 0), tw1 = make_uint4(0, 0, 0, 0);
      if (gl == 0 && valid) {
        tw0 = *reinterpret_cast<const uint4 *>(p.tab + row * p.zs);
        if (p.zs == 16) tw1 = *reinterpret_cast<const uint4 *>(p.tab + row * p.zs + 8);
      }
      const int64_t row0 = rb * G;
      const int nrow = (p.rows - row0) < G ? (int)(p.rows - row0) : G;
      for (int g = 0; g < nrow; ++g) {
        const int L = g * LPR;
        const XT v = (XT)__shfl_sync(0xffffffffu, yv, L);
        const uint32_t a0 = __shfl_sync(0xffffffffu, tw0.x, L), a1 = __shfl_sync(0xffffffffu, tw0.y, L);
        const uint32_t a2 = __shfl_sync(0xffffffffu, tw0.z, L), a3 = __shfl_sync(0xffffffffu, tw0.w, L);
        uint32_t b0 = 0, b1 = 0, b2 = 0, b3 = 0;
        if (p.zs == 16) {
          b0 = __shfl_sync(0xffffffffu, tw1.x, L); b1 = __shfl_sync(0xffffffffu, tw1.y, L);
          b2 = __shfl_sync(0xffffffffu, tw1.z, L); b3 = __shfl_sync(0xffffffffu, tw1.w, L);
        }
        if (lane < p.zeta) {
          const int wq = lane >> 1;
          const uint32_t wsel = wq == 0 ? a0 : wq == 1 ? a1 : wq == 2 ? a2 : wq == 3 ? a3
                              : wq == 4 ? b0 : wq == 5 ? b1 : wq == 6 ? b2 : b3;
          const uint32_t ent = (lane & 1) ? (wsel >> 16) : (wsel & 0xFFFFu);
          const int r = (int)(ent & 0x7FFFu);
          myacc[r] += (ent & 0x8000u) ? -v : v;
        }
        __syncwarp();
      }
    }
  }
  if (!reduce) return;

  // ---- CTA totals in fixed order
  {
    double v = warp_sum(nacc);
    if (lane == 0) wtmp[warp * (kMaxWindow + 3)] = v;
#pragma unroll
    for (int a = 0; a < kMaxWindow + 2; ++a) {
      if (a < nd) {
        v = warp_sum(dacc[a]);
        if (lane == 0) wtmp[warp * (kMaxWindow + 3) + 1 + a] = v;
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < 1 + nd; i += blockDim.x) {
    double acc = 0.0;
    for (int w = 0; w < kWarps; ++w) acc += wtmp[w * (kMaxWindow + 3) + i];
    vals[i] = acc;
  }
  if (sketch) {
    for (int i = tid; i < p.s; i += blockDim.x) {
      double acc = 0.0;
      for (int w = 0; w < kWarps; ++w) acc += (double)skacc[w * p.s + i];
      vals[1 + nd + i] = acc;
    }
  }
  __syncthreads();
  if (grid_reduce(vals, nvals, p.red, vals, &s_flag)) spmv_finish(p, k, lo, nd, vals, wtmp);
}

// ---------------------------------------------------------------- orthogonalization updates

template <typename XT>
struct OrthParams {
  SolveState *st;
  int side;            // 0: z side (p ring, tau, Z), 1: w side (w ring)
  int ell;
  int64_t len;
  const XT *raw;       // z (n) or w (m) before orthogonalization
  XT *ring; int64_t stride; int R;
  XT *Z; int64_t zstride;   // z side: Z columns
  double *sigZ;
  int precond;
  const double *diag_w;     // SFL_PRECOND_DIAG
  const double *y;          // LS solution y_{k-1} (SFL_PRECOND_REWEIGHT)
  double *Hband;            // sFLSMR: H_{k+1,k}
  int method;
  RedScratch red;
};

// z side: p~_k = z - sum_{j=lo}^{k-1} c_j p_j, z~_k = tau_k(p~_k);
// w side: w~_{k+1} = w - sum_{j=lo}^{k} h_j w_j.
// Reduces ||new||^2 and <new, v_j> over the window (for the next Gram rows).
template <typename XT>
__global__ void __launch_bounds__(kThreads) orth_update_kernel(OrthParams<XT> p) {
  SolveState *st = p.st;
  if (st->stop) return;
  const int k = st->k + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int lo, hi, newj;
  if (p.side == 0) { lo = max(1, k - p.ell); hi = k - 1; newj = k; }
  else { lo = max(1, k - p.ell); hi = k; newj = k + 1; }
  const int nd = hi - lo + 1 > 0 ? hi - lo + 1 : 0;
  double coef[kMaxWindow + 2];
  const XT *vj[kMaxWindow + 2];
#pragma unroll
  for (int a = 0; a < kMaxWindow + 2; ++a) {
    coef[a] = 0.0;
    vj[a] = p.ring;
    if (a < nd) {
      const int slot = ring_slot(lo + a, p.R);
      const double sg = (p.side == 0) ? st->sig_p[slot] : st->sig_w[slot];
      coef[a] = ((p.side == 0) ? st->cz[a] : st->hw[a]) * sg;
      vj[a] = p.ring + (size_t)slot * p.stride;
    }
  }
  XT *out = p.ring + (size_t)ring_slot(newj, p.R) * p.stride;
  XT *zout = (p.side == 0) ? p.Z + (size_t)(k - 1) * p.zstride : nullptr;
  // reweighting: coefficients c_j = sig_j y_j of x_{k-1} = sum_j z~_j c_j
  __shared__ double s_c[kMaxIt];
  const bool reweight = p.side == 0 && p.precond == SFL_PRECOND_REWEIGHT;
  if (reweight) {
    for (int j = tid; j < k - 1; j += blockDim.x) s_c[j] = p.sigZ[j] * p.y[j];
    __syncthreads();
  }

  double nacc = 0.0, dacc[kMaxWindow + 2];
#pragma unroll
  for (int a = 0; a < kMaxWindow + 2; ++a) dacc[a] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + tid; i < p.len; i += stride) {
    double v = (double)p.raw[i];
    double old[kMaxWindow + 2];
#pragma unroll
    for (int a = 0; a < kMaxWindow + 2; ++a) {
      old[a] = 0.0;
      if (a < nd) { old[a] = (double)vj[a][i]; v -= coef[a] * old[a]; }
    }
    const XT vx = (XT)v;
    out[i] = vx;
    const double vd = (double)vx;
    nacc += vd * vd;
#pragma unroll
    for (int a = 0; a < kMaxWindow + 2; ++a)
      if (a < nd) dacc[a] += vd * old[a];
    if (p.side == 0) {
      double zt = vd;
      if (p.precond == SFL_PRECOND_DIAG) {
        zt = p.diag_w[i] * vd;
      } else if (reweight) {
        // x_{k-1}[i] = sum_j z~_j[i] c_j, four independent partial sums
        const XT *zi = p.Z + i;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int j = 0;
        for (; j + 3 < k - 1; j += 4) {
          a0 += (double)zi[(size_t)j * p.zstride] * s_c[j];
          a1 += (double)zi[(size_t)(j + 1) * p.zstride] * s_c[j + 1];
          a2 += (double)zi[(size_t)(j + 2) * p.zstride] * s_c[j + 2];
          a3 += (double)zi[(size_t)(j + 3) * p.zstride] * s_c[j + 3];
        }
        for (; j < k - 1; ++j) a0 += (double)zi[(size_t)j * p.zstride] * s_c[j];
        const double xv = (a0 + a1) + (a2 + a3);
        zt = sqrt(sqrt(xv * xv + st->irw_eps)) * vd;
      }
      zout[i] = (XT)zt;
    }
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *vals = reinterpret_cast<double *>(smem_raw);
  double *wtmp = vals + (kMaxWindow + 3);
  __shared__ int s_flag;
  {
    double v = warp_sum(nacc);
    if (lane == 0) wtmp[warp * (kMaxWindow + 3)] = v;
#pragma unroll
    for (int a = 0; a < kMaxWindow + 2; ++a) {
      if (a < nd) {
        v = warp_sum(dacc[a]);
        if (lane == 0) wtmp[warp * (kMaxWindow + 3) + 1 + a] = v;
      }
    }
  }
  __syncthreads();
  if (tid < 1 + nd) {
    double acc = 0.0;
    for (int w = 0; w < kWarps; ++w) acc += wtmp[w * (kMaxWindow + 3) + tid];
    vals[tid] = acc;
  }
  __syncthreads();
  if (!grid_reduce(vals, 1 + nd, p.red, vals, &s_flag)) return;
  if (tid != 0) return;
  const double nrm = sqrt(vals[0]);
  const int ns = ring_slot(newj, p.R);
  if (p.side == 0) {
    const double raw = sqrt(st->znorm_raw2);
    if (!(nrm > 1e-300) || !(nrm > 1e-14 * raw)) { st->stop = isfinite(vals[0]) ? SFL_STOP_BREAKDOWN : kStopNonfinite; return; }
    st->alpha = nrm;
    st->sig_p[ns] = 1.0 / nrm;
    p.sigZ[k - 1] = 1.0 / nrm;
    for (int a = 0; a < nd; ++a) {
      const int sa = ring_slot(lo + a, p.R);
      const double g = vals[1 + a] * st->sig_p[sa] / nrm;
      st->gram_p[ns][sa] = g; st->gram_p[sa][ns] = g;
    }
  } else {
    const double raw = sqrt(st->wnorm_raw2);
    if (!isfinite(vals[0])) { st->stop = kStopNonfinite; return; }
    if (!(nrm > 1e-300) || !(nrm > 1e-14 * raw)) {
      st->lucky = 1;       // step k is still solved; no w_{k+1}
      st->betak = 0.0;
      return;
    }
    st->betak = nrm;
    st->sig_w[ns] = 1.0 / nrm;
    if (p.method == kSFLSMR) p.Hband[(size_t)(k - 1) * (p.ell + 2) + p.ell + 1] = nrm;
    for (int a = 0; a < nd; ++a) {
      const int sa = ring_slot(lo + a, p.R);
      const double g = vals[1 + a] * st->sig_w[sa] / nrm;
      st->gram_w[ns][sa] = g; st->gram_w[sa][ns] = g;
    }
  }
}

// ---------------------------------------------------------------- small FP64 least squares

struct LsParams {
  SolveState *st;
  int method, s, maxit, ell, stop_rule;
  double *Q;          // s x maxit, column-major: orthonormal basis of the sketched columns
  double *Rinv;       // maxit x maxit, row-major: inverse of the triangular factor
  double *y;          // maxit
  double *e;          // s: residual of the small problem
  const double *SAZ;  // sFLSQR: LS columns; sFLSMR: m-side columns for the residual rule
  const double *SAtW; // sFLSMR
  const double *Hband;
  const double *sbm;  // sFLSMR residual rule: S_m b
  double *relres_hist;
  cudaGraphConditionalHandle cond;
  int use_cond;
};

// One thread-block cluster appends column k of the sketched matrix to an
// explicit-Q QR by classical Gram-Schmidt applied twice (CGS2), updates the
// residual e, the inverse triangular factor and y_k = y_{k-1} + gamma_k
// Rinv[:,k], and evaluates the stop test.  Rows of Q are split in blocks over
// the CTAs of the cluster; partial sums are exchanged through distributed
// shared memory and summed in CTA order (deterministic).
static __global__ void __launch_bounds__(kThreads) ls_step_kernel(LsParams p) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), CL = (int)cl.num_blocks();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  SolveState *st = p.st;
  // Every CTA reads the flags before the first cluster barrier; rank 0 writes
  // them only after the last one, so all CTAs take the same branches.
  const int stop0 = st->stop, lucky = st->lucky;
  if (stop0) {
    if (rank == 0 && tid == 0 && p.use_cond) cudaGraphSetConditional(p.cond, 0u);
    return;
  }
  const int k = st->k + 1, kk = k - 1;
  const int s = p.s;
  const int RB = (s + CL - 1) / CL;
  const int r0 = min(s, rank * RB), r1 = min(s, r0 + RB), nr = r1 - r0;
  const int KP = p.maxit + 2;

  extern __shared__ __align__(16) double lsm[];
  double *part0 = lsm;              // [KP] partial vectors exchanged in the cluster (double-buffered)
  double *part1 = part0 + KP;
  double *red = part1 + KP;         // [KP] cluster-reduced vector
  double *rr = red + KP;            // [KP] R column above the diagonal
  double *crow = rr + KP;           // [RB] my rows of the working column
  double *tmp = crow + RB;          // [max(kThreads, RB) + RB] partial sums of (row, column slice)
  const int H = max(1, kThreads / max(RB, 1));   // column slices per row
  __shared__ double s_w[kWarps];
  __shared__ double s_sc[8];        // scalar partials exchanged in the cluster
  __shared__ double s_res[8];

  // CTA total of one value per thread, fixed order; valid in all threads.
  auto cta_total = [&](double v) -> double {
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    double a = 0.0;
    for (int w = 0; w < kWarps; ++w) a += s_w[w];
    return a;
  };
  // Cluster total of a scalar: each CTA publishes s_sc[slot], then every CTA
  // sums the published values in rank order.
  auto cluster_total = [&](double cta_val, int slot) -> double {
    if (tid == 0) s_sc[slot] = cta_val;
    cl.sync();
    if (tid == 0) {
      double a = 0.0;
      for (int b = 0; b < CL; ++b) a += cl.map_shared_rank(s_sc, b)[slot];
      s_res[slot] = a;
    }
    __syncthreads();
    return s_res[slot];
  };
  auto cluster_sum_vec = [&](double *buf, int cnt, double *dst) {
    cl.sync();
    for (int j = tid; j < cnt; j += blockDim.x) {
      double acc = 0.0;
      for (int b = 0; b < CL; ++b) acc += cl.map_shared_rank(buf, b)[j];
      dst[j] = acc;
    }
    __syncthreads();
  };
  // partial Q^T c over my rows -> buf[0..kk-1]
  auto qt_partial = [&](double *buf) {
    for (int j = warp; j < kk; j += kWarps) {
      double v = 0.0;
      for (int i = lane; i < nr; i += 32) v += p.Q[(size_t)j * s + r0 + i] * crow[i];
      v = warp_sum(v);
      if (lane == 0) buf[j] = v;
    }
    __syncthreads();
  };
  // out[i] = sum_{j < ncol} Mat[j*s + r0 + i] * coef[j] for my rows; thread
  // (row i, slice h) sums the columns j = h (mod H), slices combined in order.
  auto rows_times_vec = [&](const double *Mat, const double *coef, int ncol, double *out) {
    for (int t = tid; t < H * RB; t += blockDim.x) {
      const int i = t % RB, h = t / RB;
      double v = 0.0;
      if (i < nr)
        for (int j = h; j < ncol; j += H) v += Mat[(size_t)j * s + r0 + i] * coef[j];
      tmp[t] = v;
    }
    __syncthreads();
    for (int i = tid; i < nr; i += blockDim.x) {
      double a = 0.0;
      for (int h = 0; h < H; ++h) a += tmp[h * RB + i];
      out[i] = a;
    }
    __syncthreads();
  };
  // crow -= Q coef over my rows
  auto q_update = [&](const double *coef) {
    rows_times_vec(p.Q, coef, kk, tmp + H * RB);
    for (int i = tid; i < nr; i += blockDim.x) crow[i] -= tmp[H * RB + i];
    __syncthreads();
  };

  // ---- 0. the new column, my rows
  for (int i = tid; i < nr; i += blockDim.x) {
    const int row = r0 + i;
    double c;
    if (p.method == kSFLSQR) {
      c = p.SAZ[(size_t)kk * s + row];
    } else {
      // column k of [S A^T W, S z] H_{k+1,k}: a sum over the band of H
      const double *hb = p.Hband + (size_t)kk * (p.ell + 2);
      c = 0.0;
      const int lo = max(1, k - p.ell);
      for (int j = lo; j <= k + 1; ++j) {
        if (j == k + 1 && lucky) continue;
        c += p.SAtW[(size_t)(j - 1) * s + row] * hb[j - k + p.ell];
      }
    }
    crow[i] = c;
  }
  __syncthreads();

  // ---- 1-4. classical Gram-Schmidt twice against the first kk columns
  if (kk > 0) {
    qt_partial(part0);
    cluster_sum_vec(part0, kk, red);
    q_update(red);
    for (int j = tid; j < kk; j += blockDim.x) rr[j] = red[j];
    __syncthreads();
    qt_partial(part1);
    cluster_sum_vec(part1, kk, red);
    q_update(red);
    for (int j = tid; j < kk; j += blockDim.x) rr[j] += red[j];
    __syncthreads();
  }
  double v = 0.0;
  for (int i = tid; i < nr; i += blockDim.x) v += crow[i] * crow[i];
  const double rho = sqrt(cluster_total(cta_total(v), 0));
  const double R11 = (k == 1) ? rho : st->R11;
  if (!(rho > 1e-300) || !(rho > 1e-14 * R11) || !isfinite(rho)) {
    cl.sync();   // no CTA leaves while a peer may still read its shared memory
    if (rank == 0 && tid == 0) {
      st->stop = isfinite(rho) ? SFL_STOP_BREAKDOWN : kStopNonfinite;
      if (p.use_cond) cudaGraphSetConditional(p.cond, 0u);
    }
    return;
  }
  // ---- 5. q_k = c / rho, gamma_k = <q_k, e>, e -= gamma_k q_k
  const double irho = 1.0 / rho;
  v = 0.0;
  for (int i = tid; i < nr; i += blockDim.x) {
    const double q = crow[i] * irho;
    p.Q[(size_t)kk * s + r0 + i] = q;
    crow[i] = q;
    v += q * p.e[r0 + i];
  }
  const double gamma = cluster_total(cta_total(v), 1);
  v = 0.0;
  for (int i = tid; i < nr; i += blockDim.x) {
    const double ei = p.e[r0 + i] - gamma * crow[i];
    p.e[r0 + i] = ei;
    v += ei * ei;
  }
  const double enorm2_cta = cta_total(v);
  // ---- 6. column kk of R^{-1} and y_k = [y_{k-1}; 0] + gamma_k R^{-1}[:, kk]
  for (int i = rank * kWarps + warp; i < kk; i += CL * kWarps) {
    double a = 0.0;
    for (int j = i + lane; j < kk; j += 32) a += p.Rinv[(size_t)i * p.maxit + j] * rr[j];
    a = warp_sum(a);
    if (lane == 0) {
      const double u = -a * irho;
      p.Rinv[(size_t)i * p.maxit + kk] = u;
      p.y[i] += gamma * u;
    }
  }
  if (rank == 0 && tid == 0) {
    p.Rinv[(size_t)kk * p.maxit + kk] = irho;
    p.y[kk] = gamma * irho;
  }
  __threadfence();
  double res2 = cluster_total(enorm2_cta, 2);   // its barrier also publishes y in the cluster
  if (p.method == kSFLSMR && p.stop_rule == SFL_STOP_RULE_RESIDUAL) {
    // || S_m b - S_m A Z_k y_k ||, my rows (y staged in shared memory)
    for (int j = tid; j < k; j += blockDim.x) red[j] = __ldcg(p.y + j);
    __syncthreads();
    rows_times_vec(p.SAZ, red, k, tmp + H * RB);
    v = 0.0;
    for (int t = tid; t < nr; t += blockDim.x) {
      const double a = p.sbm[r0 + t] - tmp[H * RB + t];
      v += a * a;
    }
    res2 = cluster_total(cta_total(v), 3);
  }
  cl.sync();   // no CTA leaves while a peer may still read its shared memory
  if (rank == 0 && tid == 0) {
    const double rel = sqrt(res2) / st->stop_den;
    st->relres = rel;
    if (p.relres_hist) p.relres_hist[kk] = rel;
    if (k == 1) st->R11 = rho;
    st->k = k;
    st->hist_pending = 1;
    int stop = 0;
    if (rel < st->tol) stop = SFL_STOP_DISCREPANCY;
    else if (lucky) stop = SFL_STOP_BREAKDOWN;
    else if (k >= p.maxit) stop = SFL_STOP_MAXIT;
    if (!isfinite(rel)) stop = kStopNonfinite;
    st->stop = stop;
    if (p.use_cond) cudaGraphSetConditional(p.cond, stop ? 0u : 1u);
  }
}

// ---------------------------------------------------------------- x = Z y

// x[i] = sum_{j<k} z~_j[i] sig_j y_j (FP64 accumulation).  history: writes x_k
// at row k-1 of `hist` when a step finished since the last call.
template <typename XT>
__global__ void __launch_bounds__(kThreads) solution_kernel(SolveState *st, const XT *Z, int64_t zstride,
                                                            const double *sigZ, const double *y, int64_t n,
                                                            double *x, double *hist) {
  const int k = st->k;
  double *out = x;
  if (hist) {
    if (!st->hist_pending) return;
    out = hist + (size_t)(k - 1) * n;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    double v = 0.0;
    for (int j = 0; j < k; ++j) v += (double)Z[(size_t)j * zstride + i] * (sigZ[j] * y[j]);
    out[i] = v;
  }
}

static __global__ void clear_hist_flag_kernel(SolveState *st) { st->hist_pending = 0; }

// Start-of-solve state: everything zero except the solve parameters.
static __global__ void reset_state_kernel(SolveState *st, uint64_t seed, double eta, double noise_norm, double irw_eps) {
  *st = SolveState();
  st->seed = seed;
  st->eta = eta;
  st->noise_norm = noise_norm;
  st->irw_eps = irw_eps;
}

}  // namespace sfl
