// Batched sFLSQR: Algorithm 1 run independently for R right-hand sides
// through one operator (the multi-sinogram form).  Vectors are interleaved,
// V[i * ld + r] with ld a power of two >= R, so a gather of entry c reads the
// R values of c contiguously and the two products of a step are SpMMs that
// read the matrix once for all right-hand sides.  Every basis vector is kept
// (w~_1..w~_{k+1}, p~_1..p~_k, unnormalised, with per-RHS scales; A z~_j too
// on request), which is what the fixed-k adjoint needs.  A right-hand side
// whose stop test fired is masked out of all later work; the loop runs while
// any right-hand side is active.
//
// Per step k (sFLSQR, Algorithm 1; the MGS coefficients come from one pass of
// window dots through the window Gram matrix, as in the single solve):
//   bscal Z    MGS coefficients of z against p~_{k-l}..p~_{k-1}
//   borth z    p~_k = z - sum c p~ ; z~_k = tau(p~_k)          records ||p~||^2, Gram row
//   bscal A    alpha_k, breakdown, Gram row of p
//   bspmm fwd  A z~_k                                           records ||Az||^2, <w~_j, Az>
//   bscal W    MGS coefficients of A z_k against w~_{k-l}..w~_k (column k of H)
//   borth w    w~_{k+1} = A z_k - sum h w~                     records ||w~||^2, Gram row
//   bscal B    beta_{k+1}, lucky breakdown, Gram row of w
//   bspmm bwd  A^T w~_{k+1}                                     records ||A^T w||^2, <p~_j, A^T w>
//   bsketch    column k of S A Z (per RHS)
//   LS         one thread-block cluster per RHS (ls_step_kernel)
//   bcond      loop condition: any RHS still running
#pragma once
#include "kernels.cuh"

namespace sfl {

constexpr int kBMaxRhs = 256;

enum BScalMode : int { kBScalZ = 0, kBScalAlpha = 1, kBScalW = 2, kBScalBeta = 3 };
enum BSpmmMode : int { kBSpmmInit = 0, kBSpmmFwd = 1, kBSpmmBwd = 2, kBSpmmExplicit = 3 };

template <typename XT>
struct BParams {
  int R, ld;                 // right-hand sides; interleave stride (power of two >= R)
  int64_t m, n;
  int ell, maxit, s;
  int RW, RP;                // ring sizes of the window scalars kept in SolveState
  int *kstep;                // steps completed by the right-hand sides still running
  SolveState *st;            // [R]
  XT *W;                     // [maxit + 1][m][ld]: w~_j in slot j - 1
  XT *P;                     // [maxit][n][ld]: p~_j in slot j - 1
  XT *zbuf;                  // [n][ld]: z~_k = tau(p~_k)
  XT *what;                  // [m][ld], or [maxit][m][ld] when keep_what: A z~_k
  int keep_what;
  XT *zraw;                  // [n][ld]: A^T w~_{k+1}
  double *sigW;              // [R][maxit + 2]: 1/||w~_j||
  double *sigP;              // [R][maxit + 1]: 1/||p~_j||
  double *coef;              // [R][kMaxWindow + 2]: coefficients of the current update (unnormalised basis)
  double *rawscale;          // [R]: scale of the unscaled product output being updated
  double *hband;             // [R][maxit][ell + 2]: h_{jk} (window), h_{k+1,k} last
  double *tband;             // [R][maxit][ell + 1]: MGS coefficients of p (window), alpha_k last
  const double *dw;          // [n] diagonal of tau, or null (identity)
  double *rec;               // per-CTA records [(q * R + r) * rcap + cta]
  int rcap;
  // small problem (per RHS, FP64)
  double *SAZ, *rhs, *e;     // [R][maxit][s], [R][s], [R][s]
  double isz;                // 1/sqrt(zeta)
  const int32_t *skrow; const uint32_t *skent;   // row-major sparse-sign table of S_m
};

__device__ __forceinline__ bool b_active(const SolveState *st, int r) { return __ldcg(&st[r].stop) == 0; }

__device__ __forceinline__ double *b_rec(double *rec, int R, int rcap, int q, int r) {
  return rec + ((size_t)q * R + r) * rcap;
}

// ---------------------------------------------------------------- per-RHS scalars

// One warp per right-hand side: totals of the previous kernel's records
// (lane-strided loads issued together, fixed tree, butterfly), then the
// step's scalars on lane 0.  G: CTAs of the producing kernel.
template <typename XT>
__global__ void __launch_bounds__(kThreads) bscal_kernel(BParams<XT> p, int mode, int G) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x * kWarps + warp;
  if (r >= p.R) return;
  SolveState *st = p.st + r;
  if (__ldcg(&st->stop)) return;
  const int k = *p.kstep + 1;
  int lo, nd;
  if (mode == kBScalZ || mode == kBScalAlpha) { lo = max(1, k - p.ell); nd = k - lo; }
  else { lo = max(1, k - p.ell); nd = k - lo + 1; }
  const int nq = 1 + nd;
  double tot[kMaxWindow + 2];
#pragma unroll
  for (int q = 0; q < kMaxWindow + 2; ++q) {
    double a = 0.0;
    if (q < nq) {
      const double *rq = b_rec(p.rec, p.R, p.rcap, q, r);
      double v[kRedLoads];
#pragma unroll
      for (int t = 0; t < kRedLoads; ++t) {
        const int b = lane + 32 * t;
        v[t] = b < G ? __ldcg(rq + b) : 0.0;
      }
#pragma unroll
      for (int w = kRedLoads / 2; w >= 1; w >>= 1)
#pragma unroll
        for (int t = 0; t < w; ++t) v[t] += v[t + w];
      a = v[0];
      for (int b = lane + 32 * kRedLoads; b < G; b += 32) a += __ldcg(rq + b);
      a = warp_sum(a);
    }
    tot[q] = a;
  }
  if (lane != 0) return;
  const int MW = kMaxWindow + 2;
  double *coef = p.coef + (size_t)r * MW;
  double *sigW = p.sigW + (size_t)r * (p.maxit + 2);
  double *sigP = p.sigP + (size_t)r * (p.maxit + 1);
  if (mode == kBScalZ) {
    // z = A^T w~_k (unscaled): true vector is z / ||w~_k||
    const double rs = sigW[k];
    tot[0] *= rs * rs;
    for (int a = 1; a < nq; ++a) tot[a] *= rs;
    double c[kMaxWindow + 2];
    mgs_coefficients(tot + 1, nd, lo, p.RP, st->sig_p, st->gram_p, c);
    double *tb = p.tband + ((size_t)r * p.maxit + (k - 1)) * (p.ell + 1);
    for (int a = 0; a < nd; ++a) {
      coef[a] = c[a] * sigP[lo + a];             // coefficient of the stored p~
      tb[(lo + a) - k + p.ell] = c[a];
    }
    p.rawscale[r] = rs;
    st->znorm_raw2 = tot[0];
  } else if (mode == kBScalAlpha) {
    const double alpha = sqrt(tot[0]);
    const bool bad = !(alpha > 1e-300) || !(alpha > 1e-14 * sqrt(st->znorm_raw2)) || !isfinite(tot[0]);
    if (bad) { st->stop = isfinite(tot[0]) ? SFL_STOP_BREAKDOWN : kStopNonfinite; return; }
    const double ia = 1.0 / alpha;
    const int ns = ring_slot(k, p.RP);
    st->alpha = alpha;
    st->sig_p[ns] = ia;
    sigP[k] = ia;
    p.tband[((size_t)r * p.maxit + (k - 1)) * (p.ell + 1) + p.ell] = alpha;
    for (int a = 0; a < nd; ++a) {
      const int sa = ring_slot(lo + a, p.RP);
      const double g = tot[1 + a] * st->sig_p[sa] * ia;
      st->gram_p[ns][sa] = g; st->gram_p[sa][ns] = g;
    }
  } else if (mode == kBScalW) {
    // A z~_k (unscaled): true A z_k is it times 1/alpha_k
    const double rs = sigP[k];
    tot[0] *= rs * rs;
    for (int a = 1; a < nq; ++a) tot[a] *= rs;
    double c[kMaxWindow + 2];
    mgs_coefficients(tot + 1, nd, lo, p.RW, st->sig_w, st->gram_w, c);
    double *hb = p.hband + ((size_t)r * p.maxit + (k - 1)) * (p.ell + 2);
    for (int q = 0; q < p.ell + 2; ++q) hb[q] = 0.0;
    for (int a = 0; a < nd; ++a) {
      coef[a] = c[a] * sigW[lo + a];
      hb[(lo + a) - k + p.ell] = c[a];
    }
    p.rawscale[r] = rs;
    st->wnorm_raw2 = tot[0];
  } else {   // kBScalBeta
    const double beta = sqrt(tot[0]);
    if (!isfinite(tot[0])) { st->stop = kStopNonfinite; return; }
    if (!(beta > 1e-300) || !(beta > 1e-14 * sqrt(st->wnorm_raw2))) {
      st->lucky = 1;              // step k is still solved; there is no w_{k+1}
      st->betak = 0.0;
      return;
    }
    const double ib = 1.0 / beta;
    const int ns = ring_slot(k + 1, p.RW);
    st->betak = beta;
    st->sig_w[ns] = ib;
    sigW[k + 1] = ib;
    p.hband[((size_t)r * p.maxit + (k - 1)) * (p.ell + 2) + p.ell + 1] = beta;
    for (int a = 0; a < nd; ++a) {
      const int sa = ring_slot(lo + a, p.RW);
      const double g = tot[1 + a] * st->sig_w[sa] * ib;
      st->gram_w[ns][sa] = g; st->gram_w[sa][ns] = g;
    }
  }
}

// ---------------------------------------------------------------- window updates

// Records of a CTA: per-thread values acc[q] of right-hand side r = tid % ld
// are parked in shared memory and summed over the threads sharing r in order.
template <int NQ>
__device__ __forceinline__ void b_store_records(const double (&acc)[NQ], int nq, double *scr, double *rec, int R,
                                                int rcap, int ld) {
  const int tid = threadIdx.x, per = kThreads / ld;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    if (q < nq) scr[q * kThreads + tid] = acc[q];
  __syncthreads();
  for (int t = tid; t < nq * ld; t += kThreads) {
    const int q = t / ld, r = t % ld;
    if (r >= R) continue;
    double a = 0.0;
    for (int g = 0; g < per; ++g) a += scr[q * kThreads + g * ld + r];
    b_rec(rec, R, rcap, q, r)[blockIdx.x] = a;
  }
}

// Element pass of a window update for every running RHS: thread (row offset
// tid / ld, RHS tid % ld), one contiguous chunk of rows per CTA.
//   side 0: p~_k = z * rawscale - sum_a coef_a p~_{lo+a}; z~_k = tau(p~_k)
//   side 1: w~_{k+1} = A z~_k * rawscale - sum_a coef_a w~_{lo+a}
template <typename XT, int ND>
__device__ __forceinline__ void borth_run(const BParams<XT> &p, int side, int k, int lo, bool act, int r,
                                          double *scr) {
  const int tid = threadIdx.x, per = kThreads / p.ld;
  const int64_t len = side == 0 ? p.n : p.m;
  const XT *raw = side == 0 ? p.zraw : p.what + (p.keep_what ? (size_t)(k - 1) * p.m * p.ld : 0);
  XT *base = side == 0 ? p.P : p.W;
  const int64_t slot_stride = len * p.ld;
  XT *out = base + (size_t)(side == 0 ? k - 1 : k) * slot_stride;
  double coef[ND > 0 ? ND : 1];
  const XT *bv[ND > 0 ? ND : 1];
  double rs = 0.0;
  if (act) {
    rs = p.rawscale[r];
#pragma unroll
    for (int a = 0; a < ND; ++a) {
      coef[a] = p.coef[(size_t)r * (kMaxWindow + 2) + a];
      bv[a] = base + (size_t)(lo + a - 1) * slot_stride;
    }
  }
  double acc[ND + 1];
#pragma unroll
  for (int a = 0; a <= ND; ++a) acc[a] = 0.0;
  const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(len, i0 + chunk);
  if (act)
    for (int64_t i = i0 + tid / p.ld; i < i1; i += per) {
      const size_t e = (size_t)i * p.ld + r;
      double v = (double)raw[e] * rs;
      double old[ND > 0 ? ND : 1];
#pragma unroll
      for (int a = 0; a < ND; ++a) { old[a] = (double)bv[a][e]; v -= coef[a] * old[a]; }
      const XT vx = (XT)v;
      out[e] = vx;
      const double vd = (double)vx;
      acc[0] += vd * vd;
#pragma unroll
      for (int a = 0; a < ND; ++a) acc[1 + a] += vd * old[a];
      if (side == 0) p.zbuf[e] = (XT)(p.dw ? p.dw[i] * vd : vd);
    }
  b_store_records<ND + 1>(acc, ND + 1, scr, p.rec, p.R, p.rcap, p.ld);
}

template <typename XT>
__global__ void __launch_bounds__(kThreads) borth_kernel(BParams<XT> p, int side) {
  __shared__ double scr[(kMaxWindow + 2) * kThreads];
  const int r = threadIdx.x % p.ld;
  const int k = *p.kstep + 1;
  const bool act = r < p.R && b_active(p.st, r);
  const int lo = max(1, k - p.ell), nd = side == 0 ? k - lo : k - lo + 1;
  switch (nd) {
    case 0: borth_run<XT, 0>(p, side, k, lo, act, r, scr); break;
    case 1: borth_run<XT, 1>(p, side, k, lo, act, r, scr); break;
    case 2: borth_run<XT, 2>(p, side, k, lo, act, r, scr); break;
    case 3: borth_run<XT, 3>(p, side, k, lo, act, r, scr); break;
    case 4: borth_run<XT, 4>(p, side, k, lo, act, r, scr); break;
    case 5: borth_run<XT, 5>(p, side, k, lo, act, r, scr); break;
    case 6: borth_run<XT, 6>(p, side, k, lo, act, r, scr); break;
    case 7: borth_run<XT, 7>(p, side, k, lo, act, r, scr); break;
    case 8: borth_run<XT, 8>(p, side, k, lo, act, r, scr); break;
    default: borth_run<XT, 9>(p, side, k, lo, act, r, scr); break;
  }
}

// ---------------------------------------------------------------- SpMM

struct BSpmmArgs {
  const int32_t *rowptr, *col;
  const void *val;
  int64_t rows;
  const int32_t *crow;       // row range of every CTA (gridDim.x + 1), balanced by cost
  int mode;
  // kBSpmmExplicit: y (=|+=) A x for the given interleaved vectors, no records;
  // a right-hand side takes part iff jstep <= kr[r]
  const void *xe;
  void *ye;
  int accumulate;
  const int *kr;
  int jstep;
  const int32_t *orig;       // stored row i is operator row orig[i] (used by the ORIG instances)
  int slot;                  // entries per lane-interleaved chunk slot (used by the ILV instances)
};


// Largest chunk slot of a stored row (32 lanes x 8 entries).
constexpr int kMaxSlot = 256;

template <typename XT> struct XT2;
template <> struct XT2<double> { using T = double2; };
template <> struct XT2<float> { using T = float2; };

// Y[row][r] = sum_e val[e] * X[col[e]][r] for the RHS of tile blockIdx.y (T of
// them).  A CTA owns a contiguous range of rows and its warps take every
// kWarps-th row, so they work on adjacent rows (neighbouring rays, or pixels)
// at the same time and share the gathered lines in L1.  A warp owns one row at
// a time and walks its stored entries in order; lanes split the tile's RHS
// (T >= 32: T/32 per lane) or, for T < 32, 32/T lane groups split the entries.
// Every (row, RHS) sum is ((s0 + s1) + (s2 + s3)) with s_j the in-order sum of
// the stored entries e = j (mod 4) of the row, whatever T is, so the tile
// width chosen by the tuner never changes a result bit.  Window dots
// <v_a, y> and ||y||^2 per RHS go to the records.  ORIG: stored row i is
// operator row orig[i] (pixel-tiled plans); a compile-time flag, because the
// dependent index load costs the untiled loops 13%.  ILV: the plan stores
// every chunk slot lane-interleaved (entry q * A + c of a slot of A chunks at
// c * PL + q); the warp's lanes then load the slot's chunks at once (vector
// loads spread over the lanes) and the warp reads it back in operator order
// through shared memory, so the streams, and every bit, are those of an
// operator-order plan's walk.  Both walks are unrolled 8 deep, so a warp has up
// to 8 chunks' gathers in flight (the SpMM is bound by gather latency and L2
// bandwidth, not by the matrix stream).
template <typename VT, typename XT, int T, bool ORIG, bool ILV>
__global__ void __launch_bounds__(kThreads, 4) bspmm_kernel(BParams<XT> p, BSpmmArgs a) {
  static_assert(T == 8 || T == 16 || T == 32 || T == 64, "tile widths");
  constexpr int PL = LoadWidth<VT>::P;
  constexpr int RPL = T >= 32 ? T / 32 : 1;       // RHS per lane
  constexpr int NG = T >= 32 ? 1 : 32 / T;        // lane groups splitting the entries
  using ACC = typename AccT<XT>::T;
  __shared__ double scr[kWarps][T];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = *p.kstep + 1;
  const int tile0 = blockIdx.y * T;
  const int g = lane / (32 / NG), gl = lane % (32 / NG);   // group, lane within group
  const bool owner = NG == 1 || g == 0;                    // lanes that hold the row results
  // this lane's RHS and their activity
  int rr[RPL];
  bool act[RPL];
  bool any = false;
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    rr[q] = tile0 + (T >= 32 ? RPL * lane + q : gl);
    act[q] = rr[q] < p.R && (a.mode == kBSpmmExplicit ? a.jstep <= a.kr[rr[q]] : b_active(p.st, rr[q]));
    any |= act[q];
  }
  const bool tile_any = __syncthreads_or(any);
  const XT *x;
  XT *y;
  const XT *win = nullptr;
  int lo = 1, nd = 0;
  if (a.mode == kBSpmmInit) { x = p.W; y = p.zraw; }
  else if (a.mode == kBSpmmExplicit) { x = (const XT *)a.xe; y = (XT *)a.ye; }
  else if (a.mode == kBSpmmFwd) {
    x = p.zbuf;
    y = p.what + (p.keep_what ? (size_t)(k - 1) * p.m * p.ld : 0);
    lo = max(1, k - p.ell); nd = k - lo + 1;        // w~_lo .. w~_k
    win = p.W;
  } else {
    x = p.W + (size_t)k * p.m * p.ld;               // w~_{k+1}
    y = p.zraw;
    lo = max(1, k + 1 - p.ell); nd = k - lo + 1;    // p~_lo .. p~_k
    win = p.P;
  }
  const int64_t wslot = (a.mode == kBSpmmFwd ? p.m : p.n) * p.ld;
  const int64_t r0 = a.crow[blockIdx.x], r1 = a.crow[blockIdx.x + 1];
  double nrm[RPL];
#pragma unroll
  for (int q = 0; q < RPL; ++q) nrm[q] = 0.0;
  if (tile_any) {
    for (int64_t row = r0 + warp; row < r1; row += kWarps) {
      const int beg = a.rowptr[row], end = a.rowptr[row + 1];
      ACC s[4][RPL];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int q = 0; q < RPL; ++q) s[j][q] = (ACC)0;
      if constexpr (ILV) {
        // slot by slot: lane c < A loads chunk c and writes entry q * A + c to
        // the warp's buffer; the warp reads PL entries at a time in order
        // (slot0 and e0 are multiples of 4: entry e0 + u is in stream u mod 4)
        __shared__ int s_col[kWarps][kMaxSlot];
        __shared__ ACC s_val[kWarps][kMaxSlot];
        int *bc = s_col[warp];
        ACC *bv = s_val[warp];
        for (int slot0 = 0; slot0 < end - beg; slot0 += a.slot) {
          const int A = min(a.slot, end - beg - slot0) / PL;
          __syncwarp();
          if (lane < A) {
            Chunk<VT, PL> ch;
            ch.load(a.col, (const VT *)a.val, beg + slot0 + lane * PL);
#pragma unroll
            for (int q = 0; q < PL; ++q) {
              bc[q * A + lane] = ch.c[q];
              bv[q * A + lane] = (ACC)ch.v[q];
            }
          }
          __syncwarp();
#pragma unroll 8
          for (int e0 = 0; e0 < A * PL; e0 += PL) {
#pragma unroll
            for (int u = 0; u < PL; ++u) {
              const int j = u & 3;
              if (NG > 1 && (j % NG) != g) continue;
              const XT *xr = x + (size_t)bc[e0 + u] * p.ld + tile0;
              const ACC v = bv[e0 + u];
              if (RPL == 2) {
                if (act[0] || act[1]) {
                  const typename XT2<XT>::T xv = *reinterpret_cast<const typename XT2<XT>::T *>(xr + 2 * lane);
                  s[j][0] += v * (ACC)xv.x;
                  s[j][RPL - 1] += v * (ACC)xv.y;
                }
              } else if (act[0]) {
                s[j][0] += v * (ACC)xr[T >= 32 ? lane : gl];
              }
            }
          }
        }
      } else {
        // chunks of PL entries (rows start at multiples of PL), every lane
        // loads the same chunk (broadcast); group g takes the entries
        // e = j (mod 4) with j = g (mod NG)
#pragma unroll 8
        for (int off = beg; off < end; off += PL) {
          Chunk<VT, PL> c;
          c.load(a.col, (const VT *)a.val, off);
#pragma unroll
          for (int e = 0; e < PL; ++e) {
            const int j = e & 3;
            if (NG > 1 && (j % NG) != g) continue;
            const XT *xr = x + (size_t)c.c[e] * p.ld + tile0;
            if (RPL == 2) {
              if (act[0] || act[1]) {
                const typename XT2<XT>::T xv = *reinterpret_cast<const typename XT2<XT>::T *>(xr + 2 * lane);
                s[j][0] += (ACC)c.v[e] * (ACC)xv.x;
                s[j][RPL - 1] += (ACC)c.v[e] * (ACC)xv.y;
              }
            } else if (act[0]) {
              s[j][0] += (ACC)c.v[e] * (ACC)xr[T >= 32 ? lane : gl];
            }
          }
        }
      }
      // combine the four streams in one fixed tree (groups exchange by shuffle)
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        ACC s0 = s[0][q], s1 = s[1][q], s2 = s[2][q], s3 = s[3][q];
        if (NG == 2) {            // group 0 holds s0, s2; group 1 holds s1, s3
          s1 = __shfl_xor_sync(0xffffffffu, s[1][q], 16);
          s3 = __shfl_xor_sync(0xffffffffu, s[3][q], 16);
        } else if (NG == 4) {     // group j holds s_j
          s1 = __shfl_xor_sync(0xffffffffu, s[1][q], 8);
          s2 = __shfl_xor_sync(0xffffffffu, s[2][q], 16);
          s3 = __shfl_xor_sync(0xffffffffu, s[3][q], 24);
        }
        const ACC tot = (s0 + s1) + (s2 + s3);
        if (owner && act[q]) {
          XT *yo = y + (size_t)(ORIG ? a.orig[row] : row) * p.ld + rr[q];
          if (a.accumulate) { *yo = (XT)((ACC)*yo + tot); continue; }
          *yo = (XT)tot;
          const double yd = (double)(XT)tot;
          nrm[q] += yd * yd;
        }
      }
    }
  }
  // records: ||y||^2, then <v_w, y> one window vector at a time over the
  // warp's own rows (each lane re-reads the outputs it stored); per RHS of the
  // tile the warps are added in order
  auto store = [&](const double (&v)[RPL], int q) {
#pragma unroll
    for (int j = 0; j < RPL; ++j)
      if (owner) scr[warp][T >= 32 ? RPL * lane + j : gl] = v[j];
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += kThreads) {
      const int r = tile0 + t;
      if (r >= p.R) continue;
      double acc = 0.0;
      for (int w = 0; w < kWarps; ++w) acc += scr[w][t];
      b_rec(p.rec, p.R, p.rcap, q, r)[blockIdx.x] = acc;
    }
    __syncthreads();
  };
  if (a.mode == kBSpmmExplicit) return;
  store(nrm, 0);
  for (int w = 0; w < nd; ++w) {
    const XT *wv = win + (size_t)(lo + w - 1) * wslot;
    double d[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) d[q] = 0.0;
    if (tile_any && owner)
      for (int64_t row = r0 + warp; row < r1; row += kWarps)
#pragma unroll
        for (int q = 0; q < RPL; ++q)
          if (act[q]) {
            const size_t ei = (size_t)(ORIG ? a.orig[row] : row) * p.ld + rr[q];
            d[q] += (double)y[ei] * (double)wv[ei];
          }
    store(d, 1 + w);
  }
}

// ---------------------------------------------------------------- sketch

// Column k of S_m A Z for every running RHS (mode 0), or S_m b (mode 1, from
// the FP64 column-major right-hand sides).  CTA (sketch row, 32-RHS chunk),
// lane = RHS.  A row holds zeta * m / s entries (thousands when s is small),
// so kBSkWarps warps split them (warp w takes the entries w, w + kBSkWarps,
// ...) and each warp keeps kBSkBatch table loads, then kBSkBatch gathers, in
// flight: the walk is a chain of L2 round trips, not a bandwidth stream.
// Entry u of a warp's batch goes to accumulator u mod 2; the warps' partial
// sums are added as a fixed tree.
constexpr int kBSkWarps = 16;
constexpr int kBSkBatch = 8;

template <typename XT>
__global__ void __launch_bounds__(kBSkWarps * 32) bsketch_kernel(BParams<XT> p, int mode, const double *B) {
  __shared__ double part[kBSkWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = blockIdx.x, r = blockIdx.y * 32 + lane;
  const bool act = r < p.R && b_active(p.st, r);
  const int k = *p.kstep + 1;
  const int b0 = p.skrow[row], b1 = p.skrow[row + 1];
  constexpr int STEP = kBSkWarps * kBSkBatch;
  double a = 0.0;
  if (act) {
    if (mode == 0) {
      const XT *v = p.what + (p.keep_what ? (size_t)(k - 1) * p.m * p.ld : 0) + r;
      using ACC = typename AccT<XT>::T;
      ACC c[2] = {(ACC)0, (ACC)0};
      for (int i0 = b0 + warp; i0 < b1; i0 += STEP) {
        uint32_t e[kBSkBatch];
#pragma unroll
        for (int u = 0; u < kBSkBatch; ++u) {
          const int i = i0 + u * kBSkWarps;
          e[u] = i < b1 ? __ldg(p.skent + i) : 0u;
        }
        ACC x[kBSkBatch];
#pragma unroll
        for (int u = 0; u < kBSkBatch; ++u)
          x[u] = i0 + u * kBSkWarps < b1 ? flip_sign((ACC)v[(size_t)(e[u] & 0x7FFFFFFFu) * p.ld], e[u]) : (ACC)0;
#pragma unroll
        for (int u = 0; u < kBSkBatch; ++u)
          if (i0 + u * kBSkWarps < b1) c[u & 1] += x[u];
      }
      a = (double)(c[0] + c[1]);
    } else {
      const double *v = B + (size_t)r * p.m;
      double c[2] = {0.0, 0.0};
      for (int i0 = b0 + warp; i0 < b1; i0 += STEP) {
        uint32_t e[kBSkBatch];
#pragma unroll
        for (int u = 0; u < kBSkBatch; ++u) {
          const int i = i0 + u * kBSkWarps;
          e[u] = i < b1 ? __ldg(p.skent + i) : 0u;
        }
        double x[kBSkBatch];
#pragma unroll
        for (int u = 0; u < kBSkBatch; ++u)
          x[u] = i0 + u * kBSkWarps < b1 ? flip_sign(v[e[u] & 0x7FFFFFFFu], e[u]) : 0.0;
#pragma unroll
        for (int u = 0; u < kBSkBatch; ++u)
          if (i0 + u * kBSkWarps < b1) c[u & 1] += x[u];
      }
      a = c[0] + c[1];
    }
  }
  part[warp][lane] = a;
  __syncthreads();
  if (warp != 0 || !act) return;
  static_assert(kBSkWarps == 16, "warp totals are added as a 4-level tree");
  double w[kBSkWarps];
#pragma unroll
  for (int q = 0; q < kBSkWarps; ++q) w[q] = part[q][lane];
#pragma unroll
  for (int h = kBSkWarps / 2; h >= 1; h >>= 1)
#pragma unroll
    for (int q = 0; q < h; ++q) w[q] += w[q + h];
  const double t = w[0];
  if (mode == 0) {
    const double sc = p.isz * p.sigP[(size_t)r * (p.maxit + 1) + k];
    p.SAZ[((size_t)r * p.maxit + (k - 1)) * p.s + row] = t * sc;
  } else {
    const double v = t * p.isz;
    p.rhs[(size_t)r * p.s + row] = v;
    p.e[(size_t)r * p.s + row] = v;
  }
}

// ---------------------------------------------------------------- loop control, init, solution

// After every RHS's small solve: the loop continues while any RHS runs.
template <typename XT>
__global__ void bcond_kernel(BParams<XT> p, cudaGraphConditionalHandle h, int use_cond) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int r = threadIdx.x; r < p.R; r += blockDim.x)
    if (__ldcg(&p.st[r].stop) == 0) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    *p.kstep += 1;
    if (use_cond) cudaGraphSetConditional(h, any ? 1u : 0u);
  }
}

// Start-of-solve state for every RHS.
template <typename XT>
__global__ void breset_kernel(BParams<XT> p, uint64_t seed, double eta, const double *noise, double irw_eps) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r == 0) *p.kstep = 0;
  if (r >= p.R) return;
  SolveState s = SolveState();
  s.seed = seed;
  s.eta = eta;
  s.noise_norm = noise[r];
  s.irw_eps = irw_eps;
  p.st[r] = s;
}

// beta_r = ||b_r|| (one CTA per RHS over the FP64 column), w~_1 = b_r stored
// unscaled with scale 1/beta_r; tolerance eta * delta_r / beta_r.
template <typename XT>
__global__ void __launch_bounds__(kThreads) binit_norm_kernel(BParams<XT> p, const double *B) {
  __shared__ double wt[kWarps];
  const int r = blockIdx.x;
  const double *b = B + (size_t)r * p.m;
  double a0 = 0.0, a1 = 0.0;
  int64_t i = threadIdx.x;
  for (; i + kThreads < p.m; i += 2 * kThreads) { a0 += b[i] * b[i]; a1 += b[i + kThreads] * b[i + kThreads]; }
  if (i < p.m) a0 += b[i] * b[i];
  const double v = warp_sum(a0 + a1);
  if ((threadIdx.x & 31) == 0) wt[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double t = ((wt[0] + wt[1]) + (wt[2] + wt[3])) + ((wt[4] + wt[5]) + (wt[6] + wt[7]));
  SolveState *st = p.st + r;
  const double beta = sqrt(t);
  st->beta0 = beta;
  st->sig_w[ring_slot(1, p.RW)] = 1.0 / beta;
  p.sigW[(size_t)r * (p.maxit + 2) + 1] = 1.0 / beta;
  st->tol = (st->noise_norm > 0.0) ? st->eta * st->noise_norm / beta : 0.0;
  if (!(beta > 0.0)) st->stop = SFL_STOP_BREAKDOWN;
  if (!isfinite(t)) st->stop = kStopNonfinite;
}
static_assert(kWarps == 8, "binit_norm_kernel adds eight warp totals");

// Interleave column-major FP64 data into [len][ld] (tiles of 32 x 32):
// dst[i * ld + r] = (XT) src[r * len + i] for r < R.
template <typename XT>
__global__ void binterleave_kernel(const double *src, int64_t len, int R, int ld, XT *dst) {
  __shared__ double t[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int j = ty; j < 32; j += 8) {
    const int r = r0 + j;
    const int64_t i = i0 + tx;
    t[j][tx] = (r < R && i < len) ? src[(size_t)r * len + i] : 0.0;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t i = i0 + j;
    const int r = r0 + tx;
    if (i < len && r < ld) dst[(size_t)i * ld + r] = (XT)t[tx][j];
  }
}

// x_r = tau(sum_{j <= k_r} p~_j sigP_j y_j) written column-major FP64 (tiles
// of 32 rows x 32 RHS; the sum over j runs in FP64).
template <typename XT>
__global__ void bsolution_kernel(BParams<XT> p, const double *Y, double *X, int hist) {
  __shared__ double t[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  const int r = r0 + tx;
  // hist: inside the loop, after the small problems of step k = kstep + 1;
  // X points at the history and only right-hand sides that completed step k
  // write their iterate, to X + (k - 1) * R * n
  int kh = 0;
  if (hist) {
    kh = __ldcg(p.kstep) + 1;
    X += (size_t)(kh - 1) * p.R * p.n;
  }
  int kr = 0;
  if (r < p.R) kr = __ldcg(&p.st[r].k);
  for (int j = ty; j < 32; j += 8) {
    const int64_t i = i0 + j;
    double v = 0.0;
    if (r < p.R && i < p.n) {
      const double *y = Y + (size_t)r * p.maxit;
      const double *sp = p.sigP + (size_t)r * (p.maxit + 1);
      for (int q = 0; q < kr; ++q) v += (double)p.P[((size_t)q * p.n + i) * p.ld + r] * (sp[q + 1] * y[q]);
      if (p.dw) v *= p.dw[i];
    }
    t[j][tx] = v;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int rr = r0 + j;
    const int64_t i = i0 + tx;
    if (rr < p.R && i < p.n && (!hist || __ldcg(&p.st[rr].k) == kh)) X[(size_t)rr * p.n + i] = t[tx][j];
  }
}

}  // namespace sfl
