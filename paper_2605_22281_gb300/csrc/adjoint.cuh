// Reverse-mode adjoint of a fixed-k batched sFLSQR solve (Algorithm 1 with
// the flexible operator tau = diag(d), no stop test): given xbar = dL/dx for
// every right-hand side, it returns bbar = dL/db and dbar = dL/dd (summed over
// the right-hand sides).  The forward keeps every basis vector, A z~_j, the
// MGS coefficients, the norms and the small QR; the reverse sweep runs the
// steps backwards, each as
//   m side: normalisation and window-MGS adjoints of w (dots through the
//           window Gram matrix, as in the forward), with S^T of the sketched
//           matrix's adjoint column added to the adjoint of A z_j;
//   u = A^T (adjoint of A z_j)               (SpMM)
//   n side: p-bar_j += d * (u + y_j xbar) and dbar += p_j * (u + y_j xbar),
//           then normalisation and window-MGS adjoints of p;
//   w-bar_j += A t-bar_j                     (SpMM)
// The generic kernels below (dots of up to 8 vectors, linear combinations of
// up to 8 inputs into up to 6 outputs, per-RHS coefficients) carry it.
#pragma once
#include "batched.cuh"

namespace sfl {

constexpr int kAdjNV = 8;     // vectors per dot pass / inputs per combination
constexpr int kAdjNO = 6;     // outputs per combination
constexpr int kAdjNQ = kAdjNV * kAdjNV;   // record slots of a dot pass (pairs a <= b, slot a * 8 + b)
constexpr int kAdjRG = 8;                 // dot pairs reduced per round of the records

// One interleaved vector of a pass: element e = i * ld + r of `p` (XT, or
// FP64 when dbl), times scale[r * sstride] when scale is set, times d[i] when
// dmul.
struct AVec {
  const void *p;
  int dbl;
  const double *scale;
  int64_t sstride;
  int dmul;
};

struct AOut {
  void *p;
  int dbl;
  int accumulate;   // 0: overwrite, 1: add
};

struct AArgs {
  int R, ld;
  int64_t len;                 // rows of the vectors (n or m)
  const double *d;             // [n] or null
  const int *kr;               // [R]: steps of each right-hand side
  int jstep;                   // a right-hand side takes part iff jstep <= kr[r]
  int nv;                      // vectors (dot pass) or inputs (combination)
  AVec v[kAdjNV];
  int no;                      // outputs (combination)
  AOut o[kAdjNO];
  const double *coef;          // [R][kAdjNO][kAdjNV] (combination)
  double *rec;                 // [kAdjNQ][R][rcap] (dot pass)
  int rcap;
};

// Element arithmetic of the passes runs in AT = AccT<XT>::T: FP64 for FP64
// vectors, FP32 for FP32 vectors (whose entries are FP32-rounded anyway).  On
// this GPU an FP64 instruction costs about 64 times an FP32 one, which made
// the FP32 passes FP64-bound.  Sums across threads stay FP64.
// The per-RHS scale of every input is loaded and converted once per thread
// (a thread keeps one RHS); d[i] once per element.
template <typename AT>
struct AFactors {
  AT sc[kAdjNV];   // scale[r * sstride], or 1
  bool needd;      // some input is multiplied by d[i]
};

template <typename AT>
__device__ __forceinline__ AFactors<AT> a_factors(const AArgs &a, int r) {
  AFactors<AT> f;
  f.needd = false;
#pragma unroll
  for (int l = 0; l < kAdjNV; ++l) {
    const bool on = l < a.nv;
    f.sc[l] = (on && a.v[l].scale) ? (AT)a.v[l].scale[(size_t)r * a.v[l].sstride] : (AT)1;
    f.needd |= on && a.v[l].dmul;
  }
  return f;
}

// Element e of input v: (value * scale) * d[i], the factors precomputed.
template <typename XT, typename AT>
__device__ __forceinline__ AT a_elem(const AVec &v, size_t e, AT sc, AT di) {
  AT x = v.dbl ? (AT)((const double *)v.p)[e] : (AT)((const XT *)v.p)[e];
  if (v.scale) x *= sc;
  if (v.dmul) x *= di;
  return x;
}

__device__ __forceinline__ bool a_active(const AArgs &a, int r) { return r < a.R && a.jstep <= a.kr[r]; }

// All pairwise dots <v_a, v_b> (a <= b < nv) per right-hand side: per-CTA
// records in slot a * 8 + b.  Thread (row offset tid / ld, RHS tid % ld), one
// contiguous chunk of rows per CTA.
template <typename XT>
__global__ void __launch_bounds__(kThreads) adot_kernel(AArgs a) {
  using AT = typename AccT<XT>::T;
  __shared__ double scr[kAdjRG * kThreads];
  const int tid = threadIdx.x, per = kThreads / a.ld, r = tid % a.ld;
  const bool act = a_active(a, r);
  AT acc[kAdjNV][kAdjNV];
#pragma unroll
  for (int x = 0; x < kAdjNV; ++x)
#pragma unroll
    for (int y = 0; y < kAdjNV; ++y) acc[x][y] = (AT)0;
  const int64_t chunk = (a.len + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(a.len, i0 + chunk);
  if (act) {
    const AFactors<AT> f = a_factors<AT>(a, r);
    for (int64_t i = i0 + tid / a.ld; i < i1; i += per) {
      const size_t e = (size_t)i * a.ld + r;
      const AT di = f.needd ? (AT)a.d[i] : (AT)1;
      AT val[kAdjNV];
#pragma unroll
      for (int x = 0; x < kAdjNV; ++x) val[x] = x < a.nv ? a_elem<XT, AT>(a.v[x], e, f.sc[x], di) : (AT)0;
#pragma unroll
      for (int x = 0; x < kAdjNV; ++x)
#pragma unroll
        for (int y = x; y < kAdjNV; ++y)
          if (y < a.nv) acc[x][y] += val[x] * val[y];
    }
  }
  // records, kAdjRG pairs per round: every thread parks its values of the
  // round's pairs, then thread (pair, r) adds the per threads sharing r with
  // four interleaved partial sums (g mod 4), combined as a fixed tree
  const int npair = a.nv * (a.nv + 1) / 2;
  for (int p0 = 0; p0 < npair; p0 += kAdjRG) {
    int q = 0;
#pragma unroll
    for (int x = 0; x < kAdjNV; ++x)
#pragma unroll
      for (int y = x; y < kAdjNV; ++y) {
        if (y < a.nv) {
          if (q >= p0 && q < p0 + kAdjRG) scr[(q - p0) * kThreads + tid] = (double)acc[x][y];
          ++q;
        }
      }
    __syncthreads();
    const int nq = min(kAdjRG, npair - p0);
    for (int t = tid; t < nq * a.ld; t += kThreads) {
      const int qq = t / a.ld, rr = t - qq * a.ld;
      if (rr >= a.R) continue;
      const double *sv = scr + qq * kThreads + rr;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      for (int g = 0; g < per; g += 4) {
        s0 += sv[g * a.ld];
        if (g + 1 < per) s1 += sv[(g + 1) * a.ld];
        if (g + 2 < per) s2 += sv[(g + 2) * a.ld];
        if (g + 3 < per) s3 += sv[(g + 3) * a.ld];
      }
      const double s = (s0 + s1) + (s2 + s3);
      // pair index p0 + qq -> (x, y), row-major over the upper triangle
      int x = 0, rem = p0 + qq;
      while (rem >= a.nv - x) { rem -= a.nv - x; ++x; }
      a.rec[((size_t)(x * kAdjNV + x + rem) * a.R + rr) * a.rcap + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

// out_o (=|+=) sum_l coef[r][o][l] * v_l for every running right-hand side.
template <typename XT>
__global__ void __launch_bounds__(kThreads) alin_kernel(AArgs a) {
  using AT = typename AccT<XT>::T;
  const int tid = threadIdx.x, per = kThreads / a.ld, r = tid % a.ld;
  if (!a_active(a, r)) return;
  AT c[kAdjNO][kAdjNV];
#pragma unroll
  for (int o = 0; o < kAdjNO; ++o)
#pragma unroll
    for (int l = 0; l < kAdjNV; ++l)
      c[o][l] = (o < a.no && l < a.nv) ? (AT)a.coef[((size_t)r * kAdjNO + o) * kAdjNV + l] : (AT)0;
  const AFactors<AT> f = a_factors<AT>(a, r);
  const int64_t chunk = (a.len + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(a.len, i0 + chunk);
  for (int64_t i = i0 + tid / a.ld; i < i1; i += per) {
    const size_t e = (size_t)i * a.ld + r;
    const AT di = f.needd ? (AT)a.d[i] : (AT)1;
    AT val[kAdjNV];
#pragma unroll
    for (int l = 0; l < kAdjNV; ++l) val[l] = l < a.nv ? a_elem<XT, AT>(a.v[l], e, f.sc[l], di) : (AT)0;
#pragma unroll
    for (int o = 0; o < kAdjNO; ++o) {
      if (o >= a.no) continue;
      AT s = (AT)0;
#pragma unroll
      for (int l = 0; l < kAdjNV; ++l) s += c[o][l] * val[l];
      if (a.o[o].dbl) {
        double *q = (double *)a.o[o].p + e;
        *q = a.o[o].accumulate ? *q + (double)s : (double)s;
      } else {
        XT *q = (XT *)a.o[o].p + e;
        *q = a.o[o].accumulate ? (XT)((AT)*q + s) : (XT)s;
      }
    }
  }
}

// n side, step j: pbar_j += d * (u + y_j xbar); dbar += p_j * (u + y_j xbar),
// with p_j = sigP_j p~_j.  v[0] = u, v[1] = xbar (scale y_j), v[2] = p~_j
// (scale sigP_j); o[0] = pbar_j, o[1] = dbar accumulator (FP64).
template <typename XT>
__global__ void __launch_bounds__(kThreads) apre_kernel(AArgs a) {
  using AT = typename AccT<XT>::T;
  const int tid = threadIdx.x, per = kThreads / a.ld, r = tid % a.ld;
  if (!a_active(a, r)) return;
  const int64_t chunk = (a.len + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(a.len, i0 + chunk);
  const AFactors<AT> f = a_factors<AT>(a, r);
  for (int64_t i = i0 + tid / a.ld; i < i1; i += per) {
    const size_t e = (size_t)i * a.ld + r;
    const AT di = (AT)a.d[i];
    const AT zb = a_elem<XT, AT>(a.v[0], e, f.sc[0], di) + a_elem<XT, AT>(a.v[1], e, f.sc[1], di);
    const AT pj = a_elem<XT, AT>(a.v[2], e, f.sc[2], di);
    XT *pb = (XT *)a.o[0].p + e;
    *pb = (XT)((AT)*pb + di * zb);
    double *db = (double *)a.o[1].p + e;   // the d-bar accumulator stays FP64
    *db += (double)(pj * zb);
  }
}

// Totals of dot pass records for one right-hand side: tot[x][y] for the
// pairs x <= y < nv (and the mirrored entries).  Warp w sums the pairs w,
// w + kWarps, ...: each lane issues its kRedLoads record loads at once (lanes
// over the producer's CTAs), adds them as a fixed tree, then the lanes fold
// with a butterfly.  tot: shared memory.  All threads call.
__device__ __forceinline__ void a_totals(const double *rec, int R, int rcap, int r, int G, int nv,
                                         double (*tot)[kAdjNV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int npair = nv * (nv + 1) / 2;
  for (int q = warp; q < npair; q += kWarps) {
    int x = 0, rem = q;   // pair q in row-major order of the upper triangle
    while (rem >= nv - x) { rem -= nv - x; ++x; }
    const int y = x + rem;
    const double *rq = rec + ((size_t)(x * kAdjNV + y) * R + r) * rcap;
    double v[kRedLoads];
#pragma unroll
    for (int u = 0; u < kRedLoads; ++u) {
      const int b = lane + 32 * u;
      v[u] = b < G ? rq[b] : 0.0;
    }
#pragma unroll
    for (int w = kRedLoads / 2; w >= 1; w >>= 1)
#pragma unroll
      for (int u = 0; u < w; ++u) v[u] += v[u + w];
    double s = v[0];
    for (int b = lane + 32 * kRedLoads; b < G; b += 32) s += rq[b];
    s = warp_sum(s);
    if (lane == 0) { tot[x][y] = s; tot[y][x] = s; }
  }
  __syncthreads();
}

enum AScalMode : int { kAScalM = 0, kAScalN = 1, kAScalFinal = 2, kAScalYbar = 3 };

struct AScalArgs {
  int R, maxit, ell, j, mode, G, nv;
  const int *kr;
  const double *rec;
  int rcap;
  const double *sigW, *sigP;     // [R][maxit + 2], [R][maxit + 1]
  const double *hband, *tband;   // [R][maxit][ell + 2], [R][maxit][ell + 1]
  const SolveState *st;
  double *coef;                  // [R][kAdjNO][kAdjNV]
  double *ybar;                  // [R][maxit] (kAScalYbar: columns j0..j0+nv-2)
};

// Per-RHS algebra of a reverse step (one CTA per right-hand side: the
// record totals use every warp, the algebra runs in thread 0).
//  m side (vectors 0: wbar_{j+1}, 1: w_{j+1}, 2..: w_lo..w_j):
//    s = <w_{j+1}, wbar>; q0 = (wbar - s w_{j+1}) / beta_{j+1};
//    hbar_i = -(<w_i, q0> + sum_{i' > i} hbar_i' <w_i, w_i'>), i descending;
//    outputs (inputs also 2+nw: A z_j, 3+nw: S^T Mbar_j):
//      o0 = adjoint of A z_j = q0 + sum hbar_i w_i + S^T Mbar_j
//      o(1+t) = wbar_i += -h_ij q_i + hbar_i qprev_i  (t = i - lo)
//      o(1+nw) = 0 into wbar_{j+1}'s slot (consumed)
//  n side (vectors 0: pbar_j, 1: p_j, 2..: p_lo..p_{j-1}):
//    s = <p_j, pbar_j>; q0 = (pbar_j - s p_j) / alpha_j;
//    cbar_i = -(<p_i, q0> + sum_{i' > i} cbar_i' <p_i, p_i'>), i descending;
//    outputs: o0 = tbar_j = q0 + sum cbar_i p_i;
//             o(1+t) = pbar_i += -c_ij q_i + cbar_i qprev_i,
//               qprev_i = alpha_j p_j + sum_{i' >= i} c_i'j p_i';
//             o(1+np) = 0 into pbar_j's slot
//  final (vectors 0: wbar_1, 1: w_1): o0 = (wbar_1 - <w_1, wbar_1> w_1) / beta_0
//  ybar (vectors 0: xbar, 1..: z_j0 ...): ybar_{j0 + l - 1} = <xbar, z_{j0 + l - 1}>
__global__ void __launch_bounds__(kThreads) ascal_adj_kernel(AScalArgs a) {
  __shared__ double tot[kAdjNV][kAdjNV];
  const int r = blockIdx.x;
  if (r >= a.R) return;
  const int j = a.j;
  if (a.mode != kAScalFinal && a.mode != kAScalYbar && j > a.kr[r]) return;
  a_totals(a.rec, a.R, a.rcap, r, a.G, a.nv, tot);
  if (threadIdx.x != 0) return;
  double *c = a.coef + (size_t)r * kAdjNO * kAdjNV;
  for (int q = 0; q < kAdjNO * kAdjNV; ++q) c[q] = 0.0;
  auto C = [&](int o, int l) -> double & { return c[o * kAdjNV + l]; };
  if (a.mode == kAScalYbar) {
    for (int l = 1; l < a.nv; ++l) {
      const int jj = j + l - 1;   // j: first column of this pass (1-based)
      if (jj <= a.kr[r]) a.ybar[(size_t)r * a.maxit + jj - 1] = tot[0][l];
    }
    return;
  }
  if (a.mode == kAScalFinal) {
    const double b0 = a.st[r].beta0;
    const double s = tot[0][1];
    C(0, 0) = 1.0 / b0;
    C(0, 1) = -s / b0;
    C(0, 2) = 1.0;      // S^T sbar
    return;
  }
  const int L = a.ell;
  if (a.mode == kAScalM) {
    const int lo = max(1, j - L), nw = j - lo + 1;
    const double *hb = a.hband + ((size_t)r * a.maxit + (j - 1)) * (L + 2);
    const double beta = hb[L + 1];
    const double ib = 1.0 / beta;
    const double s = tot[0][1];
    double hbar[kAdjNV];
    // <w_i, q0> = (<w_i, wbar> - s <w_i, w_{j+1}>) / beta, i = lo + t at vector 2 + t
    for (int t = nw - 1; t >= 0; --t) {
      double v = (tot[0][2 + t] - s * tot[1][2 + t]) * ib;
      for (int u = t + 1; u < nw; ++u) v += hbar[u] * tot[2 + t][2 + u];
      hbar[t] = -v;
    }
    const int VX = 2 + nw, VS = 3 + nw;
    // o0: adjoint of A z_j
    C(0, 0) = ib;
    C(0, 1) = -s * ib;
    for (int t = 0; t < nw; ++t) C(0, 2 + t) = hbar[t];
    C(0, VS) = 1.0;
    // wbar_i updates
    for (int t = 0; t < nw; ++t) {
      const double h = hb[(lo + t) - j + L];
      C(1 + t, 0) = -h * ib;
      C(1 + t, 1) = h * s * ib;
      for (int u = t + 1; u < nw; ++u) C(1 + t, 2 + u) += -h * hbar[u];
      for (int u = 0; u < t; ++u) C(1 + t, 2 + u) += -hbar[t] * hb[(lo + u) - j + L];
      C(1 + t, VX) = hbar[t];
    }
    // 1 + nw: zero output (coefficients 0)
  } else {   // kAScalN
    const int lo = max(1, j - L), np = j - lo;
    const double *tb = a.tband + ((size_t)r * a.maxit + (j - 1)) * (L + 1);
    const double alpha = tb[L];
    const double ia = 1.0 / alpha;
    const double s = tot[0][1];
    double cbar[kAdjNV];
    for (int t = np - 1; t >= 0; --t) {
      double v = (tot[0][2 + t] - s * tot[1][2 + t]) * ia;
      for (int u = t + 1; u < np; ++u) v += cbar[u] * tot[2 + t][2 + u];
      cbar[t] = -v;
    }
    C(0, 0) = ia;
    C(0, 1) = -s * ia;
    for (int t = 0; t < np; ++t) C(0, 2 + t) = cbar[t];
    for (int t = 0; t < np; ++t) {
      const double cc = tb[(lo + t) - j + L];
      C(1 + t, 0) = -cc * ia;
      C(1 + t, 1) = cc * s * ia + cbar[t] * alpha;
      for (int u = t + 1; u < np; ++u) C(1 + t, 2 + u) += -cc * cbar[u] + cbar[t] * tb[(lo + u) - j + L];
      C(1 + t, 2 + t) += cbar[t] * cc;
    }
  }
}

// Adjoint of the small least-squares problem of every right-hand side (one
// CTA each): with M = S A Z = Q R and e = s_b - M y,
//   v = R^{-T} ybar, u = R^{-1} v, sbar = Q v, Mbar = e u^T - sbar y^T.
__global__ void __launch_bounds__(kThreads) als_adj_kernel(int R, int s, int maxit, const int *kr, const double *Q,
                                                          const double *Rinv, const double *y, const double *e,
                                                          const double *ybar, double *sbar, double *Mbar) {
  extern __shared__ double sm[];
  double *v = sm, *u = sm + maxit;
  const int r = blockIdx.x, k = kr[r];
  const double *Qr = Q + (size_t)r * s * maxit, *Ri = Rinv + (size_t)r * maxit * maxit;
  const double *yr = y + (size_t)r * maxit, *er = e + (size_t)r * s, *yb = ybar + (size_t)r * maxit;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {          // v_i = sum_{j <= i} Rinv[j][i] ybar_j
    double a = 0.0;
    for (int jj = 0; jj <= i; ++jj) a += Ri[(size_t)jj * maxit + i] * yb[jj];
    v[i] = a;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {          // u_i = sum_{j >= i} Rinv[i][j] v_j
    double a = 0.0;
    for (int jj = i; jj < k; ++jj) a += Ri[(size_t)i * maxit + jj] * v[jj];
    u[i] = a;
  }
  __syncthreads();
  double *sb = sbar + (size_t)r * s, *Mb = Mbar + (size_t)r * maxit * s;
  for (int row = threadIdx.x; row < s; row += blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < k; ++i) a += Qr[(size_t)row * maxit + i] * v[i];
    sb[row] = a;
    for (int i = 0; i < k; ++i) Mb[(size_t)i * s + row] = er[row] * u[i] - a * yr[i];
  }
}

// out[c][r] = (1/sqrt(zeta)) sum_q sign_q V_r[row_q] over the zeta draws of
// column c (S^T applied to one s-vector per RHS).  V_r = V + r * vstride.
template <typename XT>
__global__ void ast_kernel(int R, int ld, int64_t len, int zeta, double isz, const uint32_t *rows,
                           const uint32_t *ents, const double *V, int64_t vstride, const int *kr, int jstep, XT *out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t c = t / ld;
  const int r = (int)(t % ld);
  if (c >= len) return;
  double a = 0.0;
  if (r < R && jstep <= kr[r]) {
    const double *vr = V + (size_t)r * vstride;
    for (int q = 0; q < zeta; ++q) {
      const uint32_t row = rows[c * zeta + q], ent = ents[c * zeta + q];
      a += flip_sign(vr[row], ent);
    }
  }
  out[(size_t)c * ld + r] = (XT)(a * isz);
}

// dst[r * len + i] = src[i * ld + r] (column-major FP64 from interleaved XT),
// optionally adding the FP64 interleaved add[i * ld + r].
template <typename XT>
__global__ void adeinterleave_kernel(const XT *src, int64_t len, int R, int ld, double *dst) {
  __shared__ double t[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int j = ty; j < 32; j += 8) {
    const int64_t i = i0 + j;
    const int r = r0 + tx;
    t[j][tx] = (i < len && r < R) ? (double)src[(size_t)i * ld + r] : 0.0;
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int r = r0 + j;
    const int64_t i = i0 + tx;
    if (i < len && r < R) dst[(size_t)r * len + i] = t[tx][j];
  }
}

// dbar[i] = sum_r acc[i][r], right-hand sides added in order.
__global__ void adsum_kernel(const double *acc, int64_t n, int R, int ld, double *dbar) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0;
  for (int r = 0; r < R; ++r) a += acc[(size_t)i * ld + r];
  dbar[i] = a;
}

}  // namespace sfl
