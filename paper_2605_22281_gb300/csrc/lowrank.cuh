// Rank-r truncation of a basis vector by the randomized SVD (the -RND flexible
// operator of Section 4.1; the truncation operator itself is defined in
// Section 1.2).
//
// The new basis vector p~_k (length n = N1 * N2, row-major image C, N1 x N2)
// is replaced by z~_k = vec(C_r), where C_r is the rank-r approximation the
// randomized SVD of Halko, Martinsson & Tropp (SIAM Review 2011) returns for the
// test matrix Omega (N2 x l, l = r + oversampling): their Algorithm 4.4 (range
// finder with q steps of subspace iteration) followed by Algorithm 5.1 (direct
// SVD of the projected matrix), truncated to rank r:
//   Y = C Omega, Q = orth(Y); q times: Q~ = orth(C^T Q), Q = orth(C Q~);
//   B^T = C^T Q (N2 x l); eigenvectors W of B B^T = (B^T)^T B^T (l x l);
//   U = Q W_r, V = B^T W_r;  C_r = U V^T   (= Q W_r W_r^T Q^T C).
// C_r is positively homogeneous in C, so it is applied to the unnormalised
// p~_k and keeps the scale sig_p(k).
//
// Arithmetic is FP32 by default (a regularizing truncation; the FP64 oracle
// states the error), or FP64 on request (for verification), with the l x l
// problems in one CTA:
//  - orth() is shifted Cholesky QR followed by plain Cholesky QR twice
//    (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput.
//    2020): G = Y^T Y (+ shift), G = R^T R, Q = Y R^{-1};
//  - the eigenvectors come from cyclic two-sided Jacobi with the round-robin
//    pairing, rotations as in Golub & Van Loan, Algorithm 8.5.1 (sym.schur2).
// Every sum has a fixed order (split-K partials and Gram partials reduced in
// order), so results are bitwise reproducible.
#pragma once

#include "common.cuh"

namespace sfl {

constexpr int kLrTile = 32;       // rows of a product tile
constexpr int kLrK = 64;          // depth of one split-K chunk
constexpr int kLrSweeps = 10;     // most Jacobi sweeps
constexpr size_t kLrOrthSmem = 200 * 1024;   // largest M x l block the one-CTA orthonormalization holds

// Per compute type (FP32 default, FP64 for verification): largest r +
// oversampling, rows per CTA of the Gram partials, unit roundoff, and the
// Jacobi rotation threshold (a pair is rotated while |a_pq| exceeds it times
// the largest diagonal entry, about ten unit roundoffs).
template <typename RT> struct LrLim;
template <> struct LrLim<float> {
  static constexpr int L = 64, GR = 64;
  static constexpr float u = 5.9604645e-8f, rot_tol = 6e-7f;
};
template <> struct LrLim<double> {
  static constexpr int L = 48, GR = 32;
  static constexpr double u = 1.1102230246251565e-16, rot_tol = 1e-15;
};

template <typename RT>
struct LrParams {
  SolveState *st;
  int N1, N2, l, r, q;
  const RT *Omega;                // N2 x l (row-major)
  RT *Y, *Qm, *Qt, *Bt;           // N1 x l, N1 x l, N2 x l, N2 x l
  RT *U, *V;                      // N1 x r, N2 x r
  RT *part;                       // split-K partials [KS][max(N1,N2)][l]
  RT *gpart;                      // Gram partials [CTAs][l * l]
  RT *small;                      // l x l factors (R^{-1} or W_r) of the latest small step
  int *flag;                      // nonzero: a Cholesky pivot failed (the step keeps tau = identity)
  int *ticket;                    // arrival counter of the last-CTA steps (zero between launches)
};

__device__ __forceinline__ bool lr_running(const SolveState *st) { return __ldcg(&st->stop) == 0; }

// out_part[ks][i][c] = sum_{k in chunk ks} A(i, k) X[k][c] with A = C (TRANS
// false, M = N1, K = N2) or A = C^T (TRANS true, M = N2, K = N1).  C is read
// from the solver's vector (type XT) at column `col` of Z.  Tiles: 32 rows x l
// columns, K in chunks of 64 staged in shared memory; thread (row, c0) sums
// columns c0, c0 + 8, ...
template <typename RT, typename XT, bool TRANS>
__global__ void __launch_bounds__(kThreads) lr_mul_kernel(LrParams<RT> p, const XT *Z, int64_t zstride, const RT *X) {
  __shared__ RT As[kLrTile][kLrK + 1];
  __shared__ RT Xs[kLrK][LrLim<RT>::L];
  if (!lr_running(p.st) || __ldcg(p.flag)) return;
  const int k = __ldcg(&p.st->k) + 1;
  const XT *C = Z + (size_t)(k - 1) * zstride;   // p~_k (the z update stored it unmodified)
  const int M = TRANS ? p.N2 : p.N1, K = TRANS ? p.N1 : p.N2, L = p.l;
  const int i0 = blockIdx.x * kLrTile, k0 = blockIdx.y * kLrK;
  const int tid = threadIdx.x;
  for (int t = tid; t < kLrTile * kLrK; t += kThreads) {
    int ii, kk;
    if (TRANS) { kk = t / kLrTile; ii = t % kLrTile; }   // C[k][i]: consecutive i are contiguous
    else { ii = t / kLrK; kk = t % kLrK; }              // C[i][k]: consecutive k are contiguous
    const int i = i0 + ii, kx = k0 + kk;
    RT v = RT(0.);
    if (i < M && kx < K) v = (RT)(TRANS ? C[(size_t)kx * p.N2 + i] : C[(size_t)i * p.N2 + kx]);
    As[ii][kk] = v;
  }
  for (int t = tid; t < kLrK * L; t += kThreads) {
    const int kk = t / L, c = t % L, kx = k0 + kk;
    Xs[kk][c] = kx < K ? X[(size_t)kx * L + c] : RT(0.);
  }
  __syncthreads();
  const int row = tid >> 3, c0 = tid & 7;
  RT acc[LrLim<RT>::L / 8];
#pragma unroll
  for (int j = 0; j < LrLim<RT>::L / 8; ++j) acc[j] = RT(0.);
  for (int kk = 0; kk < kLrK; ++kk) {
    const RT a = As[row][kk];
#pragma unroll
    for (int j = 0; j < LrLim<RT>::L / 8; ++j) {
      const int c = c0 + 8 * j;
      if (c < L) acc[j] = fma(a, Xs[kk][c], acc[j]);
    }
  }
  const int i = i0 + row;
  if (i < M) {
    RT *out = p.part + ((size_t)blockIdx.y * M + i) * L;
#pragma unroll
    for (int j = 0; j < LrLim<RT>::L / 8; ++j) {
      const int c = c0 + 8 * j;
      if (c < L) out[c] = acc[j];
    }
  }
}

// Gram partials of this CTA's rows of X (LrLim<RT>::GR x l staged in Xs):
// gp[blockIdx.x][a * l + c] for a <= c, rows added in order.
template <typename RT>
__device__ __forceinline__ void lr_gram_partial(const LrParams<RT> &p, const RT (*Xs)[LrLim<RT>::L], int nr) {
  const int L = p.l;
  RT *out = p.gpart + (size_t)blockIdx.x * L * L;
  for (int t = threadIdx.x; t < L * L; t += kThreads) {
    const int a = t / L, c = t % L;
    if (a > c) continue;
    RT s = RT(0.);
    for (int i = 0; i < nr; ++i) s = fma(Xs[i][a], Xs[i][c], s);
    out[t] = s;
  }
}

// Last-arriving CTA of a launch (ticket counter, reset by that CTA): true in
// every thread of that CTA only.  The CTA's global writes are fenced first.
template <typename RT>
__device__ __forceinline__ bool lr_last_cta(const LrParams<RT> &p, int *s_last) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_last = atomicAdd(p.ticket, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!*s_last) return false;
  __threadfence();
  if (threadIdx.x == 0) *p.ticket = 0;
  return true;
}

// G = sum of the nb Gram partials (in order), both triangles.
template <typename RT>
__device__ __forceinline__ void lr_load_gram(const LrParams<RT> &p, int nb, RT (*G)[LrLim<RT>::L + 1]) {
  const int L = p.l;
  for (int t = threadIdx.x; t < L * L; t += kThreads) {
    const int a = t / L, c = t % L;
    if (a > c) continue;
    RT s = RT(0.);
    for (int b = 0; b < nb; ++b) s += __ldcg(p.gpart + (size_t)b * L * L + t);
    G[a][c] = s;
    G[c][a] = s;
  }
  __syncthreads();
}

// Cholesky G + shift I = R^T R (upper R) and R^{-1} into p.small (l x l,
// row-major, zero below the diagonal), by warp 0 of the CTA (lanes split the
// columns; __syncwarp between the dependent steps).  A pivot that is not
// positive sets *p.flag (then the step keeps tau = identity).  The CTA's
// other warps return at once; G is in shared memory, Ri is scratch of the
// same shape.
template <typename RT>
static __device__ void lr_cholesky_inverse(const LrParams<RT> &p, RT (*G)[LrLim<RT>::L + 1],
                                           RT (*Ri)[LrLim<RT>::L + 1], RT shift_rel) {
  const int L = p.l, lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  if (shift_rel > RT(0)) {
    RT tr = RT(0);
    for (int a = lane; a < L; a += 32) tr += G[a][a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    for (int a = lane; a < L; a += 32) G[a][a] += shift_rel * tr;
    __syncwarp();
  }
  // right-looking Cholesky: G's upper triangle becomes R
  for (int j = 0; j < L; ++j) {
    const RT d = G[j][j];
    if (!(d > RT(0))) {
      if (lane == 0) *p.flag = 1;
      return;
    }
    const RT rd = rsqrt(d);
    __syncwarp();
    for (int c = j + lane; c < L; c += 32) G[j][c] *= rd;
    __syncwarp();
    for (int c = j + 1 + lane; c < L; c += 32) {
      const RT gjc = G[j][c];
      for (int a = j + 1; a <= c; ++a) G[a][c] -= G[j][a] * gjc;
    }
    __syncwarp();
  }
  // R^{-1}, rows from the bottom: Ri[a][c] = -(sum_{a < t <= c} R[a][t] Ri[t][c]) / R[a][a]
  for (int a = L - 1; a >= 0; --a) {
    const RT inv = RT(1) / G[a][a];
    for (int c = lane; c < L; c += 32) {
      RT v = RT(0);
      if (c == a) {
        v = inv;
      } else if (c > a) {
        RT acc = RT(0);
        for (int t = a + 1; t <= c; ++t) acc = fma(G[a][t], Ri[t][c], acc);
        v = -acc * inv;
      }
      Ri[a][c] = v;
    }
    __syncwarp();
  }
  for (int t = lane; t < L * L; t += 32) p.small[t] = Ri[t / L][t % L];
}

// Orthonormal basis of the range of X (M x l) by one CTA, when X fits in
// shared memory: X = the sum of the KS split-K partials of a product, held
// column-major; classical Gram-Schmidt applied twice, column by column (warps
// take the dots of the earlier columns, threads the updates, fixed-order
// block sums); a column whose norm falls below 1e-5 (FP32) or 1e-12 (FP64)
// of its norm before the passes is set to zero (rank deficient: it adds
// nothing to the projector).  Q (M x l, row-major) is written to out.
template <typename RT>
static __global__ void __launch_bounds__(kThreads) lr_orth_cta_kernel(LrParams<RT> p, int M, int KS, RT *out) {
  extern __shared__ __align__(16) unsigned char lr_smem[];
  RT *X = reinterpret_cast<RT *>(lr_smem);      // [l][M]
  __shared__ RT d[LrLim<RT>::L];
  __shared__ RT wpart[kWarps];
  __shared__ RT s_norm0, s_norm;
  if (!lr_running(p.st) || __ldcg(p.flag)) return;
  const int L = p.l, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int t = tid; t < M * L; t += kThreads) {
    const int i = t / L, c = t % L;
    RT v = RT(0);
    for (int ks = 0; ks < KS; ++ks) v += p.part[(size_t)ks * M * L + t];
    X[(size_t)c * M + i] = v;
  }
  __syncthreads();
  auto block_sum = [&](RT v) -> RT {   // fixed order: lanes by butterfly, warps in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) wpart[warp] = v;
    __syncthreads();
    RT a = RT(0);
    for (int w = 0; w < kWarps; ++w) a += wpart[w];
    __syncthreads();
    return a;
  };
  const RT drop = sizeof(RT) == sizeof(float) ? RT(1e-5) : RT(1e-12);
  for (int j = 0; j < L; ++j) {
    RT *v = X + (size_t)j * M;
    RT a = RT(0);
    for (int i = tid; i < M; i += kThreads) a += v[i] * v[i];
    a = block_sum(a);
    if (tid == 0) s_norm0 = sqrt(a);
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      for (int t = warp; t < j; t += kWarps) {   // d_t = <q_t, v>
        const RT *q = X + (size_t)t * M;
        RT s = RT(0);
        for (int i = lane; i < M; i += 32) s += q[i] * v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) d[t] = s;
      }
      __syncthreads();
      for (int i = tid; i < M; i += kThreads) {   // v -= Q d
        RT s = RT(0);
        for (int t = 0; t < j; ++t) s += X[(size_t)t * M + i] * d[t];
        v[i] -= s;
      }
      __syncthreads();
    }
    a = RT(0);
    for (int i = tid; i < M; i += kThreads) a += v[i] * v[i];
    a = block_sum(a);
    if (tid == 0) s_norm = sqrt(a);
    __syncthreads();
    const RT nv = s_norm, n0 = s_norm0;
    const RT sc = (nv > drop * n0 && nv > RT(0)) ? RT(1) / nv : RT(0);
    for (int i = tid; i < M; i += kThreads) v[i] *= sc;
    __syncthreads();
  }
  for (int t = tid; t < M * L; t += kThreads) {
    const int i = t / L, c = t % L;
    out[t] = X[(size_t)c * M + i];
  }
}

// One Cholesky-QR pass over X (M x l), rows in blocks of LrLim<RT>::GR per CTA:
//   mode 0: X = the sum of the KS split-K partials of a product (written to out);
//   mode 1: out = in * p.small (the previous pass's R^{-1});
// then the Gram partials of out, and in the last CTA the Cholesky factor of
// their sum (+ shift) and its inverse into p.small.
template <typename RT>
static __global__ void __launch_bounds__(kThreads) lr_orth_kernel(LrParams<RT> p, int mode, const RT *in, RT *out, int M,
                                                           int KS, RT shift_rel) {
  constexpr int kL = LrLim<RT>::L, kGR = LrLim<RT>::GR;
  constexpr int kXs = kGR * kL > kL * (kL + 1) ? kGR * kL : kL * (kL + 1);
  __shared__ RT XR[kXs];                   // this CTA's rows (later, in the last CTA: R^{-1} scratch)
  __shared__ RT SG[kL * (kL + 1)];         // S (this pass's input factor), later G (last CTA)
  __shared__ int s_last;
  RT *S = SG;
  auto Xs = reinterpret_cast<RT (*)[kL]>(XR);
  auto G = reinterpret_cast<RT (*)[kL + 1]>(SG);
  auto Ri = reinterpret_cast<RT (*)[kL + 1]>(XR);
  if (!lr_running(p.st) || __ldcg(p.flag)) return;
  const int L = p.l, r0 = blockIdx.x * LrLim<RT>::GR, tid = threadIdx.x;
  const int nr = min(LrLim<RT>::GR, M - r0);
  if (mode == 1)
    for (int t = tid; t < L * L; t += kThreads) S[t] = __ldcg(p.small + t);
  __syncthreads();
  for (int t = tid; t < LrLim<RT>::GR * L; t += kThreads) {
    const int i = t / L, c = t % L;
    RT v = RT(0.);
    if (i < nr) {
      const size_t idx = (size_t)(r0 + i) * L + c;
      if (mode == 0) {
        for (int ks = 0; ks < KS; ++ks) v += p.part[(size_t)ks * M * L + idx];
      } else {
        const RT *x = in + (size_t)(r0 + i) * L;
        for (int j = 0; j < L; ++j) v = fma(x[j], S[j * L + c], v);
      }
      out[idx] = v;
    }
    Xs[i][c] = v;
  }
  __syncthreads();
  lr_gram_partial(p, Xs, nr);
  if (!lr_last_cta(p, &s_last)) return;
  lr_load_gram(p, gridDim.x, G);
  lr_cholesky_inverse(p, G, Ri, shift_rel);
}

// out[i][0..ncol) = in[i][0..l) * p.small (l x ncol).
template <typename RT>
__device__ __forceinline__ void lr_apply_rows(const LrParams<RT> &p, const RT *S, const RT *in, int64_t M, int ncol,
                                              RT *out, int64_t t0, int64_t stride) {
  const int L = p.l;
  for (int64_t t = t0; t < M * ncol; t += stride) {
    const int64_t i = t / ncol;
    const int c = (int)(t % ncol);
    const RT *x = in + i * L;
    RT a = RT(0.);
    for (int j = 0; j < L; ++j) a = fma(x[j], S[j * ncol + c], a);
    out[t] = a;
  }
}

template <typename RT>
static __global__ void __launch_bounds__(kThreads) lr_apply_kernel(LrParams<RT> p, const RT *in, int M, RT *out) {
  __shared__ RT S[LrLim<RT>::L * LrLim<RT>::L];
  if (!lr_running(p.st) || __ldcg(p.flag)) return;
  for (int t = threadIdx.x; t < p.l * p.l; t += kThreads) S[t] = __ldcg(p.small + t);
  __syncthreads();
  lr_apply_rows(p, S, in, M, p.l, out, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// B^T = the sum of the KS split-K partials of C^T Q (N2 x l, written to p.Bt),
// its Gram partials, and in the last CTA the eigenvectors of B B^T = (B^T)^T B^T
// by cyclic Jacobi; the r leading ones (by decreasing eigenvalue) go to p.small
// (l x r).
template <typename RT>
static __global__ void __launch_bounds__(kThreads) lr_gram_eig_kernel(LrParams<RT> p, int KS) {
  __shared__ RT XV[LrLim<RT>::L * (LrLim<RT>::L + 1)];   // the CTA's rows of B^T, later the eigenvectors (last CTA)
  __shared__ RT A[LrLim<RT>::L][LrLim<RT>::L + 1];
  auto Xs = reinterpret_cast<RT (*)[LrLim<RT>::L]>(XV);
  auto Vm = reinterpret_cast<RT (*)[LrLim<RT>::L + 1]>(XV);
  __shared__ RT cs[LrLim<RT>::L / 2][2];
  __shared__ int pr[LrLim<RT>::L / 2][2];
  __shared__ int order[LrLim<RT>::L];
  __shared__ int s_last, s_go;
  if (!lr_running(p.st) || __ldcg(p.flag)) return;
  const int L = p.l, M = p.N2, r0 = blockIdx.x * LrLim<RT>::GR, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nr = min(LrLim<RT>::GR, M - r0);
  for (int t = tid; t < LrLim<RT>::GR * L; t += kThreads) {
    const int i = t / L, c = t % L;
    RT v = RT(0.);
    if (i < nr) {
      const size_t idx = (size_t)(r0 + i) * L + c;
      for (int ks = 0; ks < KS; ++ks) v += p.part[(size_t)ks * M * L + idx];
      p.Bt[idx] = v;
    }
    Xs[i][c] = v;
  }
  __syncthreads();
  lr_gram_partial(p, Xs, nr);
  if (!lr_last_cta(p, &s_last)) return;
  lr_load_gram(p, gridDim.x, A);
  const int n = L + (L & 1);            // even order; a padded index is a zero row and column
  for (int t = tid; t < LrLim<RT>::L * LrLim<RT>::L; t += kThreads) {
    const int a = t / LrLim<RT>::L, c = t % LrLim<RT>::L;
    Vm[a][c] = a == c ? RT(1.) : RT(0.);
    if (a >= L || c >= L) A[a][c] = RT(0.);
  }
  __syncthreads();
  const int np = n / 2;
  // cyclic Jacobi, round-robin pairs (index 0 fixed, the others rotate); a
  // pair is rotated when |a_pq| > tol max_i |a_ii| (rounding-level entries are
  // left: only the leading eigenvectors are used); a sweep that rotates
  // nothing ends the iteration, and at most kLrSweeps sweeps run (the
  // convergence is quadratic)
  __shared__ RT s_amax;
  if (tid == 0) {
    RT mx = RT(0);
    for (int a = 0; a < L; ++a) mx = fmax(mx, fabs(A[a][a]));
    s_amax = mx;
  }
  __syncthreads();
  const RT thr = LrLim<RT>::rot_tol * s_amax;
  for (int sweep = 0; sweep < kLrSweeps; ++sweep) {
    if (tid == 0) s_go = 0;
    __syncthreads();
    for (int round = 0; round < n - 1; ++round) {
      if (tid < np) {
        const int u = tid, v = n - 1 - tid;
        int a = u == 0 ? 0 : 1 + (u - 1 + round) % (n - 1);
        int b = 1 + (v - 1 + round) % (n - 1);
        if (a > b) { const int t = a; a = b; b = t; }
        RT c = RT(1), sn = RT(0);
        const RT apq = A[a][b];
        if (b < L && fabs(apq) > thr) {
          const RT tau = (A[b][b] - A[a][a]) / (RT(2) * apq);
          const RT t = fabs(tau) > RT(1e15) ? RT(0.5) / tau
                                            : copysign(RT(1), tau) / (fabs(tau) + sqrt(fma(tau, tau, RT(1))));
          c = rsqrt(fma(t, t, RT(1)));
          sn = t * c;
          s_go = 1;
        }
        pr[tid][0] = a; pr[tid][1] = b;
        cs[tid][0] = c; cs[tid][1] = sn;
      }
      __syncthreads();
      // A <- J^T A J in one phase: the thread of block (u, v) (rows of pair u,
      // columns of pair v) updates its four entries; V <- V J alongside
      for (int t = tid; t < np * np; t += kThreads) {
        const int u = t / np, v = t % np;
        const int ra = pr[u][0], rb = pr[u][1], ca = pr[v][0], cb = pr[v][1];
        const RT cu = cs[u][0], su = cs[u][1], cv = cs[v][0], sv = cs[v][1];
        const RT b00 = A[ra][ca], b01 = A[ra][cb], b10 = A[rb][ca], b11 = A[rb][cb];
        const RT t00 = cu * b00 - su * b10, t01 = cu * b01 - su * b11;   // J_u^T B
        const RT t10 = su * b00 + cu * b10, t11 = su * b01 + cu * b11;
        A[ra][ca] = t00 * cv - t01 * sv;                                    // (J_u^T B) J_v
        A[ra][cb] = t00 * sv + t01 * cv;
        A[rb][ca] = t10 * cv - t11 * sv;
        A[rb][cb] = t10 * sv + t11 * cv;
      }
      for (int t = tid; t < n * np; t += kThreads) {
        const int i = t / np, v = t % np;
        const int a = pr[v][0], b = pr[v][1];
        const RT c = cs[v][0], sn = cs[v][1];
        const RT x = Vm[i][a], y = Vm[i][b];
        Vm[i][a] = c * x - sn * y;
        Vm[i][b] = sn * x + c * y;
      }
      __syncthreads();
    }
    if (!s_go) break;
  }
  for (int a = tid; a < L; a += kThreads) {   // decreasing eigenvalue, ties by index
    int rank = 0;
    for (int c = 0; c < L; ++c) rank += (A[c][c] > A[a][a]) || (A[c][c] == A[a][a] && c < a);
    order[rank] = a;
  }
  __syncthreads();
  for (int t = tid; t < L * p.r; t += kThreads) {
    const int a = t / p.r, j = t % p.r;
    p.small[t] = Vm[a][order[j]];
  }
}

// U = Q W_r (N1 x r) and V = B^T W_r (N2 x r) in one launch.
template <typename RT>
static __global__ void __launch_bounds__(kThreads) lr_uv_kernel(LrParams<RT> p) {
  __shared__ RT S[LrLim<RT>::L * LrLim<RT>::L];
  if (!lr_running(p.st) || __ldcg(p.flag)) return;
  for (int t = threadIdx.x; t < p.l * p.r; t += kThreads) S[t] = __ldcg(p.small + t);
  __syncthreads();
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  lr_apply_rows(p, S, p.Qm, p.N1, p.r, p.U, t0, st);
  lr_apply_rows(p, S, p.Bt, p.N2, p.r, p.V, t0, st);
}

// z~_k = vec(U V^T): Z[:, k-1][i * N2 + j] = sum_a U[i][a] V[j][a] (32 x 32
// output tile per CTA).  If a Cholesky pivot failed, z~_k stays p~_k.
template <typename RT, typename XT>
__global__ void __launch_bounds__(kThreads) lr_outer_kernel(LrParams<RT> p, XT *Z, int64_t zstride) {
  __shared__ RT Us[32][LrLim<RT>::L + 1];
  __shared__ RT Vs[32][LrLim<RT>::L + 1];
  if (!lr_running(p.st) || __ldcg(p.flag)) return;
  const int k = __ldcg(&p.st->k) + 1;
  XT *out = Z + (size_t)(k - 1) * zstride;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32, R = p.r;
  for (int t = threadIdx.x; t < 32 * R; t += kThreads) {
    const int a = t / R, c = t % R;
    Us[a][c] = (i0 + a < p.N1) ? p.U[(size_t)(i0 + a) * R + c] : RT(0.);
    Vs[a][c] = (j0 + a < p.N2) ? p.V[(size_t)(j0 + a) * R + c] : RT(0.);
  }
  __syncthreads();
  const int tj = threadIdx.x & 31, ti = threadIdx.x >> 5;   // 4 rows per thread
  for (int ii = ti; ii < 32; ii += kWarps) {
    const int i = i0 + ii, j = j0 + tj;
    if (i >= p.N1 || j >= p.N2) continue;
    RT a = RT(0.);
    for (int c = 0; c < R; ++c) a = fma(Us[ii][c], Vs[tj][c], a);
    out[(size_t)i * p.N2 + j] = (XT)a;
  }
}

static __global__ void lr_clear_flag_kernel(int *flag) { *flag = 0; }

// FP32 copy of the caller's FP64 test matrix.
template <typename RT>
static __global__ void lr_omega_kernel(const double *src, RT *dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (RT)src[i];
}

}  // namespace sfl
