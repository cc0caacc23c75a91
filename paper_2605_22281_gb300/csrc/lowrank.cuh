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

// Per compute type (FP32 default, FP64 for verification): largest r +
// oversampling, rows per CTA of the Gram partials, unit roundoff, and the
// Jacobi stopping threshold on (off-diagonal / diagonal) squared norms.
template <typename RT> struct LrLim;
template <> struct LrLim<float> {
  static constexpr int L = 64, GR = 64;
  static constexpr float u = 5.9604645e-8f, jacobi_tol = 1e-12f;
};
template <> struct LrLim<double> {
  static constexpr int L = 48, GR = 32;
  static constexpr double u = 1.1102230246251565e-16, jacobi_tol = 1e-30;
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
// row-major, zero below the diagonal).  All threads of one CTA.  A pivot that
// is not positive sets *p.flag (then the step keeps tau = identity).
template <typename RT>
static __device__ void lr_cholesky_inverse(const LrParams<RT> &p, RT (*G)[LrLim<RT>::L + 1], RT shift_rel, RT *s_tr) {
  const int L = p.l, tid = threadIdx.x;
  if (shift_rel > RT(0.)) {
    if (tid == 0) {
      RT tr = RT(0.);
      for (int a = 0; a < L; ++a) tr += G[a][a];
      *s_tr = tr;
    }
    __syncthreads();
    for (int a = tid; a < L; a += kThreads) G[a][a] += shift_rel * *s_tr;
  }
  for (int j = 0; j < L; ++j) {
    __syncthreads();
    const RT d = G[j][j];
    if (!(d > RT(0.))) {
      if (tid == 0) *p.flag = 1;
      return;
    }
    const RT rd = rsqrt(d);
    __syncthreads();
    for (int c = j + tid; c < L; c += kThreads) G[j][c] *= rd;
    __syncthreads();
    const int w = L - j - 1;
    for (int t = tid; t < w * w; t += kThreads) {
      const int a = j + 1 + t / w, c = j + 1 + t % w;
      if (a <= c) G[a][c] -= G[j][a] * G[j][c];
    }
  }
  __syncthreads();
  // column c of R^{-1}: back substitution, one thread per column
  for (int c = tid; c < L; c += kThreads) {
    RT col[LrLim<RT>::L];
    col[c] = RT(1.) / G[c][c];
    for (int a = c - 1; a >= 0; --a) {
      RT s = RT(0.);
      for (int t = a + 1; t <= c; ++t) s = fma(G[a][t], col[t], s);
      col[a] = -s / G[a][a];
    }
    for (int a = 0; a < L; ++a) p.small[a * L + c] = a <= c ? col[a] : RT(0.);
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
  __shared__ RT Xs[LrLim<RT>::GR][LrLim<RT>::L];
  __shared__ RT SG[LrLim<RT>::L * (LrLim<RT>::L + 1)];   // S (this pass's input factor), later G (last CTA)
  __shared__ int s_last;
  __shared__ RT s_tr;
  RT *S = SG;
  auto G = reinterpret_cast<RT (*)[LrLim<RT>::L + 1]>(SG);
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
  lr_cholesky_inverse(p, G, shift_rel, &s_tr);
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
  __shared__ RT red[2][kWarps];
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
  for (int sweep = 0; sweep < kLrSweeps; ++sweep) {   // quadratic convergence: a few sweeps
    // stop when the off-diagonal mass is below the type's threshold times the diagonal's
    RT off = RT(0.), dg = RT(0.);
    for (int t = tid; t < L * L; t += kThreads) {
      const int a = t / L, c = t % L;
      const RT v = A[a][c] * A[a][c];
      if (a == c) dg += v; else off += v;
    }
    off = warp_sum(off);
    dg = warp_sum(dg);
    if (lane == 0) { red[0][warp] = off; red[1][warp] = dg; }
    __syncthreads();
    if (tid == 0) {
      RT o = RT(0.), d = RT(0.);
      for (int w = 0; w < kWarps; ++w) { o += red[0][w]; d += red[1][w]; }
      s_go = o > LrLim<RT>::jacobi_tol * d;
    }
    __syncthreads();
    if (!s_go) break;
    for (int round = 0; round < n - 1; ++round) {
      if (tid < np) {   // round-robin pairing: index 0 fixed, the others rotate
        const int u = tid, v = n - 1 - tid;
        int a = u == 0 ? 0 : 1 + (u - 1 + round) % (n - 1);
        int b = 1 + (v - 1 + round) % (n - 1);
        if (a > b) { const int t = a; a = b; b = t; }
        RT c = RT(1.), s = RT(0.);
        const RT apq = A[a][b];
        if (b < L && fabs(apq) > RT(1e-20) * sqrt(fabs(A[a][a] * A[b][b])) && apq != RT(0.)) {
          const RT tau = (A[b][b] - A[a][a]) / (RT(2.) * apq);
          const RT t = fabs(tau) > RT(1e15) ? RT(0.5) / tau
                                             : copysign(RT(1.), tau) / (fabs(tau) + sqrt(fma(tau, tau, RT(1.))));
          c = rsqrt(fma(t, t, RT(1.)));
          s = t * c;
        }
        pr[tid][0] = a; pr[tid][1] = b;
        cs[tid][0] = c; cs[tid][1] = s;
      }
      __syncthreads();
      for (int t = tid; t < np * n; t += kThreads) {   // rows: A <- J^T A
        const int k = t / n, j = t % n;
        const int a = pr[k][0], b = pr[k][1];
        const RT c = cs[k][0], s = cs[k][1];
        const RT x = A[a][j], y = A[b][j];
        A[a][j] = c * x - s * y;
        A[b][j] = s * x + c * y;
      }
      __syncthreads();
      for (int t = tid; t < np * n; t += kThreads) {   // columns: A <- A J, V <- V J
        const int k = t / n, i = t % n;
        const int a = pr[k][0], b = pr[k][1];
        const RT c = cs[k][0], s = cs[k][1];
        const RT x = A[i][a], y = A[i][b];
        A[i][a] = c * x - s * y;
        A[i][b] = s * x + c * y;
        const RT u = Vm[i][a], w = Vm[i][b];
        Vm[i][a] = c * u - s * w;
        Vm[i][b] = s * u + c * w;
      }
      __syncthreads();
    }
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
