/* sfl.h - C ABI of the GB300 sketched flexible Golub-Kahan solvers.
 *
 * Solves  min_x || A x - b ||_2  for a large sparse A (m x n, CSR) by
 *   sFLSQR  (Algorithm 1, eq. (sFLSQR) of Section 2.3)  and
 *   sFLSMR  (Algorithm 2, eq. (sFLSMR) of Section 2.5)
 * of "Randomized Flexible LSQR and LSMR with applications to inverse problems":
 * a flexible Golub-Kahan process with window-ell partial orthogonalization
 * (eq. (FGK)), a flexible right operator z_k = tau_k(p_k) (eq. (modbasis)),
 * an s-row sketch of every new basis vector (sparse-sign, Section 2.7, or an
 * explicit dense matrix such as a Gaussian one), a small
 * FP64 sketched least-squares solve per step, and the discrepancy-principle
 * stop of eq. (discrP) in Section 1.1.
 *
 * Conventions for every entry point:
 *  - All pointers to matrix and vector data are DEVICE pointers on the current
 *    CUDA device unless stated otherwise.  Index arrays are int32.  Dense
 *    vectors are contiguous.  Host pointers are marked "host".
 *  - Every function returns an sfl_status (SFL_OK == 0).  No function aborts,
 *    throws or exits; errors are reported by the return value and
 *    sfl_error_string() gives a static description.
 *  - The library never frees or writes caller memory except the declared
 *    outputs.  A plan owns its internal copies (padded CSR, transposed CSR,
 *    workspaces, CUDA graphs) until sfl_plan_destroy.
 *  - Work is enqueued on the given stream (0 = legacy default stream); calls on
 *    one plan must not overlap in time.
 */
#ifndef SFL_H
#define SFL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sfl_stream;   /* == cudaStream_t */

typedef enum {
  SFL_OK = 0,
  SFL_EINVAL = 1,        /* bad argument: null pointer, bad CSR, bad option */
  SFL_ENOMEM = 2,        /* device allocation failed (or exceeded the plan's cap) */
  SFL_ECUDA = 3,         /* a CUDA runtime call failed */
  SFL_ENONFINITE = 4,    /* NaN or Inf in the matrix values or in b */
  SFL_ETIMEOUT = 5,      /* host wait exceeded its wall-clock limit */
  SFL_EUNSUPPORTED = 6   /* valid request the library does not implement */
} sfl_status;

typedef enum { SFL_F64 = 0, SFL_F32 = 1, SFL_BF16 = 2 } sfl_dtype;

/* Outcome of a solve (sfl_info.status). */
typedef enum {
  SFL_STOP_RUNNING = 0,
  SFL_STOP_DISCREPANCY = 1,   /* relative sketched residual < eta*||e||/||b|| (eq. (discrP)) */
  SFL_STOP_MAXIT = 2,         /* maxit steps done */
  SFL_STOP_BREAKDOWN = 3      /* ||z|| or ||w|| or |R_kk| vanished; the last completed iterate is returned */
} sfl_stop;

typedef enum {
  SFL_PRECOND_IDENTITY = 0, SFL_PRECOND_DIAG = 1, SFL_PRECOND_REWEIGHT = 2,
  SFL_PRECOND_LOWRANK = 3     /* rank-r truncation by the randomized SVD (see sfl_opts.lowrank_*) */
} sfl_precond;
typedef enum { SFL_STOP_RULE_RESIDUAL = 0, SFL_STOP_RULE_NORMAL = 1 } sfl_stop_rule;
typedef enum { SFL_SKETCH_APPLY_AUTO = 0, SFL_SKETCH_APPLY_FUSED = 1, SFL_SKETCH_APPLY_KERNEL = 2 } sfl_sketch_apply_mode;
typedef enum { SFL_SKETCH_SPARSE_SIGN = 0, SFL_SKETCH_SRHT = 1, SFL_SKETCH_GAUSSIAN = 2 } sfl_sketch_kind;

/* A CSR matrix.  rowptr has rows+1 entries with rowptr[0] = 0, nondecreasing,
 * rowptr[rows] = nnz < 2^31; colidx[i] in [0, cols).  values has nnz entries of
 * `dtype`.  Column indices need not be sorted within a row. */
typedef struct {
  int64_t rows, cols, nnz;
  const int32_t *rowptr;
  const int32_t *colidx;
  const void *values;
  sfl_dtype dtype;
} sfl_csr;

typedef struct sfl_plan sfl_plan;

/* Plan options.  value_dtype is the precision the plan stores A (and its
 * transpose or B) in: SFL_F64, SFL_F32 or SFL_BF16 (round to nearest even).
 * lanes_per_row: lanes of a warp that share one row in the single-solve
 * products (4, 8, 16 or 32), or 0 to choose it from the average row length.
 * It fixes the summation order of every row, so results (not only speed)
 * depend on it; a plan's choice never changes.  max_device_bytes caps the
 * plan's own allocations (0 = no cap).  image_rows, image_cols: 0, or the
 * shape of the n-side as an image (n = image_rows * image_cols, column index
 * = row * image_cols + col).  When given, the plan stores the rows of A^T (or
 * B) in 16 x 16 pixel tiles, so that the rays one tile's rows gather stay in
 * the L1 cache; outputs still go to each row's own index, and every row's
 * sum is formed exactly as without tiles (bit-identical products).
 * slot_layout: 0 (default) stores every chunk slot of a row (lanes_per_row x
 * load-width entries) lane-interleaved, so the lanes of one gather read
 * neighbouring entries (faster single-solve products on ray-ordered rows);
 * 1 keeps each row in the caller's entry order (faster batched SpMMs, which
 * walk a row one entry at a time).  Results depend on it only through the
 * summation order.
 * index_bits: 0 (default) lets the single-solve products read 16-bit column
 * deltas (each stored entry's column minus the column of the entry before it
 * in its lane's walk, plus one 32-bit base per row) when every delta of the
 * operator fits in 16 bits, the row layout is lane-interleaved, 8 lanes run
 * a row and the deltas fit under max_device_bytes; otherwise, and with 32,
 * they read the 32-bit column indices.
 * The products are the same bit for bit; the 16-bit form streams 2 bytes of
 * index per entry instead of 4.  The plan keeps the 32-bit indices as well
 * (batched solves read them). */
typedef struct {
  sfl_dtype value_dtype;
  int32_t lanes_per_row;
  uint64_t max_device_bytes;
  int32_t image_rows, image_cols;
  int32_t slot_layout;
  int32_t index_bits;
} sfl_plan_opts;

/* Solve options (the Require lines of Algorithms 1 and 2).
 *  s, zeta, seed : sparse-sign sketch with s rows and zeta nonzeros +-1/sqrt(zeta)
 *                  per column (zeta = 1 is CountSketch), drawn from SplitMix64
 *                  (h = first output of the generator seeded with
 *                  seed ^ (column*2^32 + draw), row = floor(h*s/2^64), sign =
 *                  bit 0).  sFLSQR sketches m-vectors with `seed`; sFLSMR
 *                  sketches n-vectors with `seed` and keeps an m-side sketch
 *                  drawn from `seed + 1` for its discrepancy test.
 *                  Requires 1 <= zeta <= 16, maxit + 1 <= s <= 2048.
 *  window        : ell, the orthogonalization window, 0 <= ell <= 8, or any
 *                  negative value for full orthogonalization (every earlier
 *                  vector, eq. (FGK) with the band filled): the new z and w are
 *                  orthogonalized against the whole stored basis by block
 *                  classical Gram-Schmidt applied twice, and the plan keeps all
 *                  p_j and w_j (n*maxit + m*(maxit+1) more vector entries).
 *                  Not with orth_against_z = 1.
 *  maxit         : 1 <= maxit <= 1024.
 *  noise_norm    : ||e||_2 of the data noise; <= 0 disables the discrepancy stop.
 *  eta           : discrepancy safety factor (eta > 1, typically 1.01).
 *  precond       : tau_k.  IDENTITY; DIAG (z = diag(diag_w) p, diag_w FP64 of
 *                  length n); REWEIGHT (z = diag((x_{k-1}^2 + irw_eps)^(1/4)) p,
 *                  x_0 = 0), the iteratively reweighted operator of Section 1.2;
 *                  LOWRANK (single solves; needs a plan with image_rows x
 *                  image_cols = n): z = vec(C_r), C the new p reshaped to the
 *                  image, C_r the rank-r approximation of the randomized SVD
 *                  (Halko, Martinsson & Tropp 2011: range finder with
 *                  lowrank_power steps of subspace iteration, then the SVD of
 *                  the projected matrix, truncated to rank r), the -RND form of
 *                  the truncation operator of Section 1.2 used in Section 4.1.
 *                  Computed in FP32 (the small l x l problems in one CTA); if
 *                  a Cholesky factorization inside it fails, that step keeps
 *                  z = p.
 *  stop_rule     : sFLSMR only.  RESIDUAL tests ||S_m (b - A x_k)|| against
 *                  eta*||e|| relative to ||S_m b||; NORMAL tests the residual of
 *                  the sketched normal equations that sFLSMR minimises.
 *  vec_dtype     : precision of the basis vectors: SFL_F64 (requires an FP64
 *                  plan) or SFL_F32 (FP32 or BF16 plans).  Coefficients, the
 *                  small QR and y are FP64 in both.
 *  x_history     : optional (may be NULL), device, maxit*n FP64: x_k is written
 *                  to x_history + (k-1)*n after every step (costs one n x k
 *                  product per step; for verification).  Batched solves:
 *                  maxit*nrhs*n FP64, x_k of right-hand side r at
 *                  x_history + ((k-1)*nrhs + r)*n for every step k it completes
 *                  (rows of later steps are left as they were).
 *  relres_history: optional (may be NULL), device, maxit FP64: the stop-test
 *                  ratio of step k at index k-1.
 *  spmm_tile     : batched solves only: RHS per CTA column of the SpMMs (8, 16,
 *                  32 or 64), or 0 to let the plan time the candidates.  The
 *                  results are identical for every width.
 *  orth_against_z: 0 (default): the new z is orthogonalized against the unit
 *                  vectors p_j of the window, as eq. (FGK) states; 1: against
 *                  the stored z_j = tau_j(p_j) themselves, as the window loop of
 *                  Algorithms 1 and 2 is printed (z <- z - <z_j, z> z_j, in
 *                  ascending j).  The two coincide for the identity operator.
 *                  Single solves only (batched and fixed-k calls: 0).
 *  sketch_dense  : NULL for the sparse-sign sketch above, or a device FP64
 *                  s x len matrix (row-major, caller-owned, read by every
 *                  sketch application of the call) used as S itself, as
 *                  given: len = m for sFLSQR, n for sFLSMR (its S_n).  zeta and
 *                  seed are then ignored.  For dense sketches (Gaussian, the
 *                  identity when s = len) and tests; every application reads
 *                  all of S.  Single solves only.
 *  sketch_dense_stop: with sketch_dense in sFLSMR, the s x m matrix of its
 *                  m-side sketch S_m (discrepancy test); required there, NULL
 *                  otherwise. */
typedef struct {
  int32_t s;
  int32_t zeta;
  uint64_t seed;
  int32_t window;
  int32_t maxit;
  double noise_norm;
  double eta;
  int32_t precond;
  int32_t stop_rule;
  const double *diag_w;
  double irw_eps;
  int32_t vec_dtype;
  int32_t spmm_tile;
  double *x_history;
  double *relres_history;
  int32_t orth_against_z;
  const double *sketch_dense;
  const double *sketch_dense_stop;
  /* SFL_PRECOND_LOWRANK: rank r (>= 1), oversampling p (l = r + p <= 64, or
   * <= 48 with lowrank_fp64, and l <= min(image_rows, image_cols)),
   * subspace-iteration steps q (0..4), the Gaussian test matrix Omega (device
   * FP64, image_cols x l, row-major, caller-owned, read at the start of every
   * solve; the same Omega serves every step), and lowrank_fp64 = 1 to compute
   * the truncation in FP64 instead of FP32 (slower; for verification).
   * Ignored for the other operators. */
  int32_t lowrank_rank;
  int32_t lowrank_oversample;
  int32_t lowrank_power;
  const double *lowrank_omega;
  int32_t lowrank_fp64;
  /* How the sparse-sign sketch of each new basis vector is applied (single
   * solves; sfl_sketch_apply_mode): FUSED adds it in the epilogue of the
   * product that makes the vector, drawing S from the hash (no stored S, no
   * sketch launch); KERNEL runs a separate gather kernel over a row-major
   * table of S built once per seed; AUTO (0, the default) takes FUSED when
   * every sketched product averages at least 512 stored entries per output
   * row (or, on a matrix-free plan, an image of at least 512 x 512), where the
   * epilogue's per-output work is small beside the row, and KERNEL
   * otherwise.  Both give the same sketch up to rounding: FUSED adds the
   * terms exactly as 64-bit fixed-point integers per CTA (scale from the
   * CTA's output norm), KERNEL in FP64.  Explicit sketches and FLSQR always
   * take KERNEL (or no sketch). */
  int32_t sketch_apply;
  /* The sketch drawn from the seed (single solves; sfl_sketch_kind), beside
   * the sparse-sign default.  Both generated kinds are s x len matrices whose
   * entries every application regenerates from (seed, row, column), with
   * E[S^T S] = I; the two kinds Section 2.7 names next to CountSketch:
   *  SRHT: a subsampled randomized Hadamard transform,
   *    S[r, c] = (-1)^(popcount(rho(r) & c) + d_c) / sqrt(s), rho(0..s-1)
   *    distinct rows of the Sylvester-Hadamard matrix of order M = 2^b >= len
   *    (a seeded bijection of [0, M)), d_c hashed sign bits; needs s <= M;
   *  GAUSSIAN: N(0, 1/s) entries by Box-Muller from two hash outputs of the
   *    counter r * len + c (costly: a logarithm and a cosine per entry and
   *    application; meant for studies at small sizes).
   * zeta is ignored; the m-side stop sketch of sFLSMR uses seed + 1.  The
   * definitions are restated in the oracle (oracle/sketch.py), which the
   * tests compare against.  Not with sketch_dense or FLSQR; always applied by
   * the separate sketch kernel. */
  int32_t sketch_kind;
} sfl_opts;

/* Result of a solve.  Filled when the call returns (the call then waits for
 * its stream). */
typedef struct {
  int32_t iters;          /* k of the returned iterate x_k */
  int32_t status;         /* sfl_stop */
  double relres;          /* stop-test ratio at step iters (sketched, relative) */
  double tol;             /* eta * noise_norm / ||b|| (0 when disabled) */
} sfl_info;

/* Statistics of a plan (host struct). */
typedef struct {
  int64_t rows, cols, nnz_A, nnz_At;     /* nnz_At: nnz of A^T (CSC copy) or of B */
  int64_t padded_nnz_A, padded_nnz_At;   /* stored entries after row padding */
  int32_t lanes_A, lanes_At;             /* lanes per row of the SpMV kernels */
  int32_t value_dtype;
  int32_t unmatched;                     /* 1 if B was given */
  uint64_t device_bytes;                 /* bytes the plan holds */
  int32_t tiled_At;                      /* 1 if A^T / B rows are stored in pixel tiles */
  int32_t matrix_free;                   /* 1 for a sfl_plan_create_ct plan (nnz fields are 0) */
  int32_t index_bytes_A, index_bytes_At; /* bytes of column index the single-solve products read per entry (2 or 4) */
} sfl_plan_stats;

/* ---- plans ------------------------------------------------------------- */

/* Build a plan for A (m x n) and, optionally, an unmatched back-projector B
 * (n x m, CSR) used in place of A^T (Section 3.2).  When B is NULL the plan
 * builds a transposed copy of A (CSC of A stored as CSR of A^T) so that A^T
 * products need no atomics and are bitwise reproducible.  Validates the CSR
 * arrays on the device (SFL_EINVAL on a bad rowptr or column index,
 * SFL_ENONFINITE on NaN/Inf values); converts values to popts->value_dtype;
 * pads every row to a multiple of the vector-load width.  A and B may be freed
 * by the caller after this call returns.  popts may be NULL (FP64, no cap). */
int sfl_plan_create(sfl_plan **plan, const sfl_csr *A, const sfl_csr *B,
                    const sfl_plan_opts *popts, sfl_stream stream);
/* A matrix-free plan: the operators of the parallel-beam CT experiments
 * (Section 4.2) computed on the fly by the product kernels instead of read from
 * a stored matrix.  Geometry: image_n x image_n unit pixels centred at the
 * origin (column iy*image_n + ix); angles a*pi/n_angles; n_bins unit bins
 * centred at d - (n_bins-1)/2; ray (a, d) = {p : p.(cos, sin) = t_d} is row
 * a*n_bins + d of A (m = n_angles*n_bins, n = image_n^2).
 *   A z       Siddon's ray-driven walk with exact chord lengths;
 *   back = 0  A^T w, pixel-driven with the exact chords (the trapezoid
 *             footprint of a unit square), matched to A up to rounding;
 *   back = 1  the unmatched pixel-driven back-projector B w: each pixel centre
 *             split linearly between its two nearest bins (Section 3.2).
 * angles_cs: host, 2*n_angles values (cos, sin of each angle), or NULL to take
 * cos/sin of a*pi/n_angles from the C library.  popts: value_dtype SFL_F64
 * computes the geometry and sums in FP64 (FP64 solves); SFL_F32 (or
 * SFL_BF16) in FP32 (solves with FP32 vectors); image_rows/image_cols are
 * set to image_n; max_device_bytes as for stored plans; the other fields are
 * ignored.  Such a plan serves the single solves and sfl_plan_apply; batched
 * and fixed-k calls return SFL_EUNSUPPORTED.  No matrix is stored, so the
 * products are bound by arithmetic rather than by memory. */
typedef struct {
  int32_t image_n;
  int32_t n_angles;
  int32_t n_bins;
  int32_t back;
  const double *angles_cs;
} sfl_ct_geometry;
int sfl_plan_create_ct(sfl_plan **plan, const sfl_ct_geometry *geom, const sfl_plan_opts *popts, sfl_stream stream);
int sfl_plan_destroy(sfl_plan *plan);
int sfl_plan_get_stats(const sfl_plan *plan, sfl_plan_stats *stats /* host */);

/* y = A x (which = 0) or y = A^T x / B x (which = 1) with the plan's stored
 * operator and the same SpMV kernel the solvers use.  x and y are FP64
 * (lengths cols/rows of the chosen operator); the product is formed in the
 * plan's value precision with FP64 accumulation for FP64 plans and FP32 for
 * FP32/BF16 plans.  The first call per operator of a stored plan computes the
 * warps' row ranges balanced by row cost (a device allocation kept by the
 * plan, and a stream synchronisation); later calls reuse them. */
int sfl_plan_apply(sfl_plan *plan, int which, const double *x, double *y, sfl_stream stream);

/* ---- solvers ------------------------------------------------------------ */

/* Algorithm 1, sFLSQR.  b: device FP64, length m.  x: device FP64, length n,
 * receives x_k = Z_k y_k at the stop step.  info: host, may be NULL; when
 * given, the call waits for the stream and fills it.  The first call for a new
 * (s, zeta, window, maxit, precond, stop rule, vec_dtype, histories,
 * orth_against_z, explicit sketch pointers) combination allocates a workspace
 * and builds a CUDA graph that later calls reuse (the graph reads the
 * explicit sketches' contents at run time). */
int sflsqr_solve(sfl_plan *plan, const double *b, const sfl_opts *opts, double *x,
                 sfl_info *info, sfl_stream stream);

/* Algorithm 2, sFLSMR (same arguments).  The small problem is
 * min_y || s_{A^T b} - [S A^T W, S z] H_{k+1,k} y ||, formed from the sketched
 * columns of A^T W (or B W) and the banded H of eq. (FGK). */
int sflsmr_solve(sfl_plan *plan, const double *b, const sfl_opts *opts, double *x,
                 sfl_info *info, sfl_stream stream);

/* FLSQR, the unsketched flexible LSQR the paper compares against (Section 2.2,
 * eq. (FLSQR); timings in Section 4): full orthogonalization of both bases
 * (opts->window must be negative) and, at every step, the exact projected
 * problem min_y || beta e_1 - H_{k+1,k} y ||, which equals min || b - A Z_k y ||
 * while W_{k+1} is orthonormal.  Its relative residual is the stop ratio, tested
 * against eta*||e||/||b|| (eq. (discrP)).  s, zeta, seed, stop_rule and the
 * sketch pointers are ignored (SFL_EINVAL for an explicit sketch); maxit <=
 * 1024.  Same arguments and outputs as sflsqr_solve. */
int flsqr_solve(sfl_plan *plan, const double *b, const sfl_opts *opts, double *x, sfl_info *info,
                sfl_stream stream);
/* flsqr_solve with HOST b and x (as sflsqr_solve_host). */
int flsqr_solve_host(sfl_plan *plan, const double *b, const sfl_opts *opts, double *x, sfl_info *info,
                     sfl_stream stream);

/* Same solves with HOST FP64 b and x (b: m doubles, x: n doubles, ordinary or
 * pinned host memory).  The host-to-device copy of b and the device-to-host
 * copy of x are part of the call, which returns when x is written. */
int sflsqr_solve_host(sfl_plan *plan, const double *b_host, const sfl_opts *opts, double *x_host,
                      sfl_info *info, sfl_stream stream);
int sflsmr_solve_host(sfl_plan *plan, const double *b_host, const sfl_opts *opts, double *x_host,
                      sfl_info *info, sfl_stream stream);

/* Same as sflsqr_solve (method 0) / sflsmr_solve (method 1) / flsqr_solve (method 2) but driven by a
 * host loop over the same per-step kernels instead of the CUDA graph's
 * device-side WHILE node: one stream synchronisation per step.  Results are
 * bitwise identical to the graph driver; meant for verification. */
int sfl_solve_host_loop(sfl_plan *plan, int method, const double *b, const sfl_opts *opts, double *x,
                        sfl_info *info, sfl_stream stream);

/* Per-kernel device time of one solve.  Index: 0 initial sketches (S b, and
 * S A^T b for sFLSMR), 1 init ||b||, 2 init A^T w_1, 3 z orthogonalization +
 * tau, 4 fused A z_k SpMV, 5 w orthogonalization, 6 fused A^T w / B w SpMV,
 * 7 small least squares, 8 x = Z y, 9 per-step sketches, 10 block CGS2 of full
 * orthogonalization (five kernels per side, counted as one launch), 11 the
 * low-rank truncation (all its kernels of a step, counted as one launch).
 * ms: total milliseconds over the launches that did work; launches: their
 * number. */
#define SFL_NUM_KERNEL_CLASSES 12
typedef struct {
  double ms[SFL_NUM_KERNEL_CLASSES];
  int32_t launches[SFL_NUM_KERNEL_CLASSES];
} sfl_kernel_times;

/* The solve of sfl_solve_host_loop with a CUDA event pair recorded on `stream`
 * around every kernel launch; steps are enqueued in chunks without host
 * synchronisation inside a chunk.  Fills *times (host).  Same results as the
 * other drivers. */
int sfl_solve_profiled(sfl_plan *plan, int method, const double *b, const sfl_opts *opts, double *x,
                       sfl_info *info, sfl_kernel_times *times, sfl_stream stream);

/* ---- sketch ------------------------------------------------------------- */

/* Export the sparse-sign sketch (Section 2.7) the solvers draw: for columns
 * c = 0..ncols-1, rows[c*zeta + t] and signs[c*zeta + t] (+1/-1) of its t-th
 * distinct row in draw order.  rows, signs: device int32 arrays of ncols*zeta. */
int sfl_sketch_export(uint64_t seed, int32_t s, int32_t zeta, int64_t ncols,
                      int32_t *rows, int32_t *signs, sfl_stream stream);

/* sk = S v for the sparse-sign sketch (seed, s, zeta) of an FP64 vector v of
 * length len; sk: device FP64, length s.  Deterministic (fixed-order sums). */
int sfl_sketch_apply(uint64_t seed, int32_t s, int32_t zeta, const double *v, int64_t len,
                     double *sk, sfl_stream stream);

/* sk = S v exactly as sfl_sketch_apply computes it, but allocating nothing.
 * The paper has no counterpart: this exists for callers that may not call
 * cudaMalloc, such as code whose device memory is handed out up front by a
 * caching allocator that owns the pool, or latency-critical loops where an
 * allocation would synchronise the device.  The draws are regenerated in the
 * kernel and the reduction scratch is a fixed ~2.2 MB array inside the
 * library, reserved on every GPU that loads it until the process exits.
 * Limits: 1 <= zeta <= 16, zeta <= s <= 1024 (larger s returns SFL_EINVAL).
 * The first call on each device looks up the scratch address on that device;
 * make that first call before any stream capture.  All calls on a device share
 * the scratch, so calls that overlap in time on the GPU (different streams or
 * threads) race; serialise them.  Same results as sfl_sketch_apply up to the
 * order of summation (relative difference ~1e-16). */
int sfl_sketch_apply_noalloc(uint64_t seed, int32_t s, int32_t zeta, const double *v, int64_t len,
                             double *sk, sfl_stream stream);

/* ---- batched solves ------------------------------------------------------ */

/* sFLSQR (Algorithm 1) for nrhs independent right-hand sides through the
 * plan's operator, run together: every step does one SpMM with A and one with
 * A^T (or B) for all right-hand sides still running, and a right-hand side
 * stops on its own discrepancy test (eq. discrP: relative sketched residual
 * below eta * noise_norms[r] / ||b_r||), after which it is masked out.
 *   B           device, FP64, column-major m x nrhs (column r = b_r)
 *   noise_norms host, nrhs values (<= 0: that column runs to opts->maxit)
 *   opts        as for sflsqr_solve; opts->noise_norm is ignored; precond
 *               must be identity or diagonal (reweighting is not batched)
 *   X           device, FP64, column-major n x nrhs (output)
 *   infos       host, nrhs entries (may be NULL: then the call does not wait)
 * 1 <= nrhs <= 256.  Vectors are kept in the plan's vector precision (FP64 for
 * an FP64 plan, FP32 otherwise); the small problems are FP64.  The plan keeps
 * every basis vector of the solve: (2 maxit + 2) * max(m, n) * ld vectors of
 * that precision (ld = next power of two >= max(nrhs, 4)) plus O(nrhs * s *
 * maxit) doubles; SFL_ENOMEM if they do not fit.  Returns SFL_EINVAL for bad
 * arguments, SFL_EUNSUPPORTED for the reweighting preconditioner, a full
 * window, orth_against_z = 1 or an explicit sketch. */
int sflsqr_solve_batched(sfl_plan *plan, int32_t nrhs, const double *B, const double *noise_norms,
                         const sfl_opts *opts, double *X, sfl_info *infos, sfl_stream stream);

/* RHS tile width the SpMM tuner picked for the plan's most recent batch
 * session: which = 0 for A, 1 for A^T / B.  0 if the plan has run no batch,
 * -1 for bad arguments.  Results never depend on it. */
int sfl_batched_tile(const sfl_plan *plan, int32_t which);

/* ---- differentiation ------------------------------------------------------ */

/* Fixed-k batched sFLSQR for differentiation: exactly opts->maxit steps of
 * Algorithm 1 (no discrepancy test; a right-hand side stops early only on a
 * breakdown), flexible operator identity or z = diag(diag_w) p, window <= 3.
 * Arguments as sflsqr_solve_batched without the noise levels.  The plan keeps
 * the whole forward state (every basis vector, A z_j, the coefficients and the
 * small QR) for sflsqr_adjoint_batched until its next batched call with other
 * sizes, or another fixed-k call.  The forward state lives in the plan, not
 * in a state object of the caller's: one plan holds one differentiable
 * forward at a time, so two forwards whose adjoints are both still needed
 * take two plans (on the same operator).  The window is capped at 3 here
 * (the adjoint's combination kernels hold the window's vectors in registers)
 * and at 8 for the solves; wider windows are full orthogonalization
 * (window < 0) in the single solves. */
int sflsqr_fixed_batched(sfl_plan *plan, int32_t nrhs, const double *B, const sfl_opts *opts, double *X,
                         sfl_info *infos, sfl_stream stream);

/* Reverse-mode adjoint of the plan's latest sflsqr_fixed_batched call: for a
 * loss L(X), given Xbar = dL/dX (device, FP64, column-major n x nrhs) it writes
 * Bbar = dL/dB (device, FP64, column-major m x nrhs) and, if dbar is not NULL,
 * dbar = dL/d(diag_w) summed over the right-hand sides (device, FP64, n; at
 * diag_w = 1 for an identity operator).  The derivative is that of the exact
 * fixed-k map (modified Gram-Schmidt windows, normalisations, sketched QR
 * solve, x = Z y), evaluated at the kept forward state.  SFL_EINVAL when the
 * plan keeps no such forward or nrhs differs from it. */
int sflsqr_adjoint_batched(sfl_plan *plan, int32_t nrhs, const double *Xbar, double *Bbar, double *dbar,
                           sfl_stream stream);

/* Number of sflsqr_fixed_batched calls made on the plan (a forward's identity
 * for the adjoint that must follow it); -1 for a NULL plan. */
int64_t sfl_fixed_calls(const sfl_plan *plan);

/* ---- misc --------------------------------------------------------------- */

const char *sfl_error_string(int status);
/* Text of the last CUDA error seen by this thread inside the library ("" if none). */
const char *sfl_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SFL_H */
