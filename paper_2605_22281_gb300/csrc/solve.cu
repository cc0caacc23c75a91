// Solve driver: per-configuration sessions (workspace + CUDA graph whose body
// is one step of Algorithm 1 / 2 inside a device-controlled WHILE node), the
// solver entry points, plan apply/destroy and the sketch entry points.
#include <cub/cub.cuh>

#include <chrono>
#include <functional>
#include <cstring>
#include <thread>

#include "engine.h"

namespace sfl {

static constexpr double kHostWaitSeconds = 1800.0;

// Host wait with a wall-clock limit (cudaEventQuery polling).
int wait_stream(cudaStream_t s) {
  cudaEvent_t ev;
  SFL_CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, s);
  if (e != cudaSuccess) { cudaEventDestroy(ev); set_cuda_error(e, "cudaEventRecord"); return SFL_ECUDA; }
  const auto t0 = std::chrono::steady_clock::now();
  int spins = 0;
  for (;;) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) { cudaEventDestroy(ev); set_cuda_error(e, "cudaEventQuery"); return SFL_ECUDA; }
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (dt > kHostWaitSeconds) { cudaEventDestroy(ev); return SFL_ETIMEOUT; }
    if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  cudaEventDestroy(ev);
  return SFL_OK;
}

static int session_alloc(Plan &pl, Session &se, void **p, size_t bytes) {
  if (pl.cap && pl.bytes + bytes > pl.cap) return SFL_ENOMEM;
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) { cudaGetLastError(); set_cuda_error(e, "cudaMalloc"); return SFL_ENOMEM; }
  se.allocs.push_back(*p);
  se.bytes += bytes;
  pl.bytes += bytes;
  return SFL_OK;
}

static void destroy_session(Plan &pl, Session &se) {
  if (se.exec) cudaGraphExecDestroy(se.exec);
  if (se.graph) cudaGraphDestroy(se.graph);
  for (void *p : se.allocs) cudaFree(p);
  se.allocs.clear();
  pl.bytes -= se.bytes;
  se.bytes = 0;
}

// Dynamic shared memory limit of the product kernels, set once for every
// session: the stash (at most 64 KB) plus, with the fused sketch, an s-vector
// of 64-bit integers.
constexpr size_t kSpmvSmemLimit = 160 * 1024;

// Smallest b with 2^b >= n (n >= 1).
static int log2_ceil(int64_t n) {
  int b = 0;
  while (((int64_t)1 << b) < n) ++b;
  return b;
}

// The Q block of a CTA is staged in shared memory when the whole plan stays
// within this budget (it then serves the four Q products of a step).
constexpr size_t kLsStageBudget = 160 * 1024;

// Staging plan: Q and SAZ blocks (SAZ only for the sFLSMR residual rule),
// else Q only, else neither.  Returns bit 0 = Q, bit 1 = SAZ.
int ls_stage_plan(int s, int maxit, int cluster, bool saz) {
  if (saz && sizeof(double) * ls_smem_doubles(s, maxit, cluster, 1, 1) <= kLsStageBudget) return 3;
  if (sizeof(double) * ls_smem_doubles(s, maxit, cluster, 1, 0) <= kLsStageBudget) return 1;
  return 0;
}

size_t ls_smem_bytes(int s, int maxit, int cluster, bool saz) {
  const int st = ls_stage_plan(s, maxit, cluster, saz);
  return sizeof(double) * ls_smem_doubles(s, maxit, cluster, st & 1, (st >> 1) & 1);
}

// The dynamic shared memory limit of a kernel is one attribute shared by all
// sessions: the small-LS kernel is allowed the device maximum once, so no
// session can lower another's limit.
static int ls_max_dynamic_smem() {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, ls_step_kernel) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return optin - (int)fa.sharedSizeBytes;   // the limit covers static plus dynamic shared memory
}

cudaError_t ls_allow_max_smem() {
  const int lim = ls_max_dynamic_smem();
  if (lim <= 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(ls_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(ls_step_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

int ls_cluster_size(int s, int maxit, bool saz, int max_cluster) {
  if (ls_allow_max_smem() != cudaSuccess) { cudaGetLastError(); return 0; }
  const int lim = ls_max_dynamic_smem();
  for (int cl : {16, 8, 4, 2, 1}) {
    if (cl > max_cluster) continue;
    static_assert(kMaxCluster == 16, "largest cluster tried");
    const size_t smem = ls_smem_bytes(s, maxit, cl, saz);
    if (smem > (size_t)lim) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, ls_step_kernel, &cfg) == cudaSuccess && n >= 1) return cl;
    cudaGetLastError();
  }
  return 0;
}

cudaError_t launch_ls(const LsParams &p, int cluster, size_t smem, cudaStream_t s, bool pdl, int nprob) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster * nprob);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, ls_step_kernel, p);
}

// Whether the warps of a product CTA take the CTA's 32-row blocks in turn
// (instead of one balanced range each): for pixel-tiled operators whose CTAs
// own at least eight 16 x 16 tiles, so the eight warps share one tile's
// gathers; below that a CTA's rows fit in about a tile anyway, and splitting
// a few blocks among eight warps would leave some idle.
bool interleave_rows(const StoredCsr &M, int row_ctas) {
  return M.orig != nullptr && row_ctas > 0 && M.rows / row_ctas >= 8 * 256;
}

// Row range of each of W warps over the rows of M, balanced by row cost
// (4 * ceil(len / unit) + 1 per row, exclusive scan, binary search per warp).
// Temporaries are freed before returning; the stream is synchronised.
int balance_rows(const StoredCsr &M, int unit, int W, int32_t *wrow, cudaStream_t s, int slot, int extra) {
  const int64_t rows = M.rows;
  int64_t *cost = nullptr, *prefix = nullptr, *cost_x = nullptr, *prefix_x = nullptr;
  void *tst = nullptr;
  size_t tb = 0;
  int r = SFL_OK;
  auto fail = [&](cudaError_t e, const char *what) {
    set_cuda_error(e, what);
    return SFL_ECUDA;
  };
  const bool two = extra > 0 && W % kWarps == 0;   // CTA ranges priced with the sketch (see balance_rows2_kernel)
  cudaError_t e = cub::DeviceScan::ExclusiveSum(nullptr, tb, (int64_t *)nullptr, (int64_t *)nullptr, (int)(rows + 1), s);
  if (e == cudaSuccess) e = cudaMalloc(&cost, sizeof(int64_t) * (rows + 1));
  if (e == cudaSuccess) e = cudaMalloc(&prefix, sizeof(int64_t) * (rows + 1));
  if (e == cudaSuccess && two) e = cudaMalloc(&cost_x, sizeof(int64_t) * (rows + 1));
  if (e == cudaSuccess && two) e = cudaMalloc(&prefix_x, sizeof(int64_t) * (rows + 1));
  if (e == cudaSuccess) e = cudaMalloc(&tst, tb ? tb : 16);
  if (e == cudaSuccess) {
    row_cost_kernel<<<(unsigned)((rows + 256) / 256), 256, 0, s>>>(M.rowptr, rows, unit, slot, extra, cost, cost_x);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(tst, tb, cost, prefix, (int)(rows + 1), s);
  if (e == cudaSuccess && two) e = cub::DeviceScan::ExclusiveSum(tst, tb, cost_x, prefix_x, (int)(rows + 1), s);
  if (e == cudaSuccess) {
    const int nc = W / kWarps;
    if (two) balance_rows2_kernel<<<(nc + 256) / 256, 256, 0, s>>>(prefix, prefix_x, rows, nc, wrow);
    else balance_rows_kernel<<<(W + 256) / 256, 256, 0, s>>>(prefix, rows, W, wrow);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { cudaGetLastError(); r = fail(e, "row balance"); }
  cudaFree(cost);
  cudaFree(prefix);
  cudaFree(cost_x);
  cudaFree(prefix_x);
  cudaFree(tst);
  return r;
}

// Row-major sparse-sign table for ncols columns: pairs (row, column|sign) in
// column-major draw order, stably sorted by row, so every row lists its
// columns in increasing order (deterministic).
int build_sketch_table(uint64_t seed, int s, int zeta, int64_t ncols, int32_t *rowptr, uint32_t *ent,
                              SketchTableTmp &t, int *err, cudaStream_t st) {
  const int64_t nent = ncols * zeta;
  sketch_pairs_kernel<<<(unsigned)((ncols + 255) / 256), 256, 0, st>>>(seed, s, zeta, ncols, t.kin, t.vin, err);
  SFL_CU(cudaGetLastError());
  int bits = 1;
  while ((1 << bits) < s) ++bits;
  size_t need = 0;
  SFL_CU(cub::DeviceRadixSort::SortPairs(nullptr, need, t.kin, t.kout, t.vin, ent, (int)nent, 0, bits, st));
  if (need > t.cub_bytes) return SFL_ENOMEM;
  SFL_CU(cub::DeviceRadixSort::SortPairs(t.cub, need, t.kin, t.kout, t.vin, ent, (int)nent, 0, bits, st));
  sketch_rowptr_kernel<<<(s + 256) / 256, 256, 0, st>>>(t.kout, nent, s, rowptr);
  SFL_CU(cudaGetLastError());
  return SFL_OK;
}

size_t sketch_sort_bytes(int64_t nent, int s) {
  int bits = 1;
  while ((1 << bits) < s) ++bits;
  size_t need = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, need, (uint32_t *)nullptr, (uint32_t *)nullptr, (uint32_t *)nullptr,
                                  (uint32_t *)nullptr, (int)nent, 0, bits);
  return need;
}

template <typename VT, typename XT>
struct Engine {
  using O = Ops<VT, XT>;
  using ACC = typename AccT<XT>::T;

  static SpmvParams<VT, XT> base_params(const Plan &pl, const Session &se, const StoredCsr &M, int mode) {
    SpmvParams<VT, XT> p{};
    p.rowptr = M.rowptr; p.col = M.col; p.val = (const VT *)M.val; p.rows = M.rows;
    p.dcol = M.dcol; p.rbase = M.rbase;
    p.orig = M.orig;
    p.mode = mode;
    p.method = se.key.method;
    p.ell = se.key.ell;
    p.st = se.st;
    p.part = se.part;
    p.orth_z = se.key.orth_z;
    if (mode == kModeFwd) { p.wrow = se.wrowA; p.G_prev = se.grid_vec; }
    else if (mode == kModeBwd) { p.wrow = se.wrowT; p.G_prev = se.grid_vec; }
    else if (mode == kModeInitBwd) { p.wrow = se.wrowT; p.G_prev = se.grid_init; }
    p.wring = (XT *)se.wring; p.wstride = pl.A.rows; p.RW = se.RW;
    p.pring = (XT *)se.pring; p.pstride = pl.A.cols; p.RP = se.RP;
    p.Z = (XT *)se.Z; p.zstride = pl.A.cols; p.sigZ = se.sigZ;
    p.wraw = (XT *)se.wraw; p.zraw = (XT *)se.zraw;
    p.Hband = se.Hband;
    p.want_h = se.key.method != kSFLSQR;
    p.hb_ell = se.hb_ell;
    if (pl.matfree) set_proj(pl, p, mode == kModeFwd || mode == kModeInitB);
    if (se.sk_fused && mode == kModeFwd && se.skw_rec) {
      p.sk_s = se.key.s; p.sk_zeta = se.key.zeta; p.sk_rec = se.skw_rec; p.sk_cap = se.grid_spmv_A;
      p.sk_seed_add = se.key.method == kSFLSMR ? 1 : 0;   // sFLSMR's m-side stop sketch is drawn from seed + 1
    } else if (se.sk_fused && mode == kModeBwd && se.skz_rec) {
      p.sk_s = se.key.s; p.sk_zeta = se.key.zeta; p.sk_rec = se.skz_rec; p.sk_cap = se.grid_spmv_T;
      p.sk_seed_add = 0;
    }
    p.full = se.full;
    if (se.full) {
      p.ell = 0;                        // the rings and scalars run as for window 0, with no window dots
      p.wfull = mode == kModeInitB ? (XT *)se.Wfull : nullptr;
      p.sigWall = se.sigWall;
    }
    return p;
  }

  // Matrix-free plans: the projector of the product (forward ray walk, or the
  // matched / unmatched pixel-driven back-projection), rows split evenly.
  static void set_proj(const Plan &pl, SpmvParams<VT, XT> &p, bool fwd) {
    p.ptab = pl.ct_tab;
    p.pfix = pl.ct_fix;
    p.pN = pl.ct_N; p.pna = pl.ct_na; p.pnb = pl.ct_nb;
    p.proj = fwd ? kProjRay : (pl.ct_back ? kProjBackLinear : kProjBackChord);
    p.wrow = nullptr;
  }

  static SketchParams<XT> sketch_params(const Session &se, int mode) {
    SketchParams<XT> q{};
    q.mode = mode; q.method = se.key.method; q.s = se.key.s; q.isz = 1.0 / std::sqrt((double)se.key.zeta);
    if (se.key.dense_S) {      // an explicit sketch is applied as given
      q.isz = 1.0;
      q.dM = se.key.method == kSFLSQR ? se.key.dense_S : se.key.dense_Sm;
      q.dN = se.key.method == kSFLSMR ? se.key.dense_S : nullptr;
      q.lenM = se.m; q.lenN = se.n;
    }
    if (se.key.sk_kind != SFL_SKETCH_SPARSE_SIGN) {   // regenerated from the seed in every application
      q.gen = se.key.sk_kind;
      q.isz = 1.0 / std::sqrt((double)se.key.s);
      q.lenM = se.m; q.lenN = se.n;
      q.bitsM = log2_ceil(se.m); q.bitsN = log2_ceil(se.n);
      q.gen_m_add = se.key.method == kSFLSMR ? 1 : 0;
    }
    q.st = se.st;
    q.v64 = se.bbuf;
    q.wraw = (const XT *)se.wraw; q.zraw = (const XT *)se.zraw;
    q.RW = se.RW; q.RP = se.RP;
    q.rowM = se.skM_row; q.entM = se.skM_ent; q.rowN = se.skN_row; q.entN = se.skN_ent;
    q.SAZ = se.SAZ; q.SAtW = se.SAtW; q.rhs = se.rhs; q.e = se.e; q.sbm = se.sbm;
    return q;
  }

  static OrthParams<XT> orth_params(const Plan &pl, const Session &se, int side) {
    OrthParams<XT> o{};
    o.st = se.st; o.side = side; o.ell = se.key.ell; o.orth_z = se.key.orth_z;
    o.method = se.key.method;
    o.part = se.part;
    o.G_prev = side == 0 ? se.grid_spmv_T : se.grid_spmv_A;
    o.Hband = se.Hband;
    o.want_h = se.key.method != kSFLSQR;
    o.full = se.full;
    o.scale_ring = side == 0 ? se.RW : se.RP;
    if (side == 0) {
      o.len = pl.A.cols; o.raw = (const XT *)se.zraw; o.ring = (XT *)se.pring; o.stride = pl.A.cols; o.R = se.RP;
      o.Z = (XT *)se.Z; o.zstride = pl.A.cols; o.sigZ = se.sigZ;
      o.precond = se.key.precond; o.diag_w = se.dw; o.y = se.y;
    } else {
      o.len = pl.A.rows; o.raw = (const XT *)se.wraw; o.ring = (XT *)se.wring; o.stride = pl.A.rows; o.R = se.RW;
      o.sigZ = se.sigZ;
    }
    if (side == 1 && se.sk_fused && se.skw_rec) {   // the A z_k product's sketch records -> S A Z column k
      o.sk_rec = se.skw_rec; o.sk_cap = se.grid_spmv_A; o.sk_s = se.key.s; o.sk_col_base = se.SAZ;
      o.sk_isz = 1.0 / std::sqrt((double)se.key.zeta);
    }
    if (se.full) {
      o.ell = 0;
      o.vfull = (XT *)(side == 0 ? se.Pfull : se.Wfull);
      o.raw = (const XT *)(side == 0 ? se.zcgs : se.wcgs);   // block CGS2 output
    }
    return o;
  }

  static LsParams ls_params(const Session &se, int use_cond, cudaGraphConditionalHandle h) {
    LsParams q{};
    // FLSQR runs the sFLSMR form of the small problem with identity columns
    q.st = se.st; q.method = se.key.method == kFLSQR ? kSFLSMR : se.key.method; q.s = se.key.s;
    q.maxit = se.key.maxit; q.ell = se.hb_ell;
    q.stop_rule = se.key.method == kFLSQR ? SFL_STOP_RULE_NORMAL : se.key.stop_rule;
    q.stage_q = se.ls_stage & 1;
    q.stage_saz = (se.ls_stage >> 1) & 1;
    q.Q = se.Q; q.Rinv = se.Rinv; q.y = se.y; q.e = se.e;
    q.SAZ = se.SAZ; q.SAtW = se.SAtW; q.Hband = se.Hband; q.sbm = se.sbm; q.rhs = se.rhs;
    q.relres_hist = se.key.r_hist;
    q.cond = h; q.use_cond = use_cond;
    if (se.sk_fused && se.skz_rec) {
      q.skz_rec = se.skz_rec; q.skz_cap = se.grid_spmv_T;
      q.sk_isz = 1.0 / std::sqrt((double)se.key.zeta);
      q.RW = se.RW;
    }
    return q;
  }

  // Kernel classes of the profiled driver (sfl_kernel_times index).
  enum { kKSketchInit = 0, kKInitB, kKInitBwd, kKOrthZ, kKFwd, kKOrthW, kKBwd, kKLs, kKSolution, kKSketch, kKOrthFull,
         kKLowRank };

  // Rank-r truncation of p~_k (Z column k - 1) by the randomized SVD: the
  // kernels of lowrank.cuh in order (range finder, subspace iteration, small
  // eigenproblem, z~_k = U V^T written over the column), in RT arithmetic.
  template <typename RT>
  static int k_lowrank_t(const Plan &pl, const Session &se, const LrParams<RT> &lp, cudaStream_t s) {
    const XT *Zc = (const XT *)se.Z;
    XT *Zw = (XT *)se.Z;
    const int64_t zs = pl.A.cols;
    const int N1 = lp.N1, N2 = lp.N2, L = lp.l;
    const int KS1 = (N1 + kLrK - 1) / kLrK, KS2 = (N2 + kLrK - 1) / kLrK;
    constexpr int GR = LrLim<RT>::GR;
    auto cdiv = [](int a, int b) { return (a + b - 1) / b; };
    // shifted Cholesky QR (shift 11 (M l + l (l + 1)) u trace), then Cholesky QR twice: the result in b
    auto orth = [&](int M, int KS, RT *a, RT *b) {
      const RT shift = RT(11) * RT((int64_t)M * L + (int64_t)L * (L + 1)) * LrLim<RT>::u;
      lr_orth_kernel<RT><<<cdiv(M, GR), kThreads, 0, s>>>(lp, 0, nullptr, a, M, KS, shift);
      lr_orth_kernel<RT><<<cdiv(M, GR), kThreads, 0, s>>>(lp, 1, a, b, M, 0, RT(0));
      lr_orth_kernel<RT><<<cdiv(M, GR), kThreads, 0, s>>>(lp, 1, b, a, M, 0, RT(0));
      lr_apply_kernel<RT><<<cdiv(M * L, kThreads), kThreads, 0, s>>>(lp, a, M, b);
    };
    lr_clear_flag_kernel<<<1, 1, 0, s>>>(lp.flag);
    lr_mul_kernel<RT, XT, false><<<dim3(cdiv(N1, kLrTile), KS2), kThreads, 0, s>>>(lp, Zc, zs, lp.Omega);
    orth(N1, KS2, lp.Y, lp.Qm);
    for (int it = 0; it < lp.q; ++it) {
      lr_mul_kernel<RT, XT, true><<<dim3(cdiv(N2, kLrTile), KS1), kThreads, 0, s>>>(lp, Zc, zs, lp.Qm);
      orth(N2, KS1, lp.Bt, lp.Qt);
      lr_mul_kernel<RT, XT, false><<<dim3(cdiv(N1, kLrTile), KS2), kThreads, 0, s>>>(lp, Zc, zs, lp.Qt);
      orth(N1, KS2, lp.Y, lp.Qm);
    }
    lr_mul_kernel<RT, XT, true><<<dim3(cdiv(N2, kLrTile), KS1), kThreads, 0, s>>>(lp, Zc, zs, lp.Qm);
    lr_gram_eig_kernel<RT><<<cdiv(N2, GR), kThreads, 0, s>>>(lp, KS1);
    lr_uv_kernel<RT><<<cdiv((N1 + N2) * lp.r, kThreads), kThreads, 0, s>>>(lp);
    lr_outer_kernel<RT, XT><<<dim3(cdiv(N2, 32), cdiv(N1, 32)), kThreads, 0, s>>>(lp, Zw, zs);
    return cudaGetLastError() == cudaSuccess ? SFL_OK : SFL_ECUDA;
  }
  static int k_lowrank(const Plan &pl, const Session &se, cudaStream_t s) {
    return se.key.lr_fp64 ? k_lowrank_t<double>(pl, se, se.lr64, s) : k_lowrank_t<float>(pl, se, se.lr32, s);
  }

  template <typename RT>
  static int alloc_lowrank(Plan &pl, Session &se, const SessionKey &key, LrParams<RT> &lp, cudaStream_t s) {
    lp.st = se.st;
    lp.N1 = pl.img_rows; lp.N2 = pl.img_cols;
    lp.r = key.lr_rank; lp.l = key.lr_rank + key.lr_over; lp.q = key.lr_power;
    const int64_t N1 = lp.N1, N2 = lp.N2, L = lp.l, Nm = std::max(N1, N2);
    const int64_t KSm = (Nm + kLrK - 1) / kLrK, GBm = (Nm + LrLim<RT>::GR - 1) / LrLim<RT>::GR;
    int r;
#define LA(ptr, bytes) if ((r = session_alloc(pl, se, (void **)&(ptr), (bytes)))) return r;
    LA(lp.Omega, sizeof(RT) * N2 * L);
    LA(lp.Y, sizeof(RT) * N1 * L);
    LA(lp.Qm, sizeof(RT) * N1 * L);
    LA(lp.Qt, sizeof(RT) * N2 * L);
    LA(lp.Bt, sizeof(RT) * N2 * L);
    LA(lp.U, sizeof(RT) * N1 * lp.r);
    LA(lp.V, sizeof(RT) * N2 * lp.r);
    LA(lp.part, sizeof(RT) * KSm * Nm * L);
    LA(lp.gpart, sizeof(RT) * GBm * L * L);
    LA(lp.small, sizeof(RT) * LrLim<RT>::L * LrLim<RT>::L);
    LA(lp.flag, sizeof(int));
    LA(lp.ticket, sizeof(int));
#undef LA
    SFL_CU(cudaMemsetAsync(lp.flag, 0, sizeof(int), s));
    SFL_CU(cudaMemsetAsync(lp.ticket, 0, sizeof(int), s));
    return SFL_OK;
  }

  static CgsParams<XT> cgs_params(const Plan &pl, const Session &se, int side) {
    CgsParams<XT> c{};
    c.st = se.st; c.side = side; c.want_h = se.key.method != kSFLSQR;
    c.len = side == 0 ? pl.A.cols : pl.A.rows;
    c.x = (const XT *)(side == 0 ? se.zraw : se.wraw);
    c.xo = (XT *)(side == 0 ? se.zcgs : se.wcgs);
    c.V = (const XT *)(side == 0 ? se.Pfull : se.Wfull);
    c.vstride = c.len;
    c.sigV = side == 0 ? se.sigZ : se.sigWall;
    c.sigP = se.sigZ;
    c.rec = se.cgs_rec; c.cap = se.grid_cgs;
    c.coef = se.cgs_coef;
    c.Hband = se.Hband; c.hb_ell = se.hb_ell;
    return c;
  }
  // Block CGS2 of the raw product output against the whole stored basis (five launches).
  static int k_cgs(const Plan &pl, const Session &se, int side, cudaStream_t s) {
    const CgsParams<XT> c = cgs_params(pl, se, side);
    const int gred = (se.key.maxit + 1 + kWarps - 1) / kWarps;
    cgs_dots_kernel<XT><<<se.grid_cgs, kThreads, 0, s>>>(c, 1);
    cgs_reduce_kernel<XT><<<gred, kThreads, 0, s>>>(c, 1, se.grid_cgs);
    cgs_dots_kernel<XT><<<se.grid_cgs, kThreads, 0, s>>>(c, 2);
    cgs_reduce_kernel<XT><<<gred, kThreads, 0, s>>>(c, 2, se.grid_cgs);
    cgs_update_kernel<XT><<<se.grid_vec, kThreads, 0, s>>>(c);
    return cudaGetLastError() == cudaSuccess ? SFL_OK : SFL_ECUDA;
  }

  template <typename F> static int launch_one(int cls, F &&f, const std::function<int(int, std::function<int()>)> *tm) {
    if (tm) return (*tm)(cls, std::function<int()>(f));
    return f();
  }

  static int k_sketch(const Session &se, int mode, int rows, cudaStream_t s, bool pdl = false) {
    return launch_k(sketch_rows_kernel<XT>, dim3(rows), dim3(kSkWarps * 32), 0, s, pdl, sketch_params(se, mode),
                    rows) == cudaSuccess ? SFL_OK : SFL_ECUDA;
  }
  static int k_spmv(const Plan &pl, const Session &se, int mode, cudaStream_t s, bool pdl = false) {
    const bool fwd = (mode == kModeFwd || mode == kModeInitB);
    const StoredCsr &M = fwd ? pl.A : pl.T;
    SpmvParams<VT, XT> p = base_params(pl, se, M, mode);
    if (mode == kModeInitB) {
      p.rows = pl.A.rows;
      p.b = se.bbuf;
      return O::spmv(p, 1, false, se.grid_init, se.smem_init, s) == cudaSuccess ? SFL_OK : SFL_ECUDA;
    }
    const int grid = fwd ? se.grid_spmv_A : se.grid_spmv_T;
    const size_t smem = fwd ? se.smem_A : se.smem_T;
    p.interleave = interleave_rows(M, grid - 1);
    return O::spmv(p, M.lpr, true, grid, smem, s, pdl) == cudaSuccess ? SFL_OK : SFL_ECUDA;
  }
  static int k_orth(const Plan &pl, const Session &se, int side, cudaStream_t s, bool pdl = false) {
    return O::orth(orth_params(pl, se, side), se.grid_vec, se.smem_orth, s, pdl) == cudaSuccess ? SFL_OK
                                                                                                  : SFL_ECUDA;
  }

  using Timer = std::function<int(int, std::function<int()>)>;

  static int enqueue_prologue(const Plan &pl, const Session &se, cudaStream_t s, const Timer *tm = nullptr) {
    int r;
    if ((r = launch_one(kKInitB, [&] { return k_spmv(pl, se, kModeInitB, s); }, tm))) return r;
    if ((r = launch_one(kKInitBwd, [&] { return k_spmv(pl, se, kModeInitBwd, s); }, tm))) return r;
    if (se.key.method == kFLSQR) {   // no sketch: the small problem's right-hand side is beta e_1
      flsqr_rhs_kernel<<<1, kThreads, 0, s>>>(se.st, se.rhs, se.e, se.key.s);
      SFL_CU(cudaGetLastError());
      return SFL_OK;
    }
    if ((r = launch_one(kKSketchInit, [&] {
           int q = k_sketch(se, kSkInitB, se.key.s, s);
           if (!q && se.key.method == kSFLSMR) q = k_sketch(se, kSkInitBwd, se.key.s, s);
           return q;
         }, tm)))
      return r;
    return SFL_OK;
  }

  // One step; pdl: kernels after the first depend programmatically on their
  // predecessor (graph body only), except the sketch.
  static int enqueue_body(const Plan &pl, const Session &se, cudaStream_t s, int use_cond,
                          cudaGraphConditionalHandle h, const Timer *tm = nullptr, bool pdl = false) {
    int r;
    if (se.full && (r = launch_one(kKOrthFull, [&] { return k_cgs(pl, se, 0, s); }, tm))) return r;
    if ((r = launch_one(kKOrthZ, [&] { return k_orth(pl, se, 0, s); }, tm))) return r;
    if (se.lowrank && (r = launch_one(kKLowRank, [&] { return k_lowrank(pl, se, s); }, tm))) return r;
    if ((r = launch_one(kKFwd, [&] { return k_spmv(pl, se, kModeFwd, s, pdl); }, tm))) return r;
    if (se.full && (r = launch_one(kKOrthFull, [&] { return k_cgs(pl, se, 1, s); }, tm))) return r;
    if ((r = launch_one(kKOrthW, [&] { return k_orth(pl, se, 1, s, pdl); }, tm))) return r;
    if ((r = launch_one(kKBwd, [&] { return k_spmv(pl, se, kModeBwd, s, pdl); }, tm))) return r;
    const int gsk = se.key.s * (se.key.method == kSFLSMR ? 2 : 1);
    // no programmatic edge into the sketch: its small CTAs, launched early,
    // would pile onto the first SMs the product frees (measured 2x slower)
    if (se.key.method != kFLSQR && !se.sk_fused &&
        (r = launch_one(kKSketch, [&] { return k_sketch(se, kSkStep, gsk, s); }, tm)))
      return r;
    if ((r = launch_one(kKLs, [&] {
           return launch_ls(ls_params(se, use_cond, h), se.ls_cluster, se.smem_ls, s, pdl) == cudaSuccess
                      ? SFL_OK
                      : SFL_ECUDA;
         }, tm)))
      return r;
    if (se.key.x_hist) {
      SFL_CU(O::solution(se.st, (const XT *)se.Z, pl.A.cols, se.sigZ, se.y, pl.A.cols, nullptr, se.key.x_hist,
                         se.grid_vec, s));
      clear_hist_flag_kernel<<<1, 1, 0, s>>>(se.st);
      SFL_CU(cudaGetLastError());
    }
    return SFL_OK;
  }

  static int enqueue_epilogue(const Plan &pl, const Session &se, cudaStream_t s, const Timer *tm = nullptr) {
    return launch_one(kKSolution, [&] {
      return O::solution(se.st, (const XT *)se.Z, pl.A.cols, se.sigZ, se.y, pl.A.cols, se.xbuf, nullptr, se.grid_vec,
                         s) == cudaSuccess ? SFL_OK : SFL_ECUDA;
    }, tm);
  }

  static int build_graph(const Plan &pl, Session &se) {
    // programmatic edges inside the loop body first; plain edges if refused
    const int r = build_graph_pdl(pl, se, true);
    if (r != SFL_ECUDA) return r;
    cudaGetLastError();
    return build_graph_pdl(pl, se, false);
  }

  static int build_graph_pdl(const Plan &pl, Session &se, bool pdl) {
    cudaStream_t cs;
    SFL_CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    int r = SFL_OK;
    cudaGraph_t g = nullptr, gp = nullptr, ge = nullptr;
    do {
      if (cudaGraphCreate(&g, 0) != cudaSuccess) { r = SFL_ECUDA; break; }
      // prologue
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { r = SFL_ECUDA; break; }
      r = enqueue_prologue(pl, se, cs);
      if (cudaStreamEndCapture(cs, &gp) != cudaSuccess || r) { r = r ? r : SFL_ECUDA; break; }
      cudaGraphNode_t np, nw, ne;
      if (cudaGraphAddChildGraphNode(&np, g, nullptr, 0, gp) != cudaSuccess) { r = SFL_ECUDA; break; }
      // loop: WHILE node whose condition the small-LS kernel sets every step
      cudaGraphConditionalHandle h;
      if (cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault) != cudaSuccess) { r = SFL_ECUDA; break; }
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      if (cudaGraphAddNode(&nw, g, &np, nullptr, 1, &cp) != cudaSuccess) { r = SFL_ECUDA; break; }
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        r = SFL_ECUDA; break;
      }
      r = enqueue_body(pl, se, cs, 1, h, nullptr, pdl);
      cudaGraph_t body_out = body;
      if (cudaStreamEndCapture(cs, &body_out) != cudaSuccess || r) { r = r ? r : SFL_ECUDA; break; }
      // epilogue
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { r = SFL_ECUDA; break; }
      r = enqueue_epilogue(pl, se, cs);
      if (cudaStreamEndCapture(cs, &ge) != cudaSuccess || r) { r = r ? r : SFL_ECUDA; break; }
      if (cudaGraphAddChildGraphNode(&ne, g, &nw, 1, ge) != cudaSuccess) { r = SFL_ECUDA; break; }
      cudaError_t e = cudaGraphInstantiate(&se.exec, g, 0);
      if (e != cudaSuccess) { set_cuda_error(e, "cudaGraphInstantiate"); r = SFL_ECUDA; break; }
      se.graph = g;
      g = nullptr;
    } while (0);
    if (r == SFL_ECUDA) {
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) set_cuda_error(e, "graph build");
    }
    if (g) cudaGraphDestroy(g);
    if (gp) cudaGraphDestroy(gp);
    if (ge) cudaGraphDestroy(ge);
    cudaStreamDestroy(cs);
    return r;
  }

  static int create(Plan &pl, const SessionKey &key, cudaStream_t s, Session **out) {
    auto se = std::make_unique<Session>();
    se->key = key;
    const int64_t m = pl.A.rows, n = pl.A.cols;
    se->m = m; se->n = n;
    const int S = key.s, K = key.maxit, Z = key.zeta;
    const size_t xs = sizeof(XT);
    se->full = key.ell < 0;
    const int ell = se->full ? 0 : key.ell;        // window of the ring machinery
    se->hb_ell = se->full ? K : ell;
    se->RW = ell + 2;
    se->RP = ell + 1;
    int r;
#define SA(ptr, bytes) if ((r = session_alloc(pl, *se, (void **)&(ptr), (bytes)))) { destroy_session(pl, *se); return r; }
    SA(se->st, sizeof(SolveState));
    SA(se->wring, xs * se->RW * m);
    SA(se->pring, xs * se->RP * n);
    SA(se->wraw, xs * m);
    SA(se->zraw, xs * n);
    SA(se->Z, xs * (size_t)n * K);
    SA(se->sigZ, sizeof(double) * K);
    if (se->full) {
      SA(se->Pfull, xs * (size_t)n * K);
      SA(se->Wfull, xs * (size_t)m * (K + 1));
      SA(se->sigWall, sizeof(double) * (K + 2));
      SA(se->zcgs, xs * n);
      SA(se->wcgs, xs * m);
      se->grid_cgs = (int)std::max<int64_t>(pl.num_sms * 2, (std::max(m, n) + kCgsChunk - 1) / kCgsChunk);
      SA(se->cgs_rec, sizeof(double) * (size_t)(K + 2) * se->grid_cgs);
      SA(se->cgs_coef, sizeof(double) * 2 * (kMaxIt + 2));
    }
    if (key.precond == SFL_PRECOND_LOWRANK) {
      se->lowrank = true;
      r = key.lr_fp64 ? alloc_lowrank<double>(pl, *se, key, se->lr64, s) : alloc_lowrank<float>(pl, *se, key, se->lr32, s);
      if (r) { destroy_session(pl, *se); return r; }
    }
    SA(se->skM_row, sizeof(int32_t) * (S + 1));
    SA(se->skM_ent, sizeof(uint32_t) * (size_t)Z * m);
    if (key.method == kSFLSMR) {
      SA(se->skN_row, sizeof(int32_t) * (S + 1));
      SA(se->skN_ent, sizeof(uint32_t) * (size_t)Z * n);
    }
    const int64_t nent = (int64_t)Z * std::max(m, n);
    SA(se->sk_kin, sizeof(uint32_t) * nent);
    SA(se->sk_vin, sizeof(uint32_t) * nent);
    SA(se->sk_kout, sizeof(uint32_t) * nent);
    se->sk_cub_bytes = sketch_sort_bytes(nent, S) + 256;
    SA(se->sk_cub, se->sk_cub_bytes);
    SA(se->Q, sizeof(double) * (size_t)S * K);
    SA(se->Rinv, sizeof(double) * (size_t)K * K);
    SA(se->y, sizeof(double) * K);
    SA(se->e, sizeof(double) * S);
    SA(se->rhs, sizeof(double) * S);
    SA(se->SAZ, sizeof(double) * (size_t)S * K);
    SA(se->SAtW, sizeof(double) * (size_t)S * (K + 1));
    SA(se->Hband, sizeof(double) * (size_t)K * (se->hb_ell + 2));
    SA(se->sbm, sizeof(double) * S);
    SA(se->bbuf, sizeof(double) * m);
    SA(se->xbuf, sizeof(double) * n);
    if (key.precond == SFL_PRECOND_DIAG) SA(se->dw, sizeof(double) * n);
    SA(se->err, sizeof(int));
    // launch shapes
    const size_t stashA = spmv_smem_bytes(pl.A.lpr, sizeof(ACC)), stashT = spmv_smem_bytes(pl.T.lpr, sizeof(ACC));
    se->smem_A = stashA;
    se->smem_T = stashT;
    se->smem_init = spmv_smem_bytes(1, sizeof(ACC));
    // one limit per kernel for every session (room for the fused sketch), so no session lowers another's
    SFL_CU(O::set_smem(pl.A.lpr, true, kSpmvSmemLimit));
    SFL_CU(O::set_smem(pl.T.lpr, true, kSpmvSmemLimit));
    SFL_CU(O::set_smem(1, false, se->smem_init));
    // fused sketch: a product that sketches its output keeps an s-vector of
    // 64-bit integers after its stash; fused only where that costs the
    // product no resident CTA (otherwise the separate sketch kernel runs).
    // Explicit sketches and FLSQR keep the separate kernel (or none).
    {
      const size_t sk_smem = sizeof(unsigned long long) * (size_t)S;
      auto occ_of = [&](int lpr, size_t smem) {
        return pl.matfree ? O::proj_occupancy(smem) : O::spmv_occupancy(lpr, true, smem);
      };
      auto fits = [&](int lpr, size_t stash) {
        return stash + sk_smem <= kSpmvSmemLimit && occ_of(lpr, stash + sk_smem) >= occ_of(lpr, stash);
      };
      const bool want_w = key.method == kSFLSQR || key.stop_rule == SFL_STOP_RULE_RESIDUAL;
      const bool want_z = key.method == kSFLSMR;
      // AUTO: fused where the sketched products' rows are long (measured on
      // this GPU: 1.7 % faster per solve at 1024^2, 921 entries per ray; 9 %
      // slower at 256^2, 230 per ray and 360 per pixel, where the epilogue's
      // per-output draws and the record reduction outweigh the launch saved)
      auto long_rows = [&](const StoredCsr &M) {
        if (pl.matfree) return pl.ct_N >= 512;
        return M.rows > 0 && M.nnz >= 512 * M.rows;
      };
      const bool pick = key.sk_apply == SFL_SKETCH_APPLY_FUSED ||
                        (key.sk_apply == SFL_SKETCH_APPLY_AUTO && (!want_w || long_rows(pl.A)) &&
                         (!want_z || long_rows(pl.T)));
      se->sk_fused = pick && !key.dense_S && key.method != kFLSQR && key.sk_kind == SFL_SKETCH_SPARSE_SIGN &&
                     (!want_w || fits(pl.A.lpr, stashA)) &&
                     (!want_z || fits(pl.T.lpr, stashT));
      if (se->sk_fused && want_w) se->smem_A += sk_smem;
      if (se->sk_fused && want_z) se->smem_T += sk_smem;
    }
    const bool skw = se->sk_fused && (key.method == kSFLSQR || key.stop_rule == SFL_STOP_RULE_RESIDUAL);
    const bool skz = se->sk_fused && key.method == kSFLSMR;
    auto grid_of = [&](int lpr, bool mat, size_t smem) {
      int occ = (mat && pl.matfree) ? O::proj_occupancy(smem) : O::spmv_occupancy(lpr, mat, smem);
      if (occ < 1) occ = 1;
      if (occ > 8) occ = 8;
      return std::min(pl.num_sms * occ, kGroup * kMaxGroups);
    };
    se->grid_spmv_A = std::max(2, grid_of(pl.A.lpr, true, se->smem_A));
    se->grid_spmv_T = std::max(2, grid_of(pl.T.lpr, true, se->smem_T));
    se->grid_init = grid_of(1, false, se->smem_init);
    se->grid_vec = std::min(pl.num_sms * 2, kGroup * kMaxGroups);
    se->smem_orth = orth_smem_bytes(K);
    SFL_CU(O::set_orth_smem(orth_smem_bytes(kMaxIt)));   // one limit for every session
    const bool saz_rule = key.method == kSFLSMR && key.stop_rule == SFL_STOP_RULE_RESIDUAL;   // FLSQR: normal rule
    se->ls_cluster = ls_cluster_size(S, K, saz_rule);
    if (se->ls_cluster < 1) { destroy_session(pl, *se); return SFL_EUNSUPPORTED; }
    se->smem_ls = ls_smem_bytes(S, K, se->ls_cluster, saz_rule);
    se->ls_stage = ls_stage_plan(S, K, se->ls_cluster, saz_rule);
    SFL_CU(ls_allow_max_smem());
    const int gmax = std::max(std::max(se->grid_spmv_A, se->grid_spmv_T), std::max(se->grid_init, se->grid_vec));
    if (gmax > kPartCap) { destroy_session(pl, *se); return SFL_EUNSUPPORTED; }
    const size_t pbytes = sizeof(double) * (size_t)kPartCap * kPartStride;
    SA(se->part.b, pbytes);
    SA(se->part.z, pbytes);
    SA(se->part.p, pbytes);
    SA(se->part.w, pbytes);
    SA(se->part.wn, pbytes);
    // row range of every warp of the two products, balanced by row cost; CTA 0
    // of a product books the step's scalars and runs no rows
    if (skw) SA(se->skw_rec, sizeof(double) * (size_t)S * se->grid_spmv_A);
    if (skz) SA(se->skz_rec, sizeof(double) * (size_t)S * se->grid_spmv_T);
    const int WA = (se->grid_spmv_A - 1) * kWarps, WT = (se->grid_spmv_T - 1) * kWarps;
    SA(se->wrowA, sizeof(int32_t) * (WA + 1));
    SA(se->wrowT, sizeof(int32_t) * (WT + 1));
#undef SA
    const int P = load_width(pl.vdt);
    const int nch = pl.vdt == SFL_BF16 ? SpmvTune<__nv_bfloat16>::NCH
                    : pl.vdt == SFL_F32 ? SpmvTune<float>::NCH : SpmvTune<double>::NCH;
    // FP64 products are bound by FMA issue: their rows also pay for chunk slots
    const bool fp64 = pl.vdt == SFL_F64;
    // a product with the fused sketch prices its per-output draws (about a
    // load iteration per row for zeta = 8 in FP64, a quarter of that in FP32)
    const int sk_extra = std::max(1, fp64 ? key.zeta / 2 : key.zeta / 8);
    if (!pl.matfree &&   // matrix-free products split their rows evenly
        ((r = balance_rows(pl.A, nch * pl.A.lpr * P, WA, se->wrowA, s, fp64 ? pl.A.lpr * P : 0, skw ? sk_extra : 0)) ||
         (r = balance_rows(pl.T, nch * pl.T.lpr * P, WT, se->wrowT, s, fp64 ? pl.T.lpr * P : 0, skz ? sk_extra : 0)))) {
      destroy_session(pl, *se);
      return r;
    }
    SFL_CU(cudaMemsetAsync(se->err, 0, sizeof(int), s));
    SFL_CU(cudaMemsetAsync(se->Hband, 0, sizeof(double) * (size_t)K * (se->hb_ell + 2), s));
    if (key.method == kFLSQR) {   // [I] H = H: identity columns in place of the sketched S A^T W
      identity_cols_kernel<<<64, kThreads, 0, s>>>(se->SAtW, S, K + 1);
      SFL_CU(cudaGetLastError());
    }
    SFL_CU(cudaStreamSynchronize(s));
    if ((r = build_graph(pl, *se))) { destroy_session(pl, *se); return r; }
    *out = se.get();
    pl.sessions.push_back(std::move(se));
    return SFL_OK;
  }

  // Row-major sketch tables for `seed` (kept until the seed changes).
  static int ensure_tables(const Plan &pl, Session &se, uint64_t seed, cudaStream_t s) {
    if (se.key.dense_S || se.key.method == kFLSQR || se.key.sk_kind != SFL_SKETCH_SPARSE_SIGN)
      return SFL_OK;   // explicit, generated or no sketch: no table
    if (se.tab_valid && se.tab_seed == seed) return SFL_OK;
    SketchTableTmp t;
    t.kin = se.sk_kin; t.vin = se.sk_vin; t.kout = se.sk_kout; t.cub = se.sk_cub; t.cub_bytes = se.sk_cub_bytes;
    const bool mr = se.key.method == kSFLSMR;
    int r = build_sketch_table(seed + (mr ? 1 : 0), se.key.s, se.key.zeta, pl.A.rows, se.skM_row, se.skM_ent, t, se.err, s);
    if (!r && mr) r = build_sketch_table(seed, se.key.s, se.key.zeta, pl.A.cols, se.skN_row, se.skN_ent, t, se.err, s);
    if (r) return r;
    se.tab_valid = true;
    se.tab_seed = seed;
    return SFL_OK;
  }

  // Host-driven pass with a CUDA event pair around every launch; steps are
  // enqueued in chunks without host synchronisation inside a chunk.
  static int run_profiled(const Plan &pl, const Session &se, cudaStream_t s, sfl_kernel_times *kt) {
    constexpr int kChunk = 8;
    constexpr int kEv = 2 * (8 * kChunk + 8);
    cudaEvent_t ev[kEv];
    for (int i = 0; i < kEv; ++i) SFL_CU(cudaEventCreate(&ev[i]));
    struct Rec { int cls, step; };
    std::vector<Rec> recs;
    int nev = 0, cur_step = -1;
    Timer tm = [&](int cls, std::function<int()> f) -> int {
      cudaEventRecord(ev[nev], s);
      int q = f();
      cudaEventRecord(ev[nev + 1], s);
      recs.push_back({cls, cur_step});
      nev += 2;
      return q;
    };
    auto flush = [&](int done_steps) -> int {
      if (nev == 0) return SFL_OK;
      SFL_CU(cudaEventSynchronize(ev[nev - 1]));
      for (size_t i = 0; i < recs.size(); ++i) {
        if (recs[i].step >= 0 && recs[i].step >= done_steps) continue;   // returned early after the stop
        float ms = 0.f;
        SFL_CU(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
        kt->ms[recs[i].cls] += ms;
        kt->launches[recs[i].cls] += 1;
      }
      recs.clear();
      nev = 0;
      return SFL_OK;
    };
    int r = enqueue_prologue(pl, se, s, &tm);
    if (r) return r;
    if ((r = flush(0))) return r;
    int done = 0;
    for (int it0 = 0; it0 < se.key.maxit; it0 += kChunk) {
      for (int it = it0; it < std::min(it0 + kChunk, se.key.maxit); ++it) {
        cur_step = it;
        if ((r = enqueue_body(pl, se, s, 0, 0, &tm))) return r;
      }
      int hk[2] = {0, 0};
      SFL_CU(cudaMemcpyAsync(hk, &se.st->k, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
      SFL_CU(cudaStreamSynchronize(s));
      done = hk[0];
      if ((r = flush(done))) return r;
      if (hk[1]) break;
    }
    cur_step = -1;
    if ((r = enqueue_epilogue(pl, se, s, &tm))) return r;
    if ((r = flush(done))) return r;
    for (int i = 0; i < kEv; ++i) cudaEventDestroy(ev[i]);
    return SFL_OK;
  }

  // Host-driven loop (no graph): the same kernels, stop flag read after every step.
  static int run_host_loop(const Plan &pl, const Session &se, cudaStream_t s) {
    int r = enqueue_prologue(pl, se, s);
    if (r) return r;
    for (int it = 0; it < se.key.maxit; ++it) {
      if ((r = enqueue_body(pl, se, s, 0, 0))) return r;
      int stop = 0;
      SFL_CU(cudaMemcpyAsync(&stop, &se.st->stop, sizeof(int), cudaMemcpyDeviceToHost, s));
      if ((r = wait_stream(s))) return r;
      if (stop) break;
    }
    return enqueue_epilogue(pl, se, s);
  }
};

struct SolveRequest {
  int method;
  const double *b;
  bool b_host;
  const sfl_opts *o;
  double *x;
  bool x_host;
  sfl_info *info;
  cudaStream_t s;
  bool host_loop;
  sfl_kernel_times *times = nullptr;
};

static int check_opts(const Plan &pl, int method, const sfl_opts *o) {
  if (!o) return SFL_EINVAL;
  if (o->maxit < 1 || o->maxit > kMaxIt) return SFL_EINVAL;
  const bool dense = o->sketch_dense != nullptr;
  if (!dense && method != kFLSQR && (o->zeta < 1 || o->zeta > kMaxZeta)) return SFL_EINVAL;
  if (method != kFLSQR && (o->s < o->maxit + 1 || (!dense && o->s < o->zeta) || o->s > kMaxS)) return SFL_EINVAL;
  if (dense && method == kSFLSMR && !o->sketch_dense_stop) return SFL_EINVAL;
  if (o->sketch_dense_stop && (!dense || method != kSFLSMR)) return SFL_EINVAL;
  if (o->window > kMaxWindow) return SFL_EINVAL;
  if (o->window < 0 && o->orth_against_z) return SFL_EUNSUPPORTED;   // the literal z_j loop is not a projection
  if (method == kFLSQR && (o->window >= 0 || dense)) return SFL_EINVAL;
  if (o->noise_norm > 0.0 && !(o->eta > 0.0)) return SFL_EINVAL;
  if (o->precond < 0 || o->precond > SFL_PRECOND_LOWRANK) return SFL_EINVAL;
  if (o->precond == SFL_PRECOND_LOWRANK) {
    const int64_t N1 = pl.img_rows, N2 = pl.img_cols, L = (int64_t)o->lowrank_rank + o->lowrank_oversample;
    if (N1 < 1 || N2 < 1 || N1 * N2 != pl.A.cols) return SFL_EINVAL;   // the plan must know the image shape
    const int64_t Lmax = o->lowrank_fp64 ? LrLim<double>::L : LrLim<float>::L;
    if (o->lowrank_rank < 1 || o->lowrank_oversample < 0 || L > Lmax || L > std::min(N1, N2)) return SFL_EINVAL;
    if (o->lowrank_power < 0 || o->lowrank_power > 4 || !o->lowrank_omega) return SFL_EINVAL;
    if (o->orth_against_z) return SFL_EUNSUPPORTED;
  }
  if (o->precond == SFL_PRECOND_DIAG && !o->diag_w) return SFL_EINVAL;
  if (o->precond == SFL_PRECOND_REWEIGHT && !(o->irw_eps > 0.0)) return SFL_EINVAL;
  if (o->stop_rule != SFL_STOP_RULE_RESIDUAL && o->stop_rule != SFL_STOP_RULE_NORMAL) return SFL_EINVAL;
  if (o->vec_dtype == SFL_F64 && pl.vdt != SFL_F64) return SFL_EINVAL;
  if (o->vec_dtype == SFL_F32 && pl.vdt == SFL_F64) return SFL_EUNSUPPORTED;
  if (o->vec_dtype != SFL_F64 && o->vec_dtype != SFL_F32) return SFL_EINVAL;
  if (o->orth_against_z != 0 && o->orth_against_z != 1) return SFL_EINVAL;
  if (o->sketch_apply < SFL_SKETCH_APPLY_AUTO || o->sketch_apply > SFL_SKETCH_APPLY_KERNEL) return SFL_EINVAL;
  if (o->sketch_kind < SFL_SKETCH_SPARSE_SIGN || o->sketch_kind > SFL_SKETCH_GAUSSIAN) return SFL_EINVAL;
  if (o->sketch_kind != SFL_SKETCH_SPARSE_SIGN) {
    if (dense || method == kFLSQR) return SFL_EINVAL;
    if (o->sketch_kind == SFL_SKETCH_SRHT) {   // s distinct rows of the Hadamard matrix of each sketched side
      const int64_t len = method == kSFLSQR ? pl.A.rows : std::min(pl.A.rows, pl.A.cols);
      if ((int64_t)o->s > ((int64_t)1 << log2_ceil(len))) return SFL_EINVAL;
    }
  }
  return SFL_OK;
}

template <typename VT, typename XT>
static int solve_typed(Plan &pl, const SolveRequest &q) {
  using E = Engine<VT, XT>;
  const sfl_opts *o = q.o;
  SessionKey key{q.method, o->s, o->zeta, o->window, o->maxit, o->precond,
                 q.method == kSFLSMR ? o->stop_rule : 0, o->vec_dtype, o->x_history, o->relres_history,
                 o->orth_against_z, o->sketch_dense, o->sketch_dense_stop};
  if (key.dense_S) key.zeta = 1;   // the draws are not used: one session per explicit sketch
  if (q.method == kFLSQR) {         // no sketch: the small problem has maxit + 1 rows
    key.s = o->maxit + 1;
    key.zeta = 1;
    key.stop_rule = SFL_STOP_RULE_NORMAL;
    key.ell = -1;
  }
  if (key.ell < 0) key.ell = -1;
  if (o->precond == SFL_PRECOND_LOWRANK) {
    key.lr_rank = o->lowrank_rank;
    key.lr_over = o->lowrank_oversample;
    key.lr_power = o->lowrank_power;
    key.lr_fp64 = o->lowrank_fp64 ? 1 : 0;
  }
  key.sk_apply = o->sketch_apply;
  key.sk_kind = q.method == kFLSQR ? 0 : o->sketch_kind;
  if (key.sk_kind) key.zeta = 1;   // the sparse-sign draws are not used
  Session *se = nullptr;
  for (auto &p : pl.sessions)
    if (p->key == key) { se = p.get(); break; }
  int r;
  if (!se) {
    // keep a bounded number of cached sessions (history buffers change per call)
    constexpr size_t kMaxSessions = 6;
    if (pl.sessions.size() >= kMaxSessions) {
      SFL_CU(cudaStreamSynchronize(q.s));
      destroy_session(pl, *pl.sessions.front());
      pl.sessions.erase(pl.sessions.begin());
    }
    if ((r = E::create(pl, key, q.s, &se))) return r;
  }
  const int64_t m = pl.A.rows, n = pl.A.cols;
  if ((r = E::ensure_tables(pl, *se, o->seed, q.s))) return r;
  SFL_CU(cudaMemcpyAsync(se->bbuf, q.b, sizeof(double) * m, q.b_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                         q.s));
  if (o->precond == SFL_PRECOND_DIAG)
    SFL_CU(cudaMemcpyAsync(se->dw, o->diag_w, sizeof(double) * n, cudaMemcpyDeviceToDevice, q.s));
  if (se->lowrank) {   // the caller's FP64 test matrix in the truncation's arithmetic
    const int64_t no = (int64_t)pl.img_cols * (o->lowrank_rank + o->lowrank_oversample);
    const unsigned g = (unsigned)std::min<int64_t>((no + kThreads - 1) / kThreads, 1024);
    if (se->key.lr_fp64) lr_omega_kernel<double><<<g, kThreads, 0, q.s>>>(o->lowrank_omega, (double *)se->lr64.Omega, no);
    else lr_omega_kernel<float><<<g, kThreads, 0, q.s>>>(o->lowrank_omega, (float *)se->lr32.Omega, no);
    SFL_CU(cudaGetLastError());
  }
  reset_state_kernel<<<1, 1, 0, q.s>>>(se->st, o->seed, o->eta, o->noise_norm, o->irw_eps);
  SFL_CU(cudaGetLastError());
  if (q.times) {
    memset(q.times, 0, sizeof(*q.times));
    if ((r = E::run_profiled(pl, *se, q.s, q.times))) return r;
  } else if (q.host_loop) {
    if ((r = E::run_host_loop(pl, *se, q.s))) return r;
  } else {
    SFL_CU(cudaGraphLaunch(se->exec, q.s));
  }
  SFL_CU(cudaMemcpyAsync(q.x, se->xbuf, sizeof(double) * n, q.x_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                         q.s));
  if (q.info || q.x_host) {
    if ((r = wait_stream(q.s))) return r;
    SolveState h;
    SFL_CU(cudaMemcpy(&h, se->st, sizeof(SolveState), cudaMemcpyDeviceToHost));
    int err = 0;
    SFL_CU(cudaMemcpy(&err, se->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) return SFL_ECUDA;
    if (q.info) {
      q.info->iters = h.k;
      q.info->status = h.stop == kStopNonfinite ? SFL_STOP_BREAKDOWN : h.stop;
      q.info->relres = h.relres;
      q.info->tol = h.tol;
    }
    if (h.stop == kStopNonfinite) return SFL_ENONFINITE;
  }
  return SFL_OK;
}

static int solve(sfl_plan *plan, const SolveRequest &q) {
  if (!plan || !q.b || !q.x) return SFL_EINVAL;
  Plan &pl = plan->impl;
  int r = check_opts(pl, q.method, q.o);
  if (r) return r;
  if (pl.vdt == SFL_F64) return solve_typed<double, double>(pl, q);
  if (pl.vdt == SFL_F32) return solve_typed<float, float>(pl, q);
  return solve_typed<__nv_bfloat16, float>(pl, q);
}

template <typename VT, typename XT>
static int apply_typed(Plan &pl, int which, const double *x, double *y, cudaStream_t s) {
  const StoredCsr &M = which == 0 ? pl.A : pl.T;
  SpmvParams<VT, XT> p{};
  p.rowptr = M.rowptr; p.col = M.col; p.val = (const VT *)M.val; p.rows = M.rows;
  p.dcol = M.dcol; p.rbase = M.rbase;
  p.orig = M.orig;
  p.mode = kModeApply;
  const int grid = pl.num_sms * 2;
  p.interleave = interleave_rows(M, grid);
  if (!pl.matfree) {   // warp row ranges balanced by row cost, as in a solve (first call per operator)
    if (!pl.apply_wrow[which]) {
      const int W = grid * kWarps;
      int32_t *wrow = nullptr;
      SFL_CU(cudaMalloc(&wrow, sizeof(int32_t) * (W + 1)));
      pl.allocs.push_back(wrow);
      const bool fp64 = std::is_same<VT, double>::value;
      const int P = load_width(pl.vdt);
      const int r = balance_rows(M, SpmvTune<VT>::NCH * M.lpr * P, W, wrow, s, fp64 ? M.lpr * P : 0, 0);
      if (r) return r;
      pl.apply_wrow[which] = wrow;
    }
    p.wrow = pl.apply_wrow[which];
  }
  if (pl.matfree) {
    p.ptab = pl.ct_tab;
    p.pfix = pl.ct_fix;
    p.pN = pl.ct_N; p.pna = pl.ct_na; p.pnb = pl.ct_nb;
    p.proj = which == 0 ? kProjRay : (pl.ct_back ? kProjBackLinear : kProjBackChord);
  }
  const size_t smem = spmv_smem_bytes(M.lpr, sizeof(typename AccT<XT>::T));
  SFL_CU(Ops<VT, XT>::set_smem(M.lpr, true, kSpmvSmemLimit));
  if (std::is_same<XT, double>::value) {
    p.x = (const XT *)x; p.y = (XT *)y;
    SFL_CU(Ops<VT, XT>::spmv(p, M.lpr, true, grid, smem, s));
    return SFL_OK;
  }
  if (!pl.apply_x) {
    const int64_t len = std::max(pl.A.rows, pl.A.cols);
    SFL_CU(cudaMalloc(&pl.apply_x, sizeof(XT) * len));
    SFL_CU(cudaMalloc(&pl.apply_y, sizeof(XT) * len));
    pl.allocs.push_back(pl.apply_x);
    pl.allocs.push_back(pl.apply_y);
  }
  SFL_CU(Ops<VT, XT>::convert_in(x, (XT *)pl.apply_x, M.cols, s));
  p.x = (const XT *)pl.apply_x; p.y = (XT *)pl.apply_y;
  SFL_CU(Ops<VT, XT>::spmv(p, M.lpr, true, grid, smem, s));
  SFL_CU(Ops<VT, XT>::convert_out((const XT *)pl.apply_y, y, M.rows, s));
  return SFL_OK;
}

}  // namespace sfl

using namespace sfl;

extern "C" {

int sfl_plan_destroy(sfl_plan *plan) {
  if (!plan) return SFL_EINVAL;
  Plan &pl = plan->impl;
  cudaDeviceSynchronize();
  for (auto &se : pl.sessions) destroy_session(pl, *se);
  pl.sessions.clear();
  pl.batches.clear();
  for (void *p : pl.allocs) cudaFree(p);
  pl.allocs.clear();
  delete plan;
  return SFL_OK;
}

int sfl_plan_apply(sfl_plan *plan, int which, const double *x, double *y, sfl_stream stream) {
  if (!plan || !x || !y || (which != 0 && which != 1)) return SFL_EINVAL;
  Plan &pl = plan->impl;
  cudaStream_t s = (cudaStream_t)stream;
  if (pl.vdt == SFL_F64) return apply_typed<double, double>(pl, which, x, y, s);
  if (pl.vdt == SFL_F32) return apply_typed<float, float>(pl, which, x, y, s);
  return apply_typed<__nv_bfloat16, float>(pl, which, x, y, s);
}

int sflsqr_solve(sfl_plan *plan, const double *b, const sfl_opts *opts, double *x, sfl_info *info, sfl_stream stream) {
  return solve(plan, SolveRequest{kSFLSQR, b, false, opts, x, false, info, (cudaStream_t)stream, false});
}
int sflsmr_solve(sfl_plan *plan, const double *b, const sfl_opts *opts, double *x, sfl_info *info, sfl_stream stream) {
  return solve(plan, SolveRequest{kSFLSMR, b, false, opts, x, false, info, (cudaStream_t)stream, false});
}
int sflsqr_solve_host(sfl_plan *plan, const double *b, const sfl_opts *opts, double *x, sfl_info *info,
                      sfl_stream stream) {
  return solve(plan, SolveRequest{kSFLSQR, b, true, opts, x, true, info, (cudaStream_t)stream, false});
}
int sflsmr_solve_host(sfl_plan *plan, const double *b, const sfl_opts *opts, double *x, sfl_info *info,
                      sfl_stream stream) {
  return solve(plan, SolveRequest{kSFLSMR, b, true, opts, x, true, info, (cudaStream_t)stream, false});
}
int flsqr_solve(sfl_plan *plan, const double *b, const sfl_opts *opts, double *x, sfl_info *info, sfl_stream stream) {
  return solve(plan, SolveRequest{kFLSQR, b, false, opts, x, false, info, (cudaStream_t)stream, false});
}
int flsqr_solve_host(sfl_plan *plan, const double *b, const sfl_opts *opts, double *x, sfl_info *info,
                     sfl_stream stream) {
  return solve(plan, SolveRequest{kFLSQR, b, true, opts, x, true, info, (cudaStream_t)stream, false});
}

// Same solve driven by a host loop instead of the graph's WHILE node (one
// stream synchronisation per step); used to check that both drivers agree.
int sfl_solve_host_loop(sfl_plan *plan, int method, const double *b, const sfl_opts *opts, double *x, sfl_info *info,
                        sfl_stream stream) {
  if (method != kSFLSQR && method != kSFLSMR && method != kFLSQR) return SFL_EINVAL;
  return solve(plan, SolveRequest{method, b, false, opts, x, false, info, (cudaStream_t)stream, true});
}

int sfl_solve_profiled(sfl_plan *plan, int method, const double *b, const sfl_opts *opts, double *x, sfl_info *info,
                       sfl_kernel_times *times, sfl_stream stream) {
  if (method != kSFLSQR && method != kSFLSMR && method != kFLSQR) return SFL_EINVAL;
  if (!times) return SFL_EINVAL;
  SolveRequest q{method, b, false, opts, x, false, info, (cudaStream_t)stream, true};
  q.times = times;
  return solve(plan, q);
}

int sfl_sketch_export(uint64_t seed, int32_t s, int32_t zeta, int64_t ncols, int32_t *rows, int32_t *signs,
                      sfl_stream stream) {
  if (!rows || !signs || zeta < 1 || zeta > kMaxZeta || s < zeta || s > 32768 || ncols < 0) return SFL_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int *err = nullptr;
  SFL_CU(cudaMalloc(&err, sizeof(int)));
  cudaMemsetAsync(err, 0, sizeof(int), st);
  if (ncols > 0)
    sketch_table_kernel<<<(unsigned)((ncols + 255) / 256), 256, 0, st>>>(seed, nullptr, 0, s, zeta, ncols, zeta,
                                                                          nullptr, rows, signs, err);
  int h = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(err);
  if (e != cudaSuccess) { set_cuda_error(e, "sfl_sketch_export"); return SFL_ECUDA; }
  return h ? SFL_EINVAL : SFL_OK;
}

int sfl_sketch_apply(uint64_t seed, int32_t s, int32_t zeta, const double *v, int64_t len, double *sk,
                     sfl_stream stream) {
  if (!v || !sk || zeta < 1 || zeta > kMaxZeta || s < zeta || s > kMaxS || len < 1) return SFL_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nent = len * zeta;
  SketchTableTmp t;
  int32_t *row = nullptr;
  uint32_t *ent = nullptr;
  int *err = nullptr;
  int r = SFL_OK;
  t.cub_bytes = sketch_sort_bytes(nent, s) + 256;
  if (cudaMalloc(&t.kin, 4 * nent) != cudaSuccess || cudaMalloc(&t.vin, 4 * nent) != cudaSuccess ||
      cudaMalloc(&t.kout, 4 * nent) != cudaSuccess || cudaMalloc(&t.cub, t.cub_bytes) != cudaSuccess ||
      cudaMalloc(&row, 4 * (s + 1)) != cudaSuccess || cudaMalloc(&ent, 4 * nent) != cudaSuccess ||
      cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    r = SFL_ENOMEM;
  }
  if (!r) {
    cudaMemsetAsync(err, 0, sizeof(int), st);
    r = build_sketch_table(seed, s, zeta, len, row, ent, t, err, st);
  }
  if (!r) {
    SketchParams<double> p{};
    p.mode = kSkPlain; p.s = s; p.isz = 1.0 / std::sqrt((double)zeta); p.v64 = v; p.rowM = row; p.entM = ent; p.sk_out = sk;
    sketch_rows_kernel<double><<<s, kSkWarps * 32, 0, st>>>(p, s);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) r = SFL_ECUDA;
    int h = 0;
    if (!r && cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && h) r = SFL_EINVAL;
  }
  if (r == SFL_ECUDA) set_cuda_error(cudaGetLastError(), "sfl_sketch_apply");
  cudaFree(t.kin); cudaFree(t.vin); cudaFree(t.kout); cudaFree(t.cub); cudaFree(row); cudaFree(ent); cudaFree(err);
  return r;
}

}  // extern "C"
