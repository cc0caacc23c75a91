// Batched sFLSQR engine and its C entry point (sflsqr_solve_batched).
//
// One CUDA graph per batch configuration: a prologue (state reset, ||b_r||,
// interleave b, A^T w_1 for all RHS, S_m b), a WHILE node whose body is one
// step for every running RHS, and an epilogue writing x_r.  The SpMM tile
// width (RHS per CTA column) is chosen per product by timing the candidates
// when the session is created; results do not depend on the choice.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "adjoint.cuh"
#include "engine.h"

namespace sfl {

constexpr int kBMaxRowCtas = 2048;

struct BatchKey {
  int R, s, zeta, ell, maxit, precond, keep_what, tile;   // tile: forced SpMM width, 0 = tuned
  double *x_hist;                                          // x_k of every RHS after every step, or null
  bool operator==(const BatchKey &o) const {
    return R == o.R && s == o.s && zeta == o.zeta && ell == o.ell && maxit == o.maxit && precond == o.precond &&
           keep_what == o.keep_what && tile == o.tile && x_hist == o.x_hist;
  }
};

template <typename VT, typename XT>
struct BatchSession : BatchSessionBase {
  BatchKey key{};
  int ld = 0;
  BParams<XT> bp{};
  double *noise = nullptr, *B = nullptr, *X = nullptr, *dwbuf = nullptr;
  double *Q = nullptr, *Rinv = nullptr, *y = nullptr;
  int32_t *wrowA = nullptr, *wrowT = nullptr, *err = nullptr;
  int32_t *skrow = nullptr;
  uint32_t *skent = nullptr, *kin = nullptr, *vin = nullptr, *kout = nullptr;
  void *cub = nullptr;
  size_t cub_bytes = 0;
  bool tab_valid = false;
  uint64_t tab_seed = 0;
  int G_orth = 0, G_rows = 0, tileA = 32, tileT = 32, ls_cluster = 1, ls_stage = 0;
  size_t smem_ls = 0;
  float tune_ms[2][4] = {};
  // adjoint workspace (allocated by the first adjoint call)
  bool adj_ready = false;
  XT *a_xbar = nullptr, *a_wbar = nullptr, *a_pbar = nullptr, *a_whatbar = nullptr, *a_tbar = nullptr, *a_u = nullptr,
     *a_stm = nullptr, *a_tmpA = nullptr, *a_tmpB = nullptr;
  double *a_dacc = nullptr, *a_rec = nullptr, *a_coef = nullptr, *a_ybar = nullptr, *a_sbar = nullptr,
         *a_Mbar = nullptr, *a_ones = nullptr;
  int *a_kr = nullptr;
  const double *dw_in = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void *> allocs;
  uint64_t bytes = 0;
  Plan *plan = nullptr;
  ~BatchSession() override {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (void *p : allocs) cudaFree(p);
    if (plan) plan->bytes -= bytes;
  }
};

template <typename VT, typename XT>
struct BEngine {
  using S = BatchSession<VT, XT>;

  static int alloc(S &se, void **p, size_t bytes) {
    Plan &pl = *se.plan;
    if (pl.cap && pl.bytes + bytes > pl.cap) return SFL_ENOMEM;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_cuda_error(e, "cudaMalloc");
      return SFL_ENOMEM;
    }
    se.allocs.push_back(*p);
    se.bytes += bytes;
    pl.bytes += bytes;
    return SFL_OK;
  }

  template <int T>
  static const void *spmm_fn_t(bool orig, bool ilv) {
    if (orig && ilv) return (const void *)bspmm_kernel<VT, XT, T, true, true>;
    if (orig) return (const void *)bspmm_kernel<VT, XT, T, true, false>;
    if (ilv) return (const void *)bspmm_kernel<VT, XT, T, false, true>;
    return (const void *)bspmm_kernel<VT, XT, T, false, false>;
  }
  static const void *spmm_fn(int T, bool orig, bool ilv) {
    return T == 8 ? spmm_fn_t<8>(orig, ilv) : T == 16 ? spmm_fn_t<16>(orig, ilv)
                  : T == 32 ? spmm_fn_t<32>(orig, ilv) : spmm_fn_t<64>(orig, ilv);
  }

  // the instance for the plan's row order (ORIG) and slot layout (ILV)
  template <int T>
  static void launch_spmm(const S &se, const StoredCsr &M, BSpmmArgs &a, dim3 grid, cudaStream_t s) {
    a.orig = M.orig;
    a.slot = M.lpr * load_width(se.plan->vdt);
    if (M.orig && M.interleaved) bspmm_kernel<VT, XT, T, true, true><<<grid, kThreads, 0, s>>>(se.bp, a);
    else if (M.orig) bspmm_kernel<VT, XT, T, true, false><<<grid, kThreads, 0, s>>>(se.bp, a);
    else if (M.interleaved) bspmm_kernel<VT, XT, T, false, true><<<grid, kThreads, 0, s>>>(se.bp, a);
    else bspmm_kernel<VT, XT, T, false, false><<<grid, kThreads, 0, s>>>(se.bp, a);
  }

  template <int T>
  static cudaError_t spmm_t(const S &se, const StoredCsr &M, const int32_t *wrow, int mode, cudaStream_t s) {
    BSpmmArgs a{M.rowptr, M.col, M.val, M.rows, wrow, mode};
    dim3 grid(se.G_rows, (se.key.R + T - 1) / T);
    launch_spmm<T>(se, M, a, grid, s);
    return cudaGetLastError();
  }
  static cudaError_t spmm(const S &se, int mode, cudaStream_t s) {
    const bool fwd = mode == kBSpmmFwd;
    const StoredCsr &M = fwd ? se.plan->A : se.plan->T;
    const int32_t *wrow = fwd ? se.wrowA : se.wrowT;
    switch (fwd ? se.tileA : se.tileT) {
      case 8: return spmm_t<8>(se, M, wrow, mode, s);
      case 16: return spmm_t<16>(se, M, wrow, mode, s);
      case 32: return spmm_t<32>(se, M, wrow, mode, s);
      default: return spmm_t<64>(se, M, wrow, mode, s);
    }
  }
  static cudaError_t scal(const S &se, int mode, int G, cudaStream_t s) {
    bscal_kernel<XT><<<(se.key.R + kWarps - 1) / kWarps, kThreads, 0, s>>>(se.bp, mode, G);
    return cudaGetLastError();
  }
  static cudaError_t orth(const S &se, int side, cudaStream_t s) {
    borth_kernel<XT><<<se.G_orth, kThreads, 0, s>>>(se.bp, side);
    return cudaGetLastError();
  }
  static cudaError_t sketch(const S &se, int mode, cudaStream_t s) {
    dim3 grid(se.key.s, (se.key.R + 31) / 32);
    bsketch_kernel<XT><<<grid, kBSkWarps * 32, 0, s>>>(se.bp, mode, se.B);
    return cudaGetLastError();
  }
  static LsParams ls_params(const S &se) {
    LsParams q{};
    q.st = se.bp.st; q.method = kSFLSQR; q.s = se.key.s; q.maxit = se.key.maxit; q.ell = se.key.ell;
    q.stop_rule = SFL_STOP_RULE_RESIDUAL;
    q.stage_q = se.ls_stage & 1;
    q.stage_saz = 0;
    q.Q = se.Q; q.Rinv = se.Rinv; q.y = se.y; q.e = se.bp.e;
    q.SAZ = se.bp.SAZ; q.SAtW = nullptr; q.Hband = nullptr; q.sbm = nullptr; q.rhs = se.bp.rhs;
    q.relres_hist = nullptr;
    q.use_cond = 0;
    const int64_t sk = se.key.s, K = se.key.maxit;
    q.bQ = sk * K; q.bRinv = K * K; q.by = K; q.be = sk; q.bSAZ = sk * K; q.bSAtW = 0; q.bHband = 0;
    q.bvec = sk; q.bhist = 0;
    return q;
  }

  // prologue after the reset kernel (which the solve call launches with its options)
  static int enqueue_init(const S &se, cudaStream_t s) {
    const int R = se.key.R;
    binit_norm_kernel<XT><<<R, kThreads, 0, s>>>(se.bp, se.B);
    SFL_CU(cudaGetLastError());
    dim3 tg((unsigned)((se.bp.m + 31) / 32), (se.ld + 31) / 32), tb(32, 8);
    binterleave_kernel<XT><<<tg, tb, 0, s>>>(se.B, se.bp.m, R, se.ld, se.bp.W);
    SFL_CU(cudaGetLastError());
    SFL_CU(spmm(se, kBSpmmInit, s));
    SFL_CU(sketch(se, 1, s));
    return SFL_OK;
  }

  static int enqueue_body(const S &se, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond) {
    SFL_CU(scal(se, kBScalZ, se.G_rows, s));
    SFL_CU(orth(se, 0, s));
    SFL_CU(scal(se, kBScalAlpha, se.G_orth, s));
    SFL_CU(spmm(se, kBSpmmFwd, s));
    SFL_CU(scal(se, kBScalW, se.G_rows, s));
    SFL_CU(orth(se, 1, s));
    SFL_CU(scal(se, kBScalBeta, se.G_orth, s));
    SFL_CU(spmm(se, kBSpmmBwd, s));
    SFL_CU(sketch(se, 0, s));
    SFL_CU(launch_ls(ls_params(se), se.ls_cluster, se.smem_ls, s, false, se.key.R));
    if (se.key.x_hist) {   // x_k of the right-hand sides that completed step k (before the step counter moves)
      dim3 tg((unsigned)((se.bp.n + 31) / 32), (se.key.R + 31) / 32), tb(32, 8);
      bsolution_kernel<XT><<<tg, tb, 0, s>>>(se.bp, se.y, se.key.x_hist, 1);
      SFL_CU(cudaGetLastError());
    }
    bcond_kernel<XT><<<1, 256, 0, s>>>(se.bp, h, use_cond);
    SFL_CU(cudaGetLastError());
    return SFL_OK;
  }

  static int enqueue_epilogue(const S &se, cudaStream_t s) {
    dim3 tg((unsigned)((se.bp.n + 31) / 32), (se.key.R + 31) / 32), tb(32, 8);
    bsolution_kernel<XT><<<tg, tb, 0, s>>>(se.bp, se.y, se.X, 0);
    SFL_CU(cudaGetLastError());
    return SFL_OK;
  }

  static int build_graph(S &se) {
    cudaStream_t cs;
    SFL_CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    int r = SFL_OK;
    cudaGraph_t g = nullptr, gp = nullptr, ge = nullptr;
    do {
      if (cudaGraphCreate(&g, 0) != cudaSuccess) { r = SFL_ECUDA; break; }
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { r = SFL_ECUDA; break; }
      r = enqueue_init(se, cs);
      if (cudaStreamEndCapture(cs, &gp) != cudaSuccess || r) { r = r ? r : SFL_ECUDA; break; }
      cudaGraphNode_t np, nw, ne;
      if (cudaGraphAddChildGraphNode(&np, g, nullptr, 0, gp) != cudaSuccess) { r = SFL_ECUDA; break; }
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
      r = enqueue_body(se, cs, h, 1);
      cudaGraph_t body_out = body;
      if (cudaStreamEndCapture(cs, &body_out) != cudaSuccess || r) { r = r ? r : SFL_ECUDA; break; }
      if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { r = SFL_ECUDA; break; }
      r = enqueue_epilogue(se, cs);
      if (cudaStreamEndCapture(cs, &ge) != cudaSuccess || r) { r = r ? r : SFL_ECUDA; break; }
      if (cudaGraphAddChildGraphNode(&ne, g, &nw, 1, ge) != cudaSuccess) { r = SFL_ECUDA; break; }
      cudaError_t e = cudaGraphInstantiate(&se.exec, g, 0);
      if (e != cudaSuccess) { set_cuda_error(e, "cudaGraphInstantiate"); r = SFL_ECUDA; break; }
      se.graph = g;
      g = nullptr;
    } while (0);
    if (r == SFL_ECUDA) {
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) set_cuda_error(e, "batched graph build");
    }
    if (g) cudaGraphDestroy(g);
    if (gp) cudaGraphDestroy(gp);
    if (ge) cudaGraphDestroy(ge);
    cudaStreamDestroy(cs);
    return r;
  }

  // SpMM tile width per product: time each candidate on this operator (the
  // results are identical for every width; only the speed differs).
  static int tune(S &se, cudaStream_t s) {
    const int cands[4] = {8, 16, 32, 64};
    cudaEvent_t e0, e1;
    SFL_CU(cudaEventCreate(&e0));
    SFL_CU(cudaEventCreate(&e1));
    int best[2] = {32, 32};
    for (int which = 0; which < 2; ++which) {
      float bt = 1e30f;
      for (int ci = 0; ci < 4; ++ci) {
        const int T = cands[ci];
        if ((T > se.ld && T > 8) || (T < 32 && se.ld >= 32 && T * 2 < se.ld)) continue;   // widths for this batch
        if (which == 0) se.tileA = T; else se.tileT = T;
        const int mode = which == 0 ? kBSpmmFwd : kBSpmmBwd;
        SFL_CU(spmm(se, mode, s));   // warm-up
        SFL_CU(cudaEventRecord(e0, s));
        for (int rep = 0; rep < 3; ++rep) SFL_CU(spmm(se, mode, s));
        SFL_CU(cudaEventRecord(e1, s));
        SFL_CU(cudaEventSynchronize(e1));
        float ms = 0.f;
        SFL_CU(cudaEventElapsedTime(&ms, e0, e1));
        se.tune_ms[which][ci] = ms / 3;
        if (ms < bt) { bt = ms; best[which] = T; }
      }
    }
    se.tileA = best[0];
    se.tileT = best[1];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return SFL_OK;
  }

  static int create(Plan &pl, const BatchKey &key, cudaStream_t s, S **out) {
    auto se = std::make_unique<S>();
    se->plan = &pl;
    se->key = key;
    const int R = key.R;
    int ld = 4;
    while (ld < R) ld <<= 1;
    se->ld = ld;
    const int64_t m = pl.A.rows, n = pl.A.cols;
    const int K = key.maxit, Sk = key.s, ell = key.ell;
    const size_t xs = sizeof(XT);
    BParams<XT> &b = se->bp;
    b.R = R; b.ld = ld; b.m = m; b.n = n; b.ell = ell; b.maxit = K; b.s = Sk;
    b.RW = ell + 2; b.RP = ell + 1;
    b.keep_what = key.keep_what;
    b.isz = 1.0 / std::sqrt((double)key.zeta);
    se->G_orth = pl.num_sms * 2;
    // row CTAs: as many as stay resident for every tile width (the records and
    // the row partition depend on it, so it is one number per session)
    int occ = 8;
    for (const StoredCsr *M : {&pl.A, &pl.T})
      for (int T : {8, 16, 32, 64}) {
        int nb = 0;
        SFL_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, spmm_fn(T, M->orig != nullptr, M->interleaved),
                                                             kThreads, 0));
        occ = std::min(occ, std::max(nb, 1));
      }
    se->G_rows = std::min(pl.num_sms * occ, kBMaxRowCtas);
    se->bp.rcap = std::max(se->G_orth, se->G_rows);
    int r;
#define BA(ptr, bytes) if ((r = alloc(*se, (void **)&(ptr), (bytes)))) return r;
    BA(b.kstep, sizeof(int));
    BA(b.st, sizeof(SolveState) * R);
    BA(b.W, xs * (size_t)(K + 1) * m * ld);
    BA(b.P, xs * (size_t)K * n * ld);
    BA(b.zbuf, xs * (size_t)n * ld);
    BA(b.what, xs * (size_t)(key.keep_what ? K : 1) * m * ld);
    BA(b.zraw, xs * (size_t)n * ld);
    BA(b.sigW, sizeof(double) * R * (K + 2));
    BA(b.sigP, sizeof(double) * R * (K + 1));
    BA(b.coef, sizeof(double) * R * (kMaxWindow + 2));
    BA(b.rawscale, sizeof(double) * R);
    BA(b.hband, sizeof(double) * (size_t)R * K * (ell + 2));
    BA(b.tband, sizeof(double) * (size_t)R * K * (ell + 1));
    BA(b.rec, sizeof(double) * (size_t)(kMaxWindow + 2) * R * se->bp.rcap);
    BA(b.SAZ, sizeof(double) * (size_t)R * K * Sk);
    BA(b.rhs, sizeof(double) * (size_t)R * Sk);
    BA(b.e, sizeof(double) * (size_t)R * Sk);
    BA(se->Q, sizeof(double) * (size_t)R * Sk * K);
    BA(se->Rinv, sizeof(double) * (size_t)R * K * K);
    BA(se->y, sizeof(double) * (size_t)R * K);
    BA(se->noise, sizeof(double) * R);
    BA(se->B, sizeof(double) * (size_t)R * m);
    BA(se->X, sizeof(double) * (size_t)R * n);
    if (key.precond == SFL_PRECOND_DIAG) BA(se->dwbuf, sizeof(double) * n);
    BA(se->err, sizeof(int));
    BA(se->skrow, sizeof(int32_t) * (Sk + 1));
    BA(se->skent, sizeof(uint32_t) * (size_t)key.zeta * m);
    const int64_t nent = (int64_t)key.zeta * m;
    BA(se->kin, sizeof(uint32_t) * nent);
    BA(se->vin, sizeof(uint32_t) * nent);
    BA(se->kout, sizeof(uint32_t) * nent);
    se->cub_bytes = sketch_sort_bytes(nent, Sk) + 256;
    BA(se->cub, se->cub_bytes);
    BA(se->wrowA, sizeof(int32_t) * (se->G_rows + 1));
    BA(se->wrowT, sizeof(int32_t) * (se->G_rows + 1));
#undef BA
    b.dw = se->dwbuf;
    b.skrow = se->skrow; b.skent = se->skent;
    // SpMM rows per CTA (its warps interleave them): a row costs its chunks
    const int P = load_width(pl.vdt);
    if ((r = balance_rows(pl.A, P, se->G_rows, se->wrowA, s))) return r;
    if ((r = balance_rows(pl.T, P, se->G_rows, se->wrowT, s))) return r;
    // small problems: one cluster per RHS, as many SMs each as the batch leaves
    int maxc = 1;
    while (maxc * 2 * R <= pl.num_sms && maxc < 16) maxc <<= 1;
    se->ls_cluster = ls_cluster_size(Sk, K, false, maxc);
    if (se->ls_cluster < 1) return SFL_EUNSUPPORTED;
    se->smem_ls = ls_smem_bytes(Sk, K, se->ls_cluster, false);
    se->ls_stage = ls_stage_plan(Sk, K, se->ls_cluster, false);
    SFL_CU(ls_allow_max_smem());
    // tuning runs on a reset state with zero vectors
    SFL_CU(cudaMemsetAsync(se->noise, 0, sizeof(double) * R, s));
    SFL_CU(cudaMemsetAsync(b.W, 0, xs * (size_t)(K + 1) * m * ld, s));
    SFL_CU(cudaMemsetAsync(b.zbuf, 0, xs * (size_t)n * ld, s));
    SFL_CU(cudaMemsetAsync(b.P, 0, xs * (size_t)K * n * ld, s));
    SFL_CU(cudaMemsetAsync(se->err, 0, sizeof(int), s));
    breset_kernel<XT><<<(R + 255) / 256, 256, 0, s>>>(b, 0, 0.0, se->noise, 0.0);
    SFL_CU(cudaGetLastError());
    if (key.tile) { se->tileA = se->tileT = key.tile; }
    else if ((r = tune(*se, s))) return r;
    SFL_CU(cudaStreamSynchronize(s));
    if ((r = build_graph(*se))) return r;
    *out = se.get();
    pl.batches.push_back(std::move(se));
    return SFL_OK;
  }

  static int ensure_table(S &se, uint64_t seed, cudaStream_t s) {
    if (se.tab_valid && se.tab_seed == seed) return SFL_OK;
    SketchTableTmp t;
    t.kin = se.kin; t.vin = se.vin; t.kout = se.kout; t.cub = se.cub; t.cub_bytes = se.cub_bytes;
    // the m-side sketch of sFLSQR uses the solve's seed (as the single solve)
    int r = build_sketch_table(seed, se.key.s, se.key.zeta, se.plan->A.rows, se.skrow, se.skent, t, se.err, s);
    if (r) return r;
    se.tab_valid = true;
    se.tab_seed = seed;
    return SFL_OK;
  }

  static int solve(Plan &pl, int R, const double *B, const double *noise, const sfl_opts *o, double *X, sfl_info *infos,
                   cudaStream_t s, int keep_what, S **used) {
    BatchKey key{R, o->s, o->zeta, o->window, o->maxit, o->precond, keep_what, o->spmm_tile,
                 keep_what ? nullptr : o->x_history};
    S *se = nullptr;
    for (auto &p : pl.batches) {
      S *q = dynamic_cast<S *>(p.get());
      if (q && q->key == key) { se = q; break; }
    }
    int r;
    if (!se) {
      if (pl.batches.size() >= 2) {
        SFL_CU(cudaStreamSynchronize(s));
        size_t victim = 0;
        if (pl.batches[0].get() == pl.last_fixed && !keep_what) victim = 1;   // keep a fixed forward for its adjoint
        if (pl.batches[victim].get() == pl.last_fixed) pl.last_fixed = nullptr;
        pl.batches.erase(pl.batches.begin() + victim);
      }
      if ((r = create(pl, key, s, &se))) return r;
    }
    if ((r = ensure_table(*se, o->seed, s))) return r;
    const int64_t m = pl.A.rows, n = pl.A.cols;
    SFL_CU(cudaMemcpyAsync(se->B, B, sizeof(double) * (size_t)R * m, cudaMemcpyDeviceToDevice, s));
    SFL_CU(cudaMemcpyAsync(se->noise, noise, sizeof(double) * R, cudaMemcpyHostToDevice, s));
    if (o->precond == SFL_PRECOND_DIAG)
      SFL_CU(cudaMemcpyAsync(se->dwbuf, o->diag_w, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    breset_kernel<XT><<<(R + 255) / 256, 256, 0, s>>>(se->bp, o->seed, o->eta, se->noise, 0.0);
    SFL_CU(cudaGetLastError());
    SFL_CU(cudaGraphLaunch(se->exec, s));
    SFL_CU(cudaMemcpyAsync(X, se->X, sizeof(double) * (size_t)R * n, cudaMemcpyDeviceToDevice, s));
    if (used) *used = se;
    if (infos) {
      if ((r = wait_stream(s))) return r;
      std::vector<SolveState> h(R);
      SFL_CU(cudaMemcpy(h.data(), se->bp.st, sizeof(SolveState) * R, cudaMemcpyDeviceToHost));
      int err = 0;
      SFL_CU(cudaMemcpy(&err, se->err, sizeof(int), cudaMemcpyDeviceToHost));
      if (err) return SFL_ECUDA;
      bool nonfinite = false;
      for (int j = 0; j < R; ++j) {
        infos[j].iters = h[j].k;
        infos[j].status = h[j].stop == kStopNonfinite ? SFL_STOP_BREAKDOWN : h[j].stop;
        infos[j].relres = h[j].relres;
        infos[j].tol = h[j].tol;
        nonfinite |= h[j].stop == kStopNonfinite;
      }
      if (nonfinite) return SFL_ENONFINITE;
    }
    return SFL_OK;
  }
};

// Reverse sweep of a fixed-k forward kept in a batch session (see adjoint.cuh).
template <typename VT, typename XT>
struct AEngine {
  using S = BatchSession<VT, XT>;
  using E = BEngine<VT, XT>;

  static int workspace(S &se) {
    if (se.adj_ready) return SFL_OK;
    const int R = se.key.R, ld = se.ld, K = se.key.maxit, Sk = se.key.s, L = se.key.ell;
    const int64_t m = se.bp.m, n = se.bp.n;
    const size_t xs = sizeof(XT);
    int r;
#define AA(ptr, bytes) if ((r = E::alloc(se, (void **)&(ptr), (bytes)))) return r;
    AA(se.a_xbar, xs * n * ld);
    AA(se.a_wbar, xs * (size_t)(L + 2) * m * ld);
    AA(se.a_pbar, xs * (size_t)(L + 1) * n * ld);
    AA(se.a_whatbar, xs * m * ld);
    AA(se.a_tbar, xs * n * ld);
    AA(se.a_u, xs * n * ld);
    AA(se.a_stm, xs * m * ld);
    AA(se.a_tmpA, xs * m * ld);
    AA(se.a_tmpB, xs * m * ld);
    AA(se.a_dacc, sizeof(double) * n * ld);
    AA(se.a_rec, sizeof(double) * (size_t)kAdjNQ * R * se.bp.rcap);
    AA(se.a_coef, sizeof(double) * (size_t)R * kAdjNO * kAdjNV);
    AA(se.a_ybar, sizeof(double) * (size_t)R * K);
    AA(se.a_sbar, sizeof(double) * (size_t)R * Sk);
    AA(se.a_Mbar, sizeof(double) * (size_t)R * K * Sk);
    AA(se.a_ones, sizeof(double) * n);
    AA(se.a_kr, sizeof(int) * R);
#undef AA
    se.adj_ready = true;
    return SFL_OK;
  }

  static AVec vec(const void *p, const double *scale = nullptr, int64_t sstride = 0, int dmul = 0, int dbl = 0) {
    AVec v;
    v.p = p; v.dbl = dbl; v.scale = scale; v.sstride = sstride; v.dmul = dmul;
    return v;
  }

  static AArgs args(const S &se, int64_t len, int j) {
    AArgs a{};
    a.R = se.key.R; a.ld = se.ld; a.len = len; a.kr = se.a_kr; a.jstep = j;
    a.d = se.dwbuf ? se.dwbuf : se.a_ones;
    a.coef = se.a_coef; a.rec = se.a_rec; a.rcap = se.bp.rcap;
    return a;
  }

  static AScalArgs sargs(const S &se, int mode, int j, int nv) {
    AScalArgs s{};
    s.R = se.key.R; s.maxit = se.key.maxit; s.ell = se.key.ell; s.j = j; s.mode = mode; s.G = se.G_orth; s.nv = nv;
    s.kr = se.a_kr; s.rec = se.a_rec; s.rcap = se.bp.rcap;
    s.sigW = se.bp.sigW; s.sigP = se.bp.sigP; s.hband = se.bp.hband; s.tband = se.bp.tband; s.st = se.bp.st;
    s.coef = se.a_coef; s.ybar = se.a_ybar;
    return s;
  }

  static cudaError_t dots(const S &se, const AArgs &a, cudaStream_t s) {
    adot_kernel<XT><<<se.G_orth, kThreads, 0, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t lin(const S &se, const AArgs &a, cudaStream_t s) {
    alin_kernel<XT><<<se.G_orth, kThreads, 0, s>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t scal(const S &se, const AScalArgs &a, cudaStream_t s) {
    ascal_adj_kernel<<<se.key.R, kThreads, 0, s>>>(a);
    return cudaGetLastError();
  }
  template <int T>
  static cudaError_t spmm_xt(const S &se, const StoredCsr &M, BSpmmArgs &a, cudaStream_t s) {
    dim3 grid(se.G_rows, (se.key.R + T - 1) / T);
    BEngine<VT, XT>::template launch_spmm<T>(se, M, a, grid, s);
    return cudaGetLastError();
  }
  // y (=|+=) A x or A^T x with the session's tile width for that product (the
  // forward's tuned or requested width; results do not depend on it)
  static cudaError_t spmm_x(const S &se, bool fwd, const XT *x, XT *y, int accumulate, int j, cudaStream_t s) {
    const StoredCsr &M = fwd ? se.plan->A : se.plan->T;
    BSpmmArgs a{M.rowptr, M.col, M.val, M.rows, fwd ? se.wrowA : se.wrowT, kBSpmmExplicit, x, y, accumulate,
                se.a_kr, j};
    switch (fwd ? se.tileA : se.tileT) {
      case 8: return spmm_xt<8>(se, M, a, s);
      case 16: return spmm_xt<16>(se, M, a, s);
      case 32: return spmm_xt<32>(se, M, a, s);
      default: return spmm_xt<64>(se, M, a, s);
    }
  }
  static cudaError_t st_apply(const S &se, const double *V, int64_t vstride, int j, XT *out, cudaStream_t s) {
    const int64_t tot = se.bp.m * se.ld;
    ast_kernel<XT><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(se.key.R, se.ld, se.bp.m, se.key.zeta, se.bp.isz,
                                                                 se.kin, se.vin, V, vstride, se.a_kr, j, out);
    return cudaGetLastError();
  }

  static int run(S &se, const double *Xbar, double *Bbar, double *dbar, cudaStream_t s) {
    int r;
    if ((r = workspace(se))) return r;
    const int R = se.key.R, ld = se.ld, K = se.key.maxit, Sk = se.key.s, L = se.key.ell;
    const int64_t m = se.bp.m, n = se.bp.n;
    const size_t xs = sizeof(XT);
    // steps of every right-hand side
    std::vector<SolveState> h(R);
    SFL_CU(cudaMemcpyAsync(h.data(), se.bp.st, sizeof(SolveState) * R, cudaMemcpyDeviceToHost, s));
    SFL_CU(cudaStreamSynchronize(s));
    std::vector<int> kr(R);
    int kmax = 0;
    for (int q = 0; q < R; ++q) { kr[q] = h[q].k; kmax = std::max(kmax, kr[q]); }
    SFL_CU(cudaMemcpyAsync(se.a_kr, kr.data(), sizeof(int) * R, cudaMemcpyHostToDevice, s));
    if (!se.dwbuf) {
      std::vector<double> one(n, 1.0);
      SFL_CU(cudaMemcpyAsync(se.a_ones, one.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
      SFL_CU(cudaStreamSynchronize(s));
    }
    dim3 tg((unsigned)((n + 31) / 32), (ld + 31) / 32), tb(32, 8);
    binterleave_kernel<XT><<<tg, tb, 0, s>>>(Xbar, n, R, ld, se.a_xbar);
    SFL_CU(cudaGetLastError());
    SFL_CU(cudaMemsetAsync(se.a_wbar, 0, xs * (size_t)(L + 2) * m * ld, s));
    SFL_CU(cudaMemsetAsync(se.a_pbar, 0, xs * (size_t)(L + 1) * n * ld, s));
    SFL_CU(cudaMemsetAsync(se.a_dacc, 0, sizeof(double) * n * ld, s));
    SFL_CU(cudaMemsetAsync(se.a_ybar, 0, sizeof(double) * (size_t)R * K, s));
    const XT *Wb = se.bp.W, *Pb = se.bp.P, *Hb = se.bp.what;
    auto wslot = [&](int j) { return Wb + (size_t)(j - 1) * m * ld; };     // w~_j
    auto pslot = [&](int j) { return Pb + (size_t)(j - 1) * n * ld; };     // p~_j
    auto hslot = [&](int j) { return Hb + (size_t)(j - 1) * m * ld; };     // A z~_j
    auto wbar = [&](int j) { return se.a_wbar + (size_t)(j % (L + 2)) * m * ld; };
    auto pbar = [&](int j) { return se.a_pbar + (size_t)(j % (L + 1)) * n * ld; };
    const int64_t sW = K + 2, sP = K + 1;
    // ybar_j = <z_j, xbar>, z_j = d * sigP_j p~_j (seven columns per pass)
    for (int j0 = 1; j0 <= kmax; j0 += kAdjNV - 1) {
      AArgs a = args(se, n, j0);
      a.nv = 1 + std::min(kAdjNV - 1, kmax - j0 + 1);
      a.v[0] = vec(se.a_xbar);
      for (int l = 1; l < a.nv; ++l) a.v[l] = vec(pslot(j0 + l - 1), se.bp.sigP + (j0 + l - 1), sP, 1);
      SFL_CU(dots(se, a, s));
      SFL_CU(scal(se, sargs(se, kAScalYbar, j0, a.nv), s));
    }
    als_adj_kernel<<<R, kThreads, sizeof(double) * 2 * K, s>>>(R, Sk, K, se.a_kr, se.Q, se.Rinv, se.y, se.bp.e,
                                                                 se.a_ybar, se.a_sbar, se.a_Mbar);
    SFL_CU(cudaGetLastError());
    for (int j = kmax; j >= 1; --j) {
      // ---- m side
      SFL_CU(st_apply(se, se.a_Mbar + (size_t)(j - 1) * Sk, (int64_t)K * Sk, j, se.a_stm, s));
      const int lo = std::max(1, j - L), nw = j - lo + 1;
      AArgs a = args(se, m, j);
      a.nv = 2 + nw;
      a.v[0] = vec(wbar(j + 1));
      a.v[1] = vec(wslot(j + 1), se.bp.sigW + (j + 1), sW);
      for (int t = 0; t < nw; ++t) a.v[2 + t] = vec(wslot(lo + t), se.bp.sigW + (lo + t), sW);
      SFL_CU(dots(se, a, s));
      SFL_CU(scal(se, sargs(se, kAScalM, j, a.nv), s));
      a.v[2 + nw] = vec(hslot(j), se.bp.sigP + j, sP);
      a.v[3 + nw] = vec(se.a_stm);
      a.nv = 4 + nw;
      a.no = 2 + nw;
      a.o[0] = AOut{se.a_whatbar, 0, 0};
      for (int t = 0; t < nw; ++t) a.o[1 + t] = AOut{wbar(lo + t), 0, 1};
      a.o[1 + nw] = AOut{wbar(j + 1), 0, 0};
      SFL_CU(lin(se, a, s));
      // ---- u = A^T (adjoint of A z_j)
      SFL_CU(spmm_x(se, false, se.a_whatbar, se.a_u, 0, j, s));
      // ---- n side
      AArgs pa = args(se, n, j);
      pa.nv = 3;
      pa.v[0] = vec(se.a_u);
      pa.v[1] = vec(se.a_xbar, se.y + (j - 1), K);
      pa.v[2] = vec(pslot(j), se.bp.sigP + j, sP);
      pa.no = 2;
      pa.o[0] = AOut{pbar(j), 0, 1};
      pa.o[1] = AOut{se.a_dacc, 1, 1};
      apre_kernel<XT><<<se.G_orth, kThreads, 0, s>>>(pa);
      SFL_CU(cudaGetLastError());
      const int np = j - lo;
      AArgs b = args(se, n, j);
      b.nv = 2 + np;
      b.v[0] = vec(pbar(j));
      b.v[1] = vec(pslot(j), se.bp.sigP + j, sP);
      for (int t = 0; t < np; ++t) b.v[2 + t] = vec(pslot(lo + t), se.bp.sigP + (lo + t), sP);
      SFL_CU(dots(se, b, s));
      SFL_CU(scal(se, sargs(se, kAScalN, j, b.nv), s));
      b.no = 2 + np;
      b.o[0] = AOut{se.a_tbar, 0, 0};
      for (int t = 0; t < np; ++t) b.o[1 + t] = AOut{pbar(lo + t), 0, 1};
      b.o[1 + np] = AOut{pbar(j), 0, 0};
      SFL_CU(lin(se, b, s));
      // ---- wbar_j += A tbar_j
      SFL_CU(spmm_x(se, true, se.a_tbar, wbar(j), 1, j, s));
    }
    // b-bar = S^T sbar + (wbar_1 - <w_1, wbar_1> w_1) / beta_0
    SFL_CU(st_apply(se, se.a_sbar, Sk, 1, se.a_tmpA, s));
    AArgs f = args(se, m, 1);
    f.nv = 2;
    f.v[0] = vec(wbar(1));
    f.v[1] = vec(wslot(1), se.bp.sigW + 1, sW);
    SFL_CU(dots(se, f, s));
    SFL_CU(scal(se, sargs(se, kAScalFinal, 1, 2), s));
    f.nv = 3;
    f.v[2] = vec(se.a_tmpA);
    f.no = 1;
    f.o[0] = AOut{se.a_tmpB, 0, 0};
    SFL_CU(lin(se, f, s));
    dim3 tm((unsigned)((m + 31) / 32), (R + 31) / 32);
    adeinterleave_kernel<XT><<<tm, tb, 0, s>>>(se.a_tmpB, m, R, ld, Bbar);
    SFL_CU(cudaGetLastError());
    if (dbar) {
      adsum_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(se.a_dacc, n, R, ld, dbar);
      SFL_CU(cudaGetLastError());
    }
    return SFL_OK;
  }
};

static int check_batched(const Plan &pl, int R, const sfl_opts *o) {
  if (!o || R < 1 || R > kBMaxRhs) return SFL_EINVAL;
  if (pl.matfree) return SFL_EUNSUPPORTED;   // the SpMMs read a stored matrix
  if (o->sketch_kind != SFL_SKETCH_SPARSE_SIGN) return SFL_EUNSUPPORTED;   // batched sketches are sparse-sign
  if (o->maxit < 1 || o->maxit > kMaxIt) return SFL_EINVAL;
  if (o->zeta < 1 || o->zeta > kMaxZeta) return SFL_EINVAL;
  if (o->s < o->maxit + 1 || o->s < o->zeta || o->s > kMaxS) return SFL_EINVAL;
  if (o->window < 0) return SFL_EUNSUPPORTED;
  if (o->window > kMaxWindow) return SFL_EINVAL;
  if (o->noise_norm > 0.0 && !(o->eta > 0.0)) return SFL_EINVAL;
  if (o->precond == SFL_PRECOND_REWEIGHT || o->precond == SFL_PRECOND_LOWRANK) return SFL_EUNSUPPORTED;
  if (o->precond != SFL_PRECOND_IDENTITY && o->precond != SFL_PRECOND_DIAG) return SFL_EINVAL;
  if (o->precond == SFL_PRECOND_DIAG && !o->diag_w) return SFL_EINVAL;
  if (o->orth_against_z != 0) return o->orth_against_z == 1 ? SFL_EUNSUPPORTED : SFL_EINVAL;
  if (o->sketch_dense || o->sketch_dense_stop) return SFL_EUNSUPPORTED;
  if (o->spmm_tile != 0 && o->spmm_tile != 8 && o->spmm_tile != 16 && o->spmm_tile != 32 && o->spmm_tile != 64)
    return SFL_EINVAL;
  (void)pl;
  return SFL_OK;
}

int batched_solve(sfl_plan *plan, int32_t nrhs, const double *B, const double *noise_norms, const sfl_opts *opts,
                  double *X, sfl_info *infos, sfl_stream stream, int keep_what, BatchSessionBase **used = nullptr) {
  if (!plan || !B || !noise_norms || !X) return SFL_EINVAL;
  Plan &pl = plan->impl;
  int r = check_batched(pl, nrhs, opts);
  if (r) return r;
  for (int j = 0; j < nrhs; ++j)
    if (noise_norms[j] > 0.0 && !(opts->eta > 0.0)) return SFL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (pl.vdt == SFL_F64) {
    BatchSession<double, double> *u = nullptr;
    r = BEngine<double, double>::solve(pl, nrhs, B, noise_norms, opts, X, infos, s, keep_what, &u);
    if (used) *used = u;
    return r;
  }
  if (pl.vdt == SFL_F32) {
    BatchSession<float, float> *u = nullptr;
    r = BEngine<float, float>::solve(pl, nrhs, B, noise_norms, opts, X, infos, s, keep_what, &u);
    if (used) *used = u;
    return r;
  }
  BatchSession<__nv_bfloat16, float> *u = nullptr;
  r = BEngine<__nv_bfloat16, float>::solve(pl, nrhs, B, noise_norms, opts, X, infos, s, keep_what, &u);
  if (used) *used = u;
  return r;
}

// Fixed-k forward for differentiation: no stop test, A z~_j kept.
int fixed_batched(sfl_plan *plan, int32_t nrhs, const double *B, const sfl_opts *opts, double *X, sfl_info *infos,
                  sfl_stream stream) {
  if (!plan || !opts) return SFL_EINVAL;
  if (opts->window > 3) return SFL_EUNSUPPORTED;   // the adjoint's combination kernels hold windows up to 3
  if (nrhs < 1 || nrhs > kBMaxRhs) return SFL_EINVAL;
  std::vector<double> zero(nrhs, 0.0);
  Plan &pl = plan->impl;
  pl.last_fixed = nullptr;
  BatchSessionBase *u = nullptr;
  const int r = batched_solve(plan, nrhs, B, zero.data(), opts, X, infos, stream, 1, &u);
  if (r) return r;
  pl.last_fixed = u;
  pl.fixed_calls += 1;
  return SFL_OK;
}

int adjoint_batched(sfl_plan *plan, int32_t nrhs, const double *Xbar, double *Bbar, double *dbar, sfl_stream stream) {
  if (!plan || !Xbar || !Bbar) return SFL_EINVAL;
  Plan &pl = plan->impl;
  BatchSessionBase *b = pl.last_fixed;
  bool live = false;
  for (auto &p : pl.batches) live |= p.get() == b;
  if (!b || !live) return SFL_EINVAL;   // no fixed-k forward kept by this plan
  cudaStream_t s = (cudaStream_t)stream;
  if (auto q = dynamic_cast<BatchSession<double, double> *>(b)) {
    if (q->key.R != nrhs) return SFL_EINVAL;
    return AEngine<double, double>::run(*q, Xbar, Bbar, dbar, s);
  }
  if (auto q = dynamic_cast<BatchSession<float, float> *>(b)) {
    if (q->key.R != nrhs) return SFL_EINVAL;
    return AEngine<float, float>::run(*q, Xbar, Bbar, dbar, s);
  }
  if (auto q = dynamic_cast<BatchSession<__nv_bfloat16, float> *>(b)) {
    if (q->key.R != nrhs) return SFL_EINVAL;
    return AEngine<__nv_bfloat16, float>::run(*q, Xbar, Bbar, dbar, s);
  }
  return SFL_EINVAL;
}

}  // namespace sfl

using namespace sfl;

extern "C" int sflsqr_solve_batched(sfl_plan *plan, int32_t nrhs, const double *B, const double *noise_norms,
                                    const sfl_opts *opts, double *X, sfl_info *infos, sfl_stream stream) {
  return batched_solve(plan, nrhs, B, noise_norms, opts, X, infos, stream, 0);
}

extern "C" int sflsqr_fixed_batched(sfl_plan *plan, int32_t nrhs, const double *B, const sfl_opts *opts, double *X,
                                    sfl_info *infos, sfl_stream stream) {
  return fixed_batched(plan, nrhs, B, opts, X, infos, stream);
}

extern "C" int sflsqr_adjoint_batched(sfl_plan *plan, int32_t nrhs, const double *Xbar, double *Bbar, double *dbar,
                                      sfl_stream stream) {
  return adjoint_batched(plan, nrhs, Xbar, Bbar, dbar, stream);
}

extern "C" int64_t sfl_fixed_calls(const sfl_plan *plan) { return plan ? plan->impl.fixed_calls : -1; }

extern "C" int sfl_batched_tile(const sfl_plan *plan, int32_t which) {
  if (!plan || (which != 0 && which != 1)) return -1;
  const Plan &pl = plan->impl;
  if (pl.batches.empty()) return 0;
  const BatchSessionBase *b = pl.batches.back().get();
  if (auto q = dynamic_cast<const BatchSession<double, double> *>(b)) return which ? q->tileT : q->tileA;
  if (auto q = dynamic_cast<const BatchSession<float, float> *>(b)) return which ? q->tileT : q->tileA;
  if (auto q = dynamic_cast<const BatchSession<__nv_bfloat16, float> *>(b)) return which ? q->tileT : q->tileA;
  return 0;
}
