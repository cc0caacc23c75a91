// Solve driver: per-configuration sessions (workspace + CUDA graph whose body
// is one step of Algorithm 1 / 2 inside a device-controlled WHILE node), the
// solver entry points, plan apply/destroy and the sketch entry points.
#include <chrono>
#include <cstring>
#include <thread>

#include "engine.h"

namespace sfl {

static constexpr double kHostWaitSeconds = 1800.0;

// Host wait with a wall-clock limit (cudaEventQuery polling).
static int wait_stream(cudaStream_t s) {
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

size_t ls_smem_bytes(int s, int maxit, int cluster) {
  const int RB = (s + cluster - 1) / cluster;
  return sizeof(double) * (size_t)(4 * (maxit + 2) + RB + std::max(kThreads, RB) + RB);
}

int ls_cluster_size(int s, int maxit) {
  cudaFuncSetAttribute(ls_step_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int cl : {16, 8, 4, 2, 1}) {
    const size_t smem = ls_smem_bytes(s, maxit, cl);
    if (cudaFuncSetAttribute(ls_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
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

cudaError_t launch_ls(const LsParams &p, int cluster, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, ls_step_kernel, p);
}

static size_t spmv_smem(int s, size_t xsize) {
  return xsize * (size_t)kWarps * s + sizeof(double) * (size_t)(1 + kMaxWindow + 2 + s + kWarps * (kMaxWindow + 3));
}
static size_t orth_smem() { return sizeof(double) * (size_t)(kMaxWindow + 3) * (1 + kWarps); }

template <typename VT, typename XT>
struct Engine {
  using O = Ops<VT, XT>;

  static SpmvParams<VT, XT> base_params(const Plan &pl, const Session &se, const StoredCsr &M, int mode) {
    SpmvParams<VT, XT> p{};
    p.rowptr = M.rowptr; p.col = M.col; p.val = (const VT *)M.val; p.rows = M.rows;
    p.mode = mode;
    p.method = se.key.method; p.stop_rule = se.key.stop_rule;
    p.ell = se.key.ell; p.s = se.key.s; p.zeta = se.key.zeta; p.zs = se.zs; p.maxit = se.key.maxit;
    p.st = se.st;
    p.wring = (XT *)se.wring; p.wstride = pl.A.rows; p.RW = se.RW;
    p.pring = (XT *)se.pring; p.pstride = pl.A.cols; p.RP = se.RP;
    p.Z = (XT *)se.Z; p.zstride = pl.A.cols; p.sigZ = se.sigZ;
    p.wraw = (XT *)se.wraw; p.zraw = (XT *)se.zraw;
    p.SAZ = se.SAZ; p.SAtW = se.SAtW; p.Hband = se.Hband; p.rhs = se.rhs; p.e = se.e; p.sbm = se.sbm;
    p.red = se.red;
    return p;
  }

  static OrthParams<XT> orth_params(const Plan &pl, const Session &se, int side) {
    OrthParams<XT> o{};
    o.st = se.st; o.side = side; o.ell = se.key.ell;
    o.method = se.key.method;
    o.red = se.red;
    o.Hband = se.Hband;
    if (side == 0) {
      o.len = pl.A.cols; o.raw = (const XT *)se.zraw; o.ring = (XT *)se.pring; o.stride = pl.A.cols; o.R = se.RP;
      o.Z = (XT *)se.Z; o.zstride = pl.A.cols; o.sigZ = se.sigZ;
      o.precond = se.key.precond; o.diag_w = se.dw; o.y = se.y;
    } else {
      o.len = pl.A.rows; o.raw = (const XT *)se.wraw; o.ring = (XT *)se.wring; o.stride = pl.A.rows; o.R = se.RW;
      o.sigZ = se.sigZ;
    }
    return o;
  }

  static LsParams ls_params(const Session &se, int use_cond, cudaGraphConditionalHandle h) {
    LsParams q{};
    q.st = se.st; q.method = se.key.method; q.s = se.key.s; q.maxit = se.key.maxit; q.ell = se.key.ell;
    q.stop_rule = se.key.stop_rule;
    q.Q = se.Q; q.Rinv = se.Rinv; q.y = se.y; q.e = se.e;
    q.SAZ = se.SAZ; q.SAtW = se.SAtW; q.Hband = se.Hband; q.sbm = se.sbm;
    q.relres_hist = se.key.r_hist;
    q.cond = h; q.use_cond = use_cond;
    return q;
  }

  static int enqueue_prologue(const Plan &pl, const Session &se, cudaStream_t s) {
    const int64_t m = pl.A.rows, n = pl.A.cols;
    const int method = se.key.method;
    const uint64_t *seed_src = &se.st->seed;
    // m-side sketch: S_m for sFLSQR, the stop sketch (seed + 1) for sFLSMR
    sketch_table_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(0, seed_src, method == kSFLSMR ? 1 : 0,
                                                                     se.key.s, se.key.zeta, m, se.zs, se.tab_m,
                                                                     nullptr, nullptr, se.err);
    SFL_CU(cudaGetLastError());
    if (method == kSFLSMR) {
      sketch_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(0, seed_src, 0, se.key.s, se.key.zeta, n, se.zs,
                                                                       se.tab_n, nullptr, nullptr, se.err);
      SFL_CU(cudaGetLastError());
    }
    SpmvParams<VT, XT> p = base_params(pl, se, pl.A, kModeInitB);
    p.rows = m; p.b = se.bbuf; p.tab = se.tab_m;
    SFL_CU(O::spmv(p, 32, false, se.grid_init, se.smem_init, s));
    p = base_params(pl, se, pl.T, kModeInitBwd);
    p.tab = se.tab_n;
    SFL_CU(O::spmv(p, pl.T.lpr, true, se.grid_spmv_T, se.smem_T, s));
    return SFL_OK;
  }

  static int enqueue_body(const Plan &pl, const Session &se, cudaStream_t s, int use_cond,
                          cudaGraphConditionalHandle h) {
    SFL_CU(O::orth(orth_params(pl, se, 0), se.grid_vec, se.smem_orth, s));
    SpmvParams<VT, XT> p = base_params(pl, se, pl.A, kModeFwd);
    p.tab = se.tab_m;
    SFL_CU(O::spmv(p, pl.A.lpr, true, se.grid_spmv_A, se.smem_A, s));
    SFL_CU(O::orth(orth_params(pl, se, 1), se.grid_vec, se.smem_orth, s));
    p = base_params(pl, se, pl.T, kModeBwd);
    p.tab = se.tab_n;
    SFL_CU(O::spmv(p, pl.T.lpr, true, se.grid_spmv_T, se.smem_T, s));
    SFL_CU(launch_ls(ls_params(se, use_cond, h), se.ls_cluster, se.smem_ls, s));
    if (se.key.x_hist) {
      SFL_CU(O::solution(se.st, (const XT *)se.Z, pl.A.cols, se.sigZ, se.y, pl.A.cols, nullptr, se.key.x_hist,
                         se.grid_vec, s));
      clear_hist_flag_kernel<<<1, 1, 0, s>>>(se.st);
      SFL_CU(cudaGetLastError());
    }
    return SFL_OK;
  }

  static int enqueue_epilogue(const Plan &pl, const Session &se, cudaStream_t s) {
    return O::solution(se.st, (const XT *)se.Z, pl.A.cols, se.sigZ, se.y, pl.A.cols, se.xbuf, nullptr, se.grid_vec,
                       s) == cudaSuccess ? SFL_OK : SFL_ECUDA;
  }

  static int build_graph(const Plan &pl, Session &se, cudaStream_t s) {
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
      r = enqueue_body(pl, se, cs, 1, h);
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
    (void)s;
    return r;
  }

  static int create(Plan &pl, const SessionKey &key, cudaStream_t s, Session **out) {
    auto se = std::make_unique<Session>();
    se->key = key;
    const int64_t m = pl.A.rows, n = pl.A.cols;
    const int S = key.s, K = key.maxit, ell = key.ell;
    const size_t xs = sizeof(XT);
    se->RW = ell + 2;
    se->RP = ell + 1;
    se->zs = key.zeta <= 8 ? 8 : 16;
    int r;
#define SA(ptr, bytes) if ((r = session_alloc(pl, *se, (void **)&(ptr), (bytes)))) { destroy_session(pl, *se); return r; }
    SA(se->st, sizeof(SolveState));
    SA(se->wring, xs * se->RW * m);
    SA(se->pring, xs * se->RP * n);
    SA(se->wraw, xs * m);
    SA(se->zraw, xs * n);
    SA(se->Z, xs * (size_t)n * K);
    SA(se->sigZ, sizeof(double) * K);
    SA(se->tab_m, sizeof(uint16_t) * se->zs * m);
    if (key.method == kSFLSMR) SA(se->tab_n, sizeof(uint16_t) * se->zs * n);
    SA(se->Q, sizeof(double) * (size_t)S * K);
    SA(se->Rinv, sizeof(double) * (size_t)K * K);
    SA(se->y, sizeof(double) * K);
    SA(se->e, sizeof(double) * S);
    SA(se->rhs, sizeof(double) * S);
    SA(se->SAZ, sizeof(double) * (size_t)S * K);
    SA(se->SAtW, sizeof(double) * (size_t)S * (K + 1));
    SA(se->Hband, sizeof(double) * (size_t)K * (ell + 2));
    SA(se->sbm, sizeof(double) * S);
    SA(se->bbuf, sizeof(double) * m);
    SA(se->xbuf, sizeof(double) * n);
    if (key.precond == SFL_PRECOND_DIAG) SA(se->dw, sizeof(double) * n);
    SA(se->err, sizeof(int));
    // launch shapes
    const size_t smem = spmv_smem(S, xs);
    if (smem > 200 * 1024) { destroy_session(pl, *se); return SFL_EUNSUPPORTED; }
    se->smem_A = se->smem_T = se->smem_init = smem;
    SFL_CU(O::set_smem(pl.A.lpr, true, smem));
    SFL_CU(O::set_smem(pl.T.lpr, true, smem));
    SFL_CU(O::set_smem(32, false, smem));
    auto grid_of = [&](int lpr, bool mat) {
      int occ = O::spmv_occupancy(lpr, mat, smem);
      if (occ < 1) occ = 1;
      if (occ > 8) occ = 8;
      return std::min(pl.num_sms * occ, kGroup * kMaxGroups);
    };
    se->grid_spmv_A = grid_of(pl.A.lpr, true);
    se->grid_spmv_T = grid_of(pl.T.lpr, true);
    se->grid_init = grid_of(32, false);
    se->grid_vec = std::min(pl.num_sms * 4, kGroup * kMaxGroups);
    se->smem_orth = orth_smem();
    se->ls_cluster = ls_cluster_size(S, K);
    if (se->ls_cluster < 1) { destroy_session(pl, *se); return SFL_EUNSUPPORTED; }
    se->smem_ls = ls_smem_bytes(S, K, se->ls_cluster);
    SFL_CU(cudaFuncSetAttribute(ls_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)se->smem_ls));
    const int gmax = std::max(std::max(se->grid_spmv_A, se->grid_spmv_T), std::max(se->grid_init, se->grid_vec));
    se->red.stride = S + kMaxWindow + 8;
    SA(se->red.part, sizeof(double) * (size_t)gmax * se->red.stride);
    SA(se->red.gpart, sizeof(double) * (size_t)kMaxGroups * se->red.stride);
    SA(se->red.cnt, sizeof(unsigned) * (kMaxGroups + 1));
#undef SA
    SFL_CU(cudaMemsetAsync(se->red.cnt, 0, sizeof(unsigned) * (kMaxGroups + 1), s));
    SFL_CU(cudaMemsetAsync(se->err, 0, sizeof(int), s));
    SFL_CU(cudaMemsetAsync(se->Hband, 0, sizeof(double) * (size_t)K * (ell + 2), s));
    SFL_CU(cudaStreamSynchronize(s));
    if ((r = build_graph(pl, *se, s))) { destroy_session(pl, *se); return r; }
    *out = se.get();
    pl.sessions.push_back(std::move(se));
    return SFL_OK;
  }

  // Host-driven pass with a CUDA event pair around every launch.
  static int run_profiled(const Plan &pl, const Session &se, cudaStream_t s, sfl_kernel_times *kt) {
    constexpr int kChunk = 8;
    constexpr int kEv = 2 * (6 * kChunk + 8);
    cudaEvent_t ev[kEv];
    for (int i = 0; i < kEv; ++i) SFL_CU(cudaEventCreate(&ev[i]));
    struct Rec { int cls, step; };
    std::vector<Rec> recs;
    int nev = 0;
    int r = SFL_OK;
    auto timed = [&](int cls, int step, auto &&launch) -> int {
      cudaEventRecord(ev[nev], s);
      int q = launch();
      cudaEventRecord(ev[nev + 1], s);
      recs.push_back({cls, step});
      nev += 2;
      return q;
    };
    auto flush = [&](int done_steps) -> int {
      SFL_CU(cudaEventSynchronize(ev[nev - 1]));
      for (size_t i = 0; i < recs.size(); ++i) {
        if (recs[i].step >= done_steps && recs[i].step >= 0) continue;   // returned early after the stop
        float ms = 0.f;
        SFL_CU(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
        kt->ms[recs[i].cls] += ms;
        kt->launches[recs[i].cls] += 1;
      }
      recs.clear();
      nev = 0;
      return SFL_OK;
    };
    const int64_t m = pl.A.rows, n = pl.A.cols;
    const int method = se.key.method;
    const uint64_t *seed_src = &se.st->seed;
    r = timed(0, -1, [&] {
      sketch_table_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(0, seed_src, method == kSFLSMR ? 1 : 0, se.key.s,
                                                                       se.key.zeta, m, se.zs, se.tab_m, nullptr,
                                                                       nullptr, se.err);
      if (method == kSFLSMR)
        sketch_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(0, seed_src, 0, se.key.s, se.key.zeta, n,
                                                                         se.zs, se.tab_n, nullptr, nullptr, se.err);
      return cudaGetLastError() == cudaSuccess ? SFL_OK : SFL_ECUDA;
    });
    if (r) return r;
    r = timed(1, -1, [&] {
      SpmvParams<VT, XT> p = base_params(pl, se, pl.A, kModeInitB);
      p.rows = m; p.b = se.bbuf; p.tab = se.tab_m;
      return O::spmv(p, 32, false, se.grid_init, se.smem_init, s) == cudaSuccess ? SFL_OK : SFL_ECUDA;
    });
    if (r) return r;
    r = timed(2, -1, [&] {
      SpmvParams<VT, XT> p = base_params(pl, se, pl.T, kModeInitBwd);
      p.tab = se.tab_n;
      return O::spmv(p, pl.T.lpr, true, se.grid_spmv_T, se.smem_T, s) == cudaSuccess ? SFL_OK : SFL_ECUDA;
    });
    if (r) return r;
    if ((r = flush(0))) return r;
    int done = 0;
    for (int it0 = 0; it0 < se.key.maxit; it0 += kChunk) {
      for (int it = it0; it < std::min(it0 + kChunk, se.key.maxit); ++it) {
        r = timed(3, it, [&] { return O::orth(orth_params(pl, se, 0), se.grid_vec, se.smem_orth, s) == cudaSuccess ? SFL_OK : SFL_ECUDA; });
        if (r) return r;
        r = timed(4, it, [&] {
          SpmvParams<VT, XT> p = base_params(pl, se, pl.A, kModeFwd);
          p.tab = se.tab_m;
          return O::spmv(p, pl.A.lpr, true, se.grid_spmv_A, se.smem_A, s) == cudaSuccess ? SFL_OK : SFL_ECUDA;
        });
        if (r) return r;
        r = timed(5, it, [&] { return O::orth(orth_params(pl, se, 1), se.grid_vec, se.smem_orth, s) == cudaSuccess ? SFL_OK : SFL_ECUDA; });
        if (r) return r;
        r = timed(6, it, [&] {
          SpmvParams<VT, XT> p = base_params(pl, se, pl.T, kModeBwd);
          p.tab = se.tab_n;
          return O::spmv(p, pl.T.lpr, true, se.grid_spmv_T, se.smem_T, s) == cudaSuccess ? SFL_OK : SFL_ECUDA;
        });
        if (r) return r;
        r = timed(7, it, [&] { return launch_ls(ls_params(se, 0, 0), se.ls_cluster, se.smem_ls, s) == cudaSuccess ? SFL_OK : SFL_ECUDA; });
        if (r) return r;
      }
      int hk[2] = {0, 0};
      SFL_CU(cudaMemcpyAsync(hk, &se.st->k, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
      SFL_CU(cudaStreamSynchronize(s));
      done = hk[0];
      if ((r = flush(done))) return r;
      if (hk[1]) break;
    }
    r = timed(8, -1, [&] { return enqueue_epilogue(pl, se, s); });
    if (r) return r;
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
  if (o->zeta < 1 || o->zeta > kMaxZeta) return SFL_EINVAL;
  if (o->s < o->maxit + 1 || o->s < o->zeta || o->s > kMaxS) return SFL_EINVAL;
  if (o->window < 0) return SFL_EUNSUPPORTED;   // full orthogonalization: not on the GPU path
  if (o->window > kMaxWindow) return SFL_EINVAL;
  if (o->noise_norm > 0.0 && !(o->eta > 0.0)) return SFL_EINVAL;
  if (o->precond < 0 || o->precond > 2) return SFL_EINVAL;
  if (o->precond == SFL_PRECOND_DIAG && !o->diag_w) return SFL_EINVAL;
  if (o->precond == SFL_PRECOND_REWEIGHT && !(o->irw_eps > 0.0)) return SFL_EINVAL;
  if (o->stop_rule != SFL_STOP_RULE_RESIDUAL && o->stop_rule != SFL_STOP_RULE_NORMAL) return SFL_EINVAL;
  if (o->vec_dtype == SFL_F64 && pl.vdt != SFL_F64) return SFL_EINVAL;
  if (o->vec_dtype == SFL_F32 && pl.vdt == SFL_F64) return SFL_EUNSUPPORTED;
  if (o->vec_dtype != SFL_F64 && o->vec_dtype != SFL_F32) return SFL_EINVAL;
  (void)method;
  return SFL_OK;
}

template <typename VT, typename XT>
static int solve_typed(Plan &pl, const SolveRequest &q) {
  using E = Engine<VT, XT>;
  const sfl_opts *o = q.o;
  SessionKey key{q.method, o->s, o->zeta, o->window, o->maxit, o->precond,
                 q.method == kSFLSMR ? o->stop_rule : 0, o->vec_dtype, o->x_history, o->relres_history};
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
  SFL_CU(cudaMemcpyAsync(se->bbuf, q.b, sizeof(double) * m, q.b_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                         q.s));
  if (o->precond == SFL_PRECOND_DIAG)
    SFL_CU(cudaMemcpyAsync(se->dw, o->diag_w, sizeof(double) * n, cudaMemcpyDeviceToDevice, q.s));
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
  p.mode = kModeApply;
  const int grid = pl.num_sms * 4;
  if (std::is_same<XT, double>::value) {
    p.x = (const XT *)x; p.y = (XT *)y;
    SFL_CU(Ops<VT, XT>::spmv(p, M.lpr, true, grid, 0, s));
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
  SFL_CU(Ops<VT, XT>::spmv(p, M.lpr, true, grid, 0, s));
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

// Same solve driven by a host loop instead of the graph's WHILE node (one
// stream synchronisation per step); used to check that both drivers agree.
int sfl_solve_host_loop(sfl_plan *plan, int method, const double *b, const sfl_opts *opts, double *x, sfl_info *info,
                        sfl_stream stream) {
  if (method != kSFLSQR && method != kSFLSMR) return SFL_EINVAL;
  return solve(plan, SolveRequest{method, b, false, opts, x, false, info, (cudaStream_t)stream, true});
}

int sfl_solve_profiled(sfl_plan *plan, int method, const double *b, const sfl_opts *opts, double *x, sfl_info *info,
                       sfl_kernel_times *times, sfl_stream stream) {
  if (method != kSFLSQR && method != kSFLSMR) return SFL_EINVAL;
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
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int zs = zeta <= 8 ? 8 : 16;
  const size_t smem = spmv_smem(s, sizeof(double));
  const int grid = std::min(sms * 2, kGroup * kMaxGroups);
  const int stride = s + kMaxWindow + 8;
  uint16_t *tab = nullptr;
  double *part = nullptr, *gpart = nullptr;
  unsigned *cnt = nullptr;
  int *err = nullptr;
  int r = SFL_OK;
  do {
    if (cudaMalloc(&tab, sizeof(uint16_t) * zs * len) != cudaSuccess || cudaMalloc(&part, sizeof(double) * grid * stride) != cudaSuccess ||
        cudaMalloc(&gpart, sizeof(double) * kMaxGroups * stride) != cudaSuccess ||
        cudaMalloc(&cnt, sizeof(unsigned) * (kMaxGroups + 1)) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      r = SFL_ENOMEM;
      break;
    }
    cudaMemsetAsync(cnt, 0, sizeof(unsigned) * (kMaxGroups + 1), st);
    cudaMemsetAsync(err, 0, sizeof(int), st);
    sketch_table_kernel<<<(unsigned)((len + 255) / 256), 256, 0, st>>>(seed, nullptr, 0, s, zeta, len, zs, tab, nullptr,
                                                                        nullptr, err);
    SpmvParams<double, double> p{};
    p.rows = len; p.mode = kModeSketch; p.s = s; p.zeta = zeta; p.zs = zs; p.b = v; p.tab = tab; p.sk_out = sk;
    p.red.part = part; p.red.gpart = gpart; p.red.cnt = cnt; p.red.stride = stride;
    if (Ops<double, double>::set_smem(32, false, smem) != cudaSuccess ||
        Ops<double, double>::spmv(p, 32, false, grid, smem, st) != cudaSuccess) { r = SFL_ECUDA; break; }
    if (cudaStreamSynchronize(st) != cudaSuccess) { r = SFL_ECUDA; break; }
    int h = 0;
    cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (h) r = SFL_EINVAL;
  } while (0);
  if (r == SFL_ECUDA) set_cuda_error(cudaGetLastError(), "sfl_sketch_apply");
  cudaFree(tab); cudaFree(part); cudaFree(gpart); cudaFree(cnt); cudaFree(err);
  return r;
}

}  // extern "C"
