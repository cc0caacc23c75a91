// Host-side engine of the GB300 sFLSQR / sFLSMR library: plans, sessions and
// the typed launch wrappers implemented in the inst_*.cu units.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "lowrank.cuh"

namespace sfl {

// Stored operator: CSR with every row padded to a multiple of the load width
// (padding entries repeat a valid column with value 0).
struct StoredCsr {
  int32_t *rowptr = nullptr;
  int32_t *col = nullptr;
  void *val = nullptr;
  int32_t *orig = nullptr;   // stored row i is row orig[i] of the operator (nullptr: the identity)
  bool interleaved = false;  // chunk slots stored lane-interleaved (else the caller's entry order)
  // 16-bit column deltas along each lane's walk of a row (lane-interleaved
  // slots, lpr 8) and each row's base column, when every delta fits
  int16_t *dcol = nullptr;
  int32_t *rbase = nullptr;
  int64_t rows = 0, cols = 0, nnz = 0, pnnz = 0;
  int lpr = 32;
};

struct SessionKey {
  int method, s, zeta, ell, maxit, precond, stop_rule, vdt;
  double *x_hist, *r_hist;
  int orth_z;        // 1: the z window is the stored z_j (sfl_opts.orth_against_z)
  const double *dense_S, *dense_Sm;   // explicit sketches (sfl_opts.sketch_dense, sketch_dense_stop)
  int lr_rank = 0, lr_over = 0, lr_power = 0, lr_fp64 = 0;   // low-rank truncation (SFL_PRECOND_LOWRANK)
  int sk_apply = 0;  // sfl_opts.sketch_apply
  int sk_kind = 0;   // sfl_opts.sketch_kind
  bool operator==(const SessionKey &o) const {
    return method == o.method && s == o.s && zeta == o.zeta && ell == o.ell && maxit == o.maxit &&
           precond == o.precond && stop_rule == o.stop_rule && vdt == o.vdt && x_hist == o.x_hist &&
           r_hist == o.r_hist && orth_z == o.orth_z && dense_S == o.dense_S && dense_Sm == o.dense_Sm &&
           lr_rank == o.lr_rank && lr_over == o.lr_over && lr_power == o.lr_power && lr_fp64 == o.lr_fp64 &&
           sk_apply == o.sk_apply && sk_kind == o.sk_kind;
  }
};

struct Session {
  SessionKey key{};
  int64_t m = 0, n = 0;                // the plan's operator shape
  int RW = 0, RP = 0;
  SolveState *st = nullptr;
  void *wring = nullptr, *pring = nullptr, *wraw = nullptr, *zraw = nullptr, *Z = nullptr;
  double *sigZ = nullptr;
  // row-major sparse-sign tables (S_m; S_n for sFLSMR) for the seed tab_seed
  int32_t *skM_row = nullptr, *skN_row = nullptr;
  uint32_t *skM_ent = nullptr, *skN_ent = nullptr;
  uint32_t *sk_kin = nullptr, *sk_vin = nullptr, *sk_kout = nullptr;
  void *sk_cub = nullptr;
  size_t sk_cub_bytes = 0;
  bool tab_valid = false;
  uint64_t tab_seed = 0;
  double *Q = nullptr, *Rinv = nullptr, *y = nullptr, *e = nullptr, *rhs = nullptr;
  double *SAZ = nullptr, *SAtW = nullptr, *Hband = nullptr, *sbm = nullptr;
  double *bbuf = nullptr, *xbuf = nullptr, *dw = nullptr;
  // full orthogonalization (window < 0): every basis vector, the w scales, CGS2 scratch
  bool full = false;
  int hb_ell = 0;                      // H band width minus 2 (ell, or maxit when full)
  void *Pfull = nullptr, *Wfull = nullptr;
  void *zcgs = nullptr, *wcgs = nullptr;   // orthogonalized product outputs (the raw ones stay for the sketch)
  double *sigWall = nullptr, *cgs_rec = nullptr, *cgs_coef = nullptr;
  int grid_cgs = 0;
  // fused sparse-sign sketch (the products' epilogues draw and add; the w
  // update and the small least-squares step reduce the per-CTA records): no
  // per-step sketch launch
  bool sk_fused = false;
  double *skw_rec = nullptr, *skz_rec = nullptr;   // [s][grid of the product]
  // low-rank truncation by the randomized SVD (SFL_PRECOND_LOWRANK)
  bool lowrank = false;
  LrParams<float> lr32{};       // FP32 arithmetic (default)
  LrParams<double> lr64{};      // FP64 arithmetic (sfl_opts.lowrank_fp64)
  int *err = nullptr;
  Partials part{};                     // per-CTA partial sums of the reducing kernels
  int32_t *wrowA = nullptr, *wrowT = nullptr;   // nnz-balanced row range of every warp
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int grid_spmv_A = 0, grid_spmv_T = 0, grid_vec = 0, grid_init = 0;
  size_t smem_A = 0, smem_T = 0, smem_init = 0, smem_orth = 0, smem_ls = 0;
  int ls_cluster = 8;
  int ls_stage = 0;
  std::vector<void *> allocs;
  uint64_t bytes = 0;
};

// A batched-solve session (typed; freed with its plan).
struct BatchSessionBase {
  virtual ~BatchSessionBase() = default;
};

struct Plan {
  int device = 0;
  int num_sms = 0;
  sfl_dtype vdt = SFL_F64;
  bool unmatched = false;
  int lpr_override = 0;      // lanes per row requested by the caller (0: from the row lengths)
  int img_rows = 0, img_cols = 0;   // n-side image shape: A^T / B rows stored in pixel tiles
  int slot_layout = 0;              // 0: lane-interleaved chunk slots, 1: the caller's entry order
  int index_bits = 0;               // 0: 16-bit column deltas where every delta fits, 32: 32-bit indices only
  StoredCsr A, T;   // T: CSR of A^T (transposed copy) or of B
  // matrix-free CT operator (sfl_plan_create_ct): no CSR arrays, products computed on the fly
  bool matfree = false;
  int ct_N = 0, ct_na = 0, ct_nb = 0, ct_back = 0;
  void *ct_tab = nullptr;   // per-angle constants, kProjTab each, FP64 or FP32 (the plan's arithmetic)
  long long *ct_fix = nullptr;   // FP64 plans: per angle round(cos 2^F), F = proj_bin_frac_bits(n_bins)
  uint64_t bytes = 0, cap = 0;
  std::vector<void *> allocs;
  std::vector<std::unique_ptr<Session>> sessions;
  std::vector<std::unique_ptr<BatchSessionBase>> batches;
  BatchSessionBase *last_fixed = nullptr;   // session of the latest fixed-k forward (for its adjoint)
  int64_t fixed_calls = 0;
  // scratch for sfl_plan_apply
  void *apply_x = nullptr, *apply_y = nullptr;
  int32_t *apply_wrow[2] = {nullptr, nullptr};   // warp row ranges of A and of A^T / B, balanced by row cost
  RedScratch apply_red{};
};

// Kernel launch, optionally with a programmatic dependency on the previous
// kernel of the stream (the kernel then waits in griddep_wait; inside a
// captured graph this becomes a programmatic edge).
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                     Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (pdl) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Typed launch wrappers (one instantiation unit per precision pair).
template <typename VT, typename XT>
struct Ops {
  static cudaError_t spmv(const SpmvParams<VT, XT> &p, int lpr, bool mat, int grid, size_t smem, cudaStream_t s,
                          bool pdl = false);
  static cudaError_t orth(const OrthParams<XT> &p, int grid, size_t smem, cudaStream_t s, bool pdl = false);
  static cudaError_t solution(SolveState *st, const XT *Z, int64_t zstride, const double *sigZ, const double *y,
                              int64_t n, double *x, double *hist, int grid, cudaStream_t s);
  static cudaError_t convert_in(const double *x, XT *y, int64_t n, cudaStream_t s);
  static cudaError_t convert_out(const XT *x, double *y, int64_t n, cudaStream_t s);
  static int spmv_occupancy(int lpr, bool mat, size_t smem);
  static int proj_occupancy(size_t smem);
  static cudaError_t set_smem(int lpr, bool mat, size_t smem);
  static cudaError_t set_orth_smem(size_t smem);
};

cudaError_t launch_ls(const LsParams &p, int cluster, size_t smem, cudaStream_t s, bool pdl = false, int nprob = 1);
int ls_cluster_size(int s, int maxit, bool saz, int max_cluster = 16);
cudaError_t ls_allow_max_smem();
int wait_stream(cudaStream_t s);

// Row range of each of W warps, balanced by 4 * ceil(len / unit) + 1 per row,
// plus 4 * ceil(len / slot) when slot > 0.
int balance_rows(const StoredCsr &M, int unit, int W, int32_t *wrow, cudaStream_t s, int slot = 0, int extra = 0);
bool interleave_rows(const StoredCsr &M, int row_ctas);

// Row-major sparse-sign table (rows of S with their entries column | sign bit).
struct SketchTableTmp {
  uint32_t *kin = nullptr, *vin = nullptr, *kout = nullptr;
  void *cub = nullptr;
  size_t cub_bytes = 0;
};
int build_sketch_table(uint64_t seed, int s, int zeta, int64_t ncols, int32_t *rowptr, uint32_t *ent,
                       SketchTableTmp &t, int *err, cudaStream_t st);
size_t sketch_sort_bytes(int64_t nent, int s);
size_t ls_smem_bytes(int s, int maxit, int cluster, bool saz);
int ls_stage_plan(int s, int maxit, int cluster, bool saz);

void set_cuda_error(cudaError_t e, const char *where);
size_t dtype_size(int dt);
int load_width(int dt);

#define SFL_CU(...)                  \
  do {                               \
    cudaError_t e__ = (__VA_ARGS__); \
    if (e__ != cudaSuccess) {        \
      cudaGetLastError();            \
      ::sfl::set_cuda_error(e__, #__VA_ARGS__); \
      return SFL_ECUDA;              \
    }                                \
  } while (0)

}  // namespace sfl

struct sfl_plan {
  sfl::Plan impl;
};
