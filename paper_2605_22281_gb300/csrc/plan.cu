// Plans: validation, precision conversion, row padding and the transposed copy
// of A (one-time set-up; the per-step kernels are in kernels.cuh).
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "engine.h"

namespace sfl {

static thread_local std::string g_last_cuda_error;

void set_cuda_error(cudaError_t e, const char *where) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
  g_last_cuda_error = buf;
}

const char *last_cuda_error() { return g_last_cuda_error.c_str(); }

size_t dtype_size(int dt) { return dt == SFL_F64 ? 8 : dt == SFL_F32 ? 4 : 2; }
int load_width(int dt) { return dt == SFL_BF16 ? 8 : 4; }

// ---------------------------------------------------------------- device helpers

enum : int { kErrRowptr = 1, kErrCol = 2, kErrNonfinite = 4 };

__global__ void validate_kernel(const int32_t *rowptr, const int32_t *col, const void *val, int dt, int64_t rows,
                                int64_t cols, int64_t nnz, int *err) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int e = 0;
  for (int64_t i = t0; i < rows; i += st) {
    if (rowptr[i] > rowptr[i + 1] || rowptr[i] < 0) e |= kErrRowptr;
  }
  if (t0 == 0 && (rowptr[0] != 0 || (int64_t)rowptr[rows] != nnz)) e |= kErrRowptr;
  for (int64_t i = t0; i < nnz; i += st) {
    const int c = col[i];
    if (c < 0 || (int64_t)c >= cols) e |= kErrCol;
    double v;
    if (dt == SFL_F64) v = ((const double *)val)[i];
    else if (dt == SFL_F32) v = ((const float *)val)[i];
    else v = __bfloat162float(((const __nv_bfloat16 *)val)[i]);
    if (!isfinite(v)) e |= kErrNonfinite;
  }
  if (e) atomicOr(err, e);
}

template <typename OT>
__device__ __forceinline__ OT cvt(double v);
template <> __device__ __forceinline__ double cvt<double>(double v) { return v; }
template <> __device__ __forceinline__ float cvt<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

template <typename OT>
__global__ void convert_values_kernel(const void *in, int dt, OT *out, int64_t n) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += st) {
    double v;
    if (dt == SFL_F64) v = ((const double *)in)[i];
    else if (dt == SFL_F32) v = ((const float *)in)[i];
    else v = __bfloat162float(((const __nv_bfloat16 *)in)[i]);
    out[i] = cvt<OT>(v);
  }
}

// Padded length of stored row i, which is row order[i] of the input (order
// nullptr: row i).
__global__ void padded_len_kernel(const int32_t *rowptr, int64_t rows, int P, const int32_t *order, int32_t *plen) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= rows; i += st) {
    if (i == rows) { plen[i] = 0; continue; }
    const int64_t src = order ? order[i] : i;
    const int len = rowptr[src + 1] - rowptr[src];
    plen[i] = (len + P - 1) / P * P;
  }
}

// One warp per stored row: copy input row order[r] (or r) into its padded
// slot.  Padding entries take the row's last column (or 0 for an empty row)
// and value 0.  Inside every chunk slot of str = lanes * P entries (the last
// one holding A = its length / P lanes' chunks) entry w goes to position
// (w mod A) * P + w / A: lane g's P-entry chunk holds entries g, g + A, ...
// of the slot, so the lanes of one gather instruction read consecutive
// entries of the row (neighbouring pixels along a ray share cache sectors).
// str = 0 keeps the caller's order.
template <typename OT>
__global__ void fill_padded_kernel(const int32_t *rowptr, const int32_t *col, const OT *val, int64_t rows,
                                   const int32_t *order, const int32_t *prow, int P, int str, int32_t *pcol,
                                   OT *pval) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < rows; r += nw) {
    const int64_t src = order ? order[r] : r;
    const int b = rowptr[src], e = rowptr[src + 1], pb = prow[r], pe = prow[r + 1];
    const int last = e > b ? col[e - 1] : 0;
    const int plen = pe - pb;
    for (int i = lane; i < plen; i += 32) {
      int d = pb + i;                       // str == 0: the caller's order
      if (str > 0) {
        const int slot0 = i / str * str, w = i - slot0;
        const int A = min(str, plen - slot0) / P;
        d = pb + slot0 + (w % A) * P + w / A;
      }
      if (b + i < e) { pcol[d] = col[b + i]; pval[d] = val[b + i]; }
      else { pcol[d] = last; pval[d] = cvt<OT>(0.0); }
    }
  }
}

// 16-bit column deltas of a lane-interleaved padded CSR (slots of str = lpr * P
// entries, chunk c of a slot at c * P): the entry at chunk position q > 0
// follows position q - 1 of the same chunk; position 0 of chunk c in slot k > 0
// follows the last position of chunk c in slot k - 1 (full, since only a row's
// last slot is short); position 0 of chunk c in slot 0 follows the row's base,
// the column of its first stored entry.  *overflow is set when a delta does
// not fit in 16 bits.
__global__ void delta_cols_kernel(const int32_t *prow, const int32_t *pcol, int64_t rows, int P, int str,
                                  int16_t *dcol, int32_t *rbase, int *overflow) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < rows; r += nw) {
    const int pb = prow[r], pe = prow[r + 1];
    const int base = pe > pb ? pcol[pb] : 0;
    if (lane == 0) rbase[r] = base;
    for (int i = lane; i < pe - pb; i += 32) {
      const int k = i / str, w = i - k * str, c = w / P, q = w - c * P;
      const int prev = q > 0 ? pcol[pb + i - 1] : (k > 0 ? pcol[pb + (k - 1) * str + c * P + P - 1] : base);
      const int d = pcol[pb + i] - prev;
      if (d < -32768 || d > 32767) atomicOr(overflow, 1);
      dcol[pb + i] = (int16_t)d;
    }
  }
}

__global__ void row_ids_kernel(const int32_t *rowptr, int64_t rows, int32_t *rid) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < rows; r += nw)
    for (int i = rowptr[r] + lane; i < rowptr[r + 1]; i += 32) rid[i] = (int32_t)r;
}

__global__ void iota_kernel(int32_t *v, int64_t n) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += st) v[i] = (int32_t)i;
}

// Transposed row pointer: first position of each column in the sorted keys.
__global__ void bounds_kernel(const int32_t *keys, int64_t nnz, int64_t cols, int32_t *trow) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= cols; c += st) {
    int64_t lo = 0, hi = nnz;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)keys[mid] < c) lo = mid + 1; else hi = mid;
    }
    trow[c] = (int32_t)lo;
  }
}

template <typename OT>
__global__ void gather_transpose_kernel(const int32_t *perm, const int32_t *rid, const OT *val, int64_t nnz,
                                        int32_t *tcol, OT *tval) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz; i += st) {
    const int32_t j = perm[i];
    tcol[i] = rid[j];
    tval[i] = val[j];
  }
}

// ---------------------------------------------------------------- host helpers

struct TmpAlloc {
  std::vector<void *> ptrs;
  ~TmpAlloc() { for (void *p : ptrs) cudaFree(p); }
  template <typename T> cudaError_t get(T **p, size_t bytes) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e == cudaSuccess) ptrs.push_back(q);
    *p = (T *)q;
    return e;
  }
};

static int plan_alloc(Plan &pl, void **p, size_t bytes) {
  if (pl.cap && pl.bytes + bytes > pl.cap) return SFL_ENOMEM;
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_cuda_error(e, "cudaMalloc");
    return SFL_ENOMEM;
  }
  pl.allocs.push_back(*p);
  pl.bytes += bytes;
  return SFL_OK;
}

// Give back an allocation of plan_alloc before the plan is complete.
static void plan_free(Plan &pl, void *p, size_t bytes) {
  for (size_t i = 0; i < pl.allocs.size(); ++i)
    if (pl.allocs[i] == p) {
      pl.allocs.erase(pl.allocs.begin() + (long)i);
      cudaFree(p);
      pl.bytes -= bytes;
      return;
    }
}

static int validate_csr(const sfl_csr *M, cudaStream_t s) {
  if (!M || M->rows < 0 || M->cols <= 0 || M->nnz < 0 || M->nnz >= (int64_t)1 << 31 || M->rows >= (int64_t)1 << 31 ||
      M->cols >= (int64_t)1 << 31 || !M->rowptr || (M->nnz > 0 && (!M->colidx || !M->values)) ||
      (M->dtype != SFL_F64 && M->dtype != SFL_F32 && M->dtype != SFL_BF16))
    return SFL_EINVAL;
  if (M->rows == 0) return SFL_EINVAL;
  TmpAlloc tmp;
  int *err = nullptr;
  SFL_CU(tmp.get(&err, sizeof(int)));
  SFL_CU(cudaMemsetAsync(err, 0, sizeof(int), s));
  validate_kernel<<<1024, 256, 0, s>>>(M->rowptr, M->colidx, M->values, M->dtype, M->rows, M->cols, M->nnz, err);
  SFL_CU(cudaGetLastError());
  int h = 0;
  SFL_CU(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SFL_CU(cudaStreamSynchronize(s));
  if (h & (kErrRowptr | kErrCol)) return SFL_EINVAL;
  if (h & kErrNonfinite) return SFL_ENONFINITE;
  return SFL_OK;
}

// Lanes per row: 8, or 16 only for rows long enough to give every lane of 16
// at least 48 P-wide loads (no CT operator here comes near).  Measured on the
// 1024^2 operator (921 entries per ray): 8 lanes ran A z in 1138 us against
// 1392 us at 16 in FP64, 782 against 854 us in FP32, 675 against 760 us in
// BF16; on operators of 230 to 460 entries per row 8 was the fastest too, and
// 32 the slowest everywhere.
static int choose_lpr(int64_t pnnz, int64_t rows, int P) {
  const double avg = rows > 0 ? (double)pnnz / (double)rows : 0.0;
  return avg >= 48.0 * P * 16 ? 16 : 8;
}

// Row order of 16 x 16 pixel tiles (tiles and the pixels inside one in
// row-major order) for an image_rows x image_cols n-side.
static std::vector<int32_t> tile_order(int rows, int cols) {
  constexpr int kTile = 16;
  std::vector<int32_t> o;
  o.reserve((size_t)rows * cols);
  for (int ty = 0; ty < rows; ty += kTile)
    for (int tx = 0; tx < cols; tx += kTile)
      for (int iy = ty; iy < std::min(rows, ty + kTile); ++iy)
        for (int ix = tx; ix < std::min(cols, tx + kTile); ++ix) o.push_back(iy * cols + ix);
  return o;
}

// Pad (rowptr, col, val[OT]) into plan-owned storage, rows in the plan's
// tile order when `tiled` (the n-side image shape is known).
template <typename OT>
static int store_padded(Plan &pl, StoredCsr &out, const int32_t *rowptr, const int32_t *col, const OT *val,
                        int64_t rows, int64_t cols, int64_t nnz, cudaStream_t s, bool tiled = false) {
  const int P = load_width(pl.vdt);
  TmpAlloc tmp;
  int r;
  if (tiled) {
    const std::vector<int32_t> o = tile_order(pl.img_rows, pl.img_cols);
    if ((int64_t)o.size() != rows) return SFL_EINVAL;
    if ((r = plan_alloc(pl, (void **)&out.orig, sizeof(int32_t) * rows))) return r;
    SFL_CU(cudaMemcpyAsync(out.orig, o.data(), sizeof(int32_t) * rows, cudaMemcpyHostToDevice, s));
    SFL_CU(cudaStreamSynchronize(s));
  }
  int32_t *plen = nullptr;
  SFL_CU(tmp.get(&plen, sizeof(int32_t) * (rows + 1)));
  padded_len_kernel<<<1024, 256, 0, s>>>(rowptr, rows, P, out.orig, plen);
  SFL_CU(cudaGetLastError());
  if ((r = plan_alloc(pl, (void **)&out.rowptr, sizeof(int32_t) * (rows + 1)))) return r;
  size_t tb = 0;
  SFL_CU(cub::DeviceScan::ExclusiveSum(nullptr, tb, plen, out.rowptr, (int)(rows + 1), s));
  void *tst = nullptr;
  SFL_CU(tmp.get(&tst, tb));
  SFL_CU(cub::DeviceScan::ExclusiveSum(tst, tb, plen, out.rowptr, (int)(rows + 1), s));
  int32_t pnnz32 = 0;
  SFL_CU(cudaMemcpyAsync(&pnnz32, out.rowptr + rows, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  SFL_CU(cudaStreamSynchronize(s));
  const int64_t pnnz = pnnz32;
  if (pnnz < nnz) return SFL_EINVAL;   // padded count overflowed int32
  if ((r = plan_alloc(pl, (void **)&out.col, sizeof(int32_t) * (pnnz + 8)))) return r;
  if ((r = plan_alloc(pl, (void **)&out.val, sizeof(OT) * (pnnz + 8)))) return r;
  out.rows = rows; out.cols = cols; out.nnz = nnz; out.pnnz = pnnz;
  out.lpr = pl.lpr_override ? pl.lpr_override : choose_lpr(pnnz, rows, P);
  if (rows > 0) {
    out.interleaved = pl.slot_layout == 0;
    fill_padded_kernel<OT><<<2048, 256, 0, s>>>(rowptr, col, val, rows, out.orig, out.rowptr, P,
                                                 out.interleaved ? out.lpr * P : 0, out.col, (OT *)out.val);
    SFL_CU(cudaGetLastError());
  }
  return SFL_OK;
}

// 16-bit column deltas of a stored operator for the single-solve products,
// built once both operators are stored: kept only if every delta fits, and
// left out (not an error) when they would exceed the plan's device-byte cap
// or the device has no room for them.
static int build_deltas(Plan &pl, StoredCsr &M, cudaStream_t s) {
  const int P = load_width(pl.vdt);
  const int64_t rows = M.rows, pnnz = M.pnnz;
  const size_t dbytes = sizeof(int16_t) * (pnnz + 16) + sizeof(int32_t) * rows;
  if (rows <= 0 || !M.interleaved || M.lpr != kDeltaLpr || pl.index_bits != 0 || (pl.cap && pl.bytes + dbytes > pl.cap))
    return SFL_OK;
  TmpAlloc tmp;
  int *ovf = nullptr;
  SFL_CU(tmp.get(&ovf, sizeof(int)));
  SFL_CU(cudaMemsetAsync(ovf, 0, sizeof(int), s));
  if (plan_alloc(pl, (void **)&M.dcol, sizeof(int16_t) * (pnnz + 16))) {
    M.dcol = nullptr;
    return SFL_OK;
  }
  if (plan_alloc(pl, (void **)&M.rbase, sizeof(int32_t) * rows)) {
    plan_free(pl, M.dcol, sizeof(int16_t) * (pnnz + 16));
    M.dcol = nullptr;
    M.rbase = nullptr;
    return SFL_OK;
  }
  SFL_CU(cudaMemsetAsync(M.dcol, 0, sizeof(int16_t) * (pnnz + 16), s));
  delta_cols_kernel<<<2048, 256, 0, s>>>(M.rowptr, M.col, rows, P, M.lpr * P, M.dcol, M.rbase, ovf);
  SFL_CU(cudaGetLastError());
  int h = 0;
  SFL_CU(cudaMemcpyAsync(&h, ovf, sizeof(int), cudaMemcpyDeviceToHost, s));
  SFL_CU(cudaStreamSynchronize(s));
  if (h) {   // some delta does not fit: the products read the 32-bit indices
    plan_free(pl, M.dcol, sizeof(int16_t) * (pnnz + 16));
    plan_free(pl, M.rbase, sizeof(int32_t) * rows);
    M.dcol = nullptr;
    M.rbase = nullptr;
  }
  return SFL_OK;
}

template <typename OT>
static int build_plan(Plan &pl, const sfl_csr *A, const sfl_csr *B, cudaStream_t s) {
  TmpAlloc tmp;
  OT *aval = nullptr;
  SFL_CU(tmp.get(&aval, sizeof(OT) * (A->nnz + 1)));
  if (A->nnz) {
    convert_values_kernel<OT><<<2048, 256, 0, s>>>(A->values, A->dtype, aval, A->nnz);
    SFL_CU(cudaGetLastError());
  }
  int r = store_padded<OT>(pl, pl.A, A->rowptr, A->colidx, aval, A->rows, A->cols, A->nnz, s);
  if (r) return r;
  if (B) {
    OT *bval = nullptr;
    SFL_CU(tmp.get(&bval, sizeof(OT) * (B->nnz + 1)));
    if (B->nnz) {
      convert_values_kernel<OT><<<2048, 256, 0, s>>>(B->values, B->dtype, bval, B->nnz);
      SFL_CU(cudaGetLastError());
    }
    r = store_padded<OT>(pl, pl.T, B->rowptr, B->colidx, bval, B->rows, B->cols, B->nnz, s, pl.img_rows > 0);
    SFL_CU(cudaStreamSynchronize(s));
    return r;
  }
  // Transposed copy: stable radix sort of the entries by column keeps the
  // row order inside each column, so the CSR of A^T is fully deterministic
  // and carries exactly the rounded values of the stored A.
  const int64_t nnz = A->nnz;
  int32_t *rid, *keys_out, *iota, *perm, *trow, *tcol;
  OT *tval;
  SFL_CU(tmp.get(&rid, sizeof(int32_t) * (nnz + 1)));
  SFL_CU(tmp.get(&keys_out, sizeof(int32_t) * (nnz + 1)));
  SFL_CU(tmp.get(&iota, sizeof(int32_t) * (nnz + 1)));
  SFL_CU(tmp.get(&perm, sizeof(int32_t) * (nnz + 1)));
  SFL_CU(tmp.get(&trow, sizeof(int32_t) * (A->cols + 1)));
  SFL_CU(tmp.get(&tcol, sizeof(int32_t) * (nnz + 1)));
  SFL_CU(tmp.get(&tval, sizeof(OT) * (nnz + 1)));
  if (nnz) {
    row_ids_kernel<<<2048, 256, 0, s>>>(A->rowptr, A->rows, rid);
    iota_kernel<<<2048, 256, 0, s>>>(iota, nnz);
    SFL_CU(cudaGetLastError());
    int bits = 1;
    while (((int64_t)1 << bits) < A->cols) ++bits;
    size_t tb = 0;
    SFL_CU(cub::DeviceRadixSort::SortPairs(nullptr, tb, A->colidx, keys_out, iota, perm, (int)nnz, 0, bits, s));
    void *tst = nullptr;
    SFL_CU(tmp.get(&tst, tb));
    SFL_CU(cub::DeviceRadixSort::SortPairs(tst, tb, A->colidx, keys_out, iota, perm, (int)nnz, 0, bits, s));
    gather_transpose_kernel<OT><<<2048, 256, 0, s>>>(perm, rid, aval, nnz, tcol, tval);
    SFL_CU(cudaGetLastError());
  }
  bounds_kernel<<<1024, 256, 0, s>>>(keys_out, nnz, A->cols, trow);
  SFL_CU(cudaGetLastError());
  r = store_padded<OT>(pl, pl.T, trow, tcol, tval, A->cols, A->rows, nnz, s, pl.img_rows > 0);
  SFL_CU(cudaStreamSynchronize(s));
  return r;
}

}  // namespace sfl

using namespace sfl;

extern "C" {

const char *sfl_error_string(int status) {
  switch (status) {
    case SFL_OK: return "ok";
    case SFL_EINVAL: return "invalid argument";
    case SFL_ENOMEM: return "out of device memory (or over the plan's cap)";
    case SFL_ECUDA: return "CUDA runtime error";
    case SFL_ENONFINITE: return "NaN or Inf in the input";
    case SFL_ETIMEOUT: return "host wait timed out";
    case SFL_EUNSUPPORTED: return "unsupported by the library";
    default: return "unknown status";
  }
}

const char *sfl_last_cuda_error(void) { return last_cuda_error(); }

int sfl_plan_create(sfl_plan **plan, const sfl_csr *A, const sfl_csr *B, const sfl_plan_opts *popts,
                    sfl_stream stream) {
  if (!plan) return SFL_EINVAL;
  *plan = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  int r = validate_csr(A, s);
  if (r) return r;
  if (B) {
    if ((r = validate_csr(B, s))) return r;
    if (B->rows != A->cols || B->cols != A->rows) return SFL_EINVAL;
  }
  const sfl_dtype vdt = popts ? popts->value_dtype : SFL_F64;
  if (vdt != SFL_F64 && vdt != SFL_F32 && vdt != SFL_BF16) return SFL_EINVAL;
  const int lpr = popts ? popts->lanes_per_row : 0;
  if (lpr != 0 && lpr != 4 && lpr != 8 && lpr != 16 && lpr != 32) return SFL_EINVAL;
  const int img_r = popts ? popts->image_rows : 0, img_c = popts ? popts->image_cols : 0;
  if (img_r < 0 || img_c < 0 || (img_r == 0) != (img_c == 0)) return SFL_EINVAL;
  if (img_r > 0 && (int64_t)img_r * img_c != A->cols) return SFL_EINVAL;
  const int layout = popts ? popts->slot_layout : 0;
  if (layout != 0 && layout != 1) return SFL_EINVAL;
  const int ibits = popts ? popts->index_bits : 0;
  if (ibits != 0 && ibits != 32) return SFL_EINVAL;
  sfl_plan *p = new sfl_plan();
  Plan &pl = p->impl;
  cudaGetDevice(&pl.device);
  cudaDeviceGetAttribute(&pl.num_sms, cudaDevAttrMultiProcessorCount, pl.device);
  pl.vdt = vdt;
  pl.unmatched = B != nullptr;
  pl.lpr_override = lpr;
  pl.img_rows = img_r; pl.img_cols = img_c;
  pl.slot_layout = layout;
  pl.index_bits = ibits;
  pl.cap = popts ? popts->max_device_bytes : 0;
  if (vdt == SFL_F64) r = build_plan<double>(pl, A, B, s);
  else if (vdt == SFL_F32) r = build_plan<float>(pl, A, B, s);
  else r = build_plan<__nv_bfloat16>(pl, A, B, s);
  if (!r) r = build_deltas(pl, pl.A, s);
  if (!r) r = build_deltas(pl, pl.T, s);
  if (r) {
    sfl_plan_destroy(p);
    return r;
  }
  *plan = p;
  return SFL_OK;
}

int sfl_plan_create_ct(sfl_plan **plan, const sfl_ct_geometry *g, const sfl_plan_opts *popts, sfl_stream stream) {
  if (!plan || !g) return SFL_EINVAL;
  *plan = nullptr;
  if (g->image_n < 1 || g->n_angles < 1 || g->n_bins < 1 || (g->back != 0 && g->back != 1)) return SFL_EINVAL;
  const int64_t n = (int64_t)g->image_n * g->image_n, m = (int64_t)g->n_angles * g->n_bins;
  if (n >= (int64_t)1 << 31 || m >= (int64_t)1 << 31) return SFL_EINVAL;
  const sfl_dtype vdt = popts ? popts->value_dtype : SFL_F64;
  if (vdt != SFL_F64 && vdt != SFL_F32 && vdt != SFL_BF16) return SFL_EINVAL;
  // per-angle constants (host, FP64): cos, sin, trapezoid a1, a2, H, slope, axis flag,
  // the direction's reciprocals -1/sin and 1/cos
  std::vector<double> tab((size_t)kProjTab * g->n_angles);
  for (int a = 0; a < g->n_angles; ++a) {
    const double th = (double)a * M_PI / (double)g->n_angles;
    const double c = g->angles_cs ? g->angles_cs[2 * a] : cos(th), s = g->angles_cs ? g->angles_cs[2 * a + 1] : sin(th);
    if (!std::isfinite(c) || !std::isfinite(s)) return SFL_EINVAL;
    const double ac = fabs(c), as = fabs(s);
    const double a1 = 0.5 * fabs(ac - as), a2 = 0.5 * (ac + as), H = 1.0 / std::max(ac, as);
    double *e = tab.data() + (size_t)kProjTab * a;
    e[0] = c; e[1] = s; e[2] = a1; e[3] = a2; e[4] = H;
    e[5] = a2 - a1 > 1e-15 ? H / (a2 - a1) : 0.0;
    e[6] = as < 1e-15 ? 1.0 : (ac < 1e-15 ? 2.0 : 0.0);
    e[7] = as > 1e-15 ? -1.0 / s : 0.0;
    e[8] = ac > 1e-15 ? 1.0 / c : 0.0;
  }
  sfl_plan *p = new sfl_plan();
  Plan &pl = p->impl;
  cudaGetDevice(&pl.device);
  cudaDeviceGetAttribute(&pl.num_sms, cudaDevAttrMultiProcessorCount, pl.device);
  pl.vdt = vdt == SFL_F64 ? SFL_F64 : SFL_F32;   // no stored values: BF16 means FP32 arithmetic
  pl.unmatched = g->back == 1;
  pl.matfree = true;
  pl.ct_N = g->image_n; pl.ct_na = g->n_angles; pl.ct_nb = g->n_bins; pl.ct_back = g->back;
  pl.img_rows = pl.img_cols = g->image_n;
  pl.cap = popts ? popts->max_device_bytes : 0;
  pl.A.rows = m; pl.A.cols = n; pl.A.lpr = 32;
  pl.T.rows = n; pl.T.cols = m; pl.T.lpr = 32;
  cudaStream_t s = (cudaStream_t)stream;
  int r = SFL_OK;
  std::vector<long long> fix(g->n_angles);
  if (pl.vdt == SFL_F64) {
    const int F = proj_bin_frac_bits(g->n_bins);
    for (int a = 0; a < g->n_angles; ++a) fix[a] = std::llround(std::ldexp(tab[(size_t)kProjTab * a], F));
    r = plan_alloc(pl, &pl.ct_tab, sizeof(double) * tab.size());
    if (!r && cudaMemcpyAsync(pl.ct_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
      r = SFL_ECUDA;
    if (!r) r = plan_alloc(pl, (void **)&pl.ct_fix, sizeof(long long) * fix.size());
    if (!r && cudaMemcpyAsync(pl.ct_fix, fix.data(), sizeof(long long) * fix.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
      r = SFL_ECUDA;
  } else {
    std::vector<float> tf(tab.begin(), tab.end());
    r = plan_alloc(pl, &pl.ct_tab, sizeof(float) * tf.size());
    if (!r && cudaMemcpyAsync(pl.ct_tab, tf.data(), sizeof(float) * tf.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
      r = SFL_ECUDA;
  }
  if (!r && cudaStreamSynchronize(s) != cudaSuccess) r = SFL_ECUDA;
  if (r) {
    cudaGetLastError();
    sfl_plan_destroy(p);
    return r;
  }
  *plan = p;
  return SFL_OK;
}

int sfl_plan_get_stats(const sfl_plan *plan, sfl_plan_stats *st) {
  if (!plan || !st) return SFL_EINVAL;
  const Plan &pl = plan->impl;
  st->rows = pl.A.rows; st->cols = pl.A.cols;
  st->nnz_A = pl.A.nnz; st->nnz_At = pl.T.nnz;
  st->padded_nnz_A = pl.A.pnnz; st->padded_nnz_At = pl.T.pnnz;
  st->lanes_A = pl.A.lpr; st->lanes_At = pl.T.lpr;
  st->value_dtype = pl.vdt; st->unmatched = pl.unmatched ? 1 : 0;
  st->device_bytes = pl.bytes;
  st->tiled_At = pl.T.orig != nullptr ? 1 : 0;
  st->matrix_free = pl.matfree ? 1 : 0;
  st->index_bytes_A = pl.A.dcol ? 2 : 4;
  st->index_bytes_At = pl.T.dcol ? 2 : 4;
  return SFL_OK;
}

}  // extern "C"
