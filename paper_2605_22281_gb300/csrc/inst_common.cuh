// Definitions of the typed launch wrappers; included by one .cu per precision pair.
#pragma once
#include "engine.h"

namespace sfl {

template <typename XT> __global__ void convert_in_kernel(const double *x, XT *y, int64_t n) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += st) y[i] = (XT)x[i];
}
template <typename XT> __global__ void convert_out_kernel(const XT *x, double *y, int64_t n) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += st) y[i] = (double)x[i];
}

// The product kernel for lanes per row `lpr`: the vector pass (mat false),
// the matrix form, or the matrix form writing through an original-row map
// (orig: pixel-tiled A^T / B rows); d16: the forms reading 16-bit column
// deltas (built for kDeltaLpr lanes per row only).
template <typename VT, typename XT, bool ORIG>
static void (*spmv_mat_fn(int lpr, bool d16))(SpmvParams<VT, XT>) {
  constexpr int M = ORIG ? kSpmvMatOrig : kSpmvMat;
  if (d16) return spmv_fused_kernel<VT, XT, kDeltaLpr, ORIG ? kSpmvMatOrig16 : kSpmvMat16>;
  if (lpr == 4) return spmv_fused_kernel<VT, XT, 4, M>;
  if (lpr == 8) return spmv_fused_kernel<VT, XT, 8, M>;
  if (lpr == 16) return spmv_fused_kernel<VT, XT, 16, M>;
  return spmv_fused_kernel<VT, XT, 32, M>;
}
template <typename VT, typename XT>
static void (*spmv_fn(int lpr, bool mat, bool orig, bool d16 = false))(SpmvParams<VT, XT>) {
  if (!mat) return spmv_fused_kernel<VT, XT, 1, kSpmvVec>;
  return orig ? spmv_mat_fn<VT, XT, true>(lpr, d16) : spmv_mat_fn<VT, XT, false>(lpr, d16);
}

template <typename VT, typename XT>
cudaError_t Ops<VT, XT>::spmv(const SpmvParams<VT, XT> &p, int lpr, bool mat, int grid, size_t smem, cudaStream_t s,
                              bool pdl) {
  if (mat && p.ptab)   // matrix-free projector
    return launch_k(spmv_fused_kernel<VT, XT, 32, kSpmvProj>, dim3(grid), dim3(kThreads), smem, s, pdl, p);
  const bool d16 = mat && p.dcol != nullptr && lpr == kDeltaLpr;
  return launch_k(spmv_fn<VT, XT>(lpr, mat, mat && p.orig != nullptr, d16), dim3(grid), dim3(kThreads), smem, s,
                  pdl, p);
}

template <typename VT, typename XT>
int Ops<VT, XT>::proj_occupancy(size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)spmv_fused_kernel<VT, XT, 32, kSpmvProj>,
                                                    kThreads, smem) != cudaSuccess)
    return 0;
  return nb;
}

// Both matrix forms (with and without the row map) get the same limit.
template <typename VT, typename XT>
cudaError_t Ops<VT, XT>::set_smem(int lpr, bool mat, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute((const void *)spmv_fn<VT, XT>(lpr, mat, false),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && mat && lpr == 32)
    e = cudaFuncSetAttribute((const void *)spmv_fused_kernel<VT, XT, 32, kSpmvProj>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && mat)
    e = cudaFuncSetAttribute((const void *)spmv_fn<VT, XT>(lpr, mat, true), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  for (int orig = 0; orig <= 1 && e == cudaSuccess && mat && lpr == kDeltaLpr; ++orig)
    e = cudaFuncSetAttribute((const void *)spmv_fn<VT, XT>(lpr, mat, orig != 0, true),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e;
}

template <typename VT, typename XT>
cudaError_t Ops<VT, XT>::set_orth_smem(size_t smem) {
  return cudaFuncSetAttribute((const void *)orth_update_kernel<XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

// Resident CTAs per SM of the product kernel (the smallest over the matrix forms).
template <typename VT, typename XT>
int Ops<VT, XT>::spmv_occupancy(int lpr, bool mat, size_t smem) {
  int best = 1 << 20;
  for (int form = 0; form < (mat ? (lpr == kDeltaLpr ? 4 : 2) : 1); ++form) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)spmv_fn<VT, XT>(lpr, mat, form & 1, form >= 2),
                                                      kThreads, smem) != cudaSuccess)
      return 0;
    best = std::min(best, nb);
  }
  return best;
}

template <typename VT, typename XT>
cudaError_t Ops<VT, XT>::orth(const OrthParams<XT> &p, int grid, size_t smem, cudaStream_t s, bool pdl) {
  return launch_k(orth_update_kernel<XT>, dim3(grid), dim3(kThreads), smem, s, pdl, p);
}

template <typename VT, typename XT>
cudaError_t Ops<VT, XT>::solution(SolveState *st, const XT *Z, int64_t zstride, const double *sigZ, const double *y,
                                  int64_t n, double *x, double *hist, int grid, cudaStream_t s) {
  solution_kernel<XT><<<grid, kThreads, 0, s>>>(st, Z, zstride, sigZ, y, n, x, hist);
  return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t Ops<VT, XT>::convert_in(const double *x, XT *y, int64_t n, cudaStream_t s) {
  convert_in_kernel<XT><<<1024, kThreads, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

template <typename VT, typename XT>
cudaError_t Ops<VT, XT>::convert_out(const XT *x, double *y, int64_t n, cudaStream_t s) {
  convert_out_kernel<XT><<<1024, kThreads, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

}  // namespace sfl
