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

template <typename VT, typename XT>
static const void *spmv_fn(int lpr, bool mat) {
  if (!mat) return (const void *)spmv_fused_kernel<VT, XT, 1, false>;
  if (lpr == 4) return (const void *)spmv_fused_kernel<VT, XT, 4, true>;
  if (lpr == 8) return (const void *)spmv_fused_kernel<VT, XT, 8, true>;
  if (lpr == 16) return (const void *)spmv_fused_kernel<VT, XT, 16, true>;
  return (const void *)spmv_fused_kernel<VT, XT, 32, true>;
}

template <typename VT, typename XT>
cudaError_t Ops<VT, XT>::spmv(const SpmvParams<VT, XT> &p, int lpr, bool mat, int grid, size_t smem, cudaStream_t s,
                              bool pdl) {
  void (*kern)(SpmvParams<VT, XT>);
  if (!mat) kern = spmv_fused_kernel<VT, XT, 1, false>;
  else if (lpr == 4) kern = spmv_fused_kernel<VT, XT, 4, true>;
  else if (lpr == 8) kern = spmv_fused_kernel<VT, XT, 8, true>;
  else if (lpr == 16) kern = spmv_fused_kernel<VT, XT, 16, true>;
  else kern = spmv_fused_kernel<VT, XT, 32, true>;
  return launch_k(kern, dim3(grid), dim3(kThreads), smem, s, pdl, p);
}

template <typename VT, typename XT>
cudaError_t Ops<VT, XT>::set_smem(int lpr, bool mat, size_t smem) {
  return cudaFuncSetAttribute(spmv_fn<VT, XT>(lpr, mat), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename VT, typename XT>
cudaError_t Ops<VT, XT>::set_orth_smem(size_t smem) {
  return cudaFuncSetAttribute((const void *)orth_update_kernel<XT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

template <typename VT, typename XT>
int Ops<VT, XT>::spmv_occupancy(int lpr, bool mat, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, spmv_fn<VT, XT>(lpr, mat), kThreads, smem) != cudaSuccess)
    return 0;
  return nb;
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
