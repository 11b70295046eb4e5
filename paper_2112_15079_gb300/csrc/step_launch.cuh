// Instantiation + dispatch of step_kernel for one precision (included by
// step_fp64.cu / step_mixed.cu so the two precisions compile in parallel).
#pragma once

#include "step_kernel.cuh"

namespace nb {

// grid == 0: no launch, only raise the kernel's dynamic shared-memory limit
// to `smem` (needed above 48 KB; done outside any stream capture).
template <int PREC, int THREADS, int IPT>
static cudaError_t launch_one(int grid, size_t smem, const StepArgs &a, cudaStream_t s) {
  auto k = step_kernel<PREC, THREADS, IPT>;
  if (grid == 0)
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  k<<<grid, THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int PREC>
static cudaError_t launch_prec(int threads, int ipt, int grid, size_t smem, const StepArgs &a, cudaStream_t s) {
#define NB_CASE(T, I) \
  if (threads == T && ipt == I) return launch_one<PREC, T, I>(grid, smem, a, s);
  NB_CASE(64, 1)
  NB_CASE(64, 2)
  NB_CASE(64, 4)
  NB_CASE(128, 1)
  NB_CASE(128, 2)
  NB_CASE(128, 4)
  NB_CASE(256, 1)
  NB_CASE(256, 2)
  NB_CASE(256, 4)
#undef NB_CASE
  return cudaErrorInvalidConfiguration;
}

}  // namespace nb
