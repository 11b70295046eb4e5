// Instantiation + dispatch of step_kernel for one precision (included by
// step_fp64.cu / step_mixed.cu so the two precisions compile in parallel).
#pragma once

#include "step_kernel.cuh"

namespace nb {

enum StepOp { kLaunch = 0, kSetSmem = 1, kOccupancy = 2 };

// kLaunch: launch on `grid` CTAs.  kSetSmem: raise the kernel's dynamic
// shared-memory limit to `smem` (needed above 48 KB; done outside any stream
// capture).  kOccupancy: resident CTAs per SM at `smem` bytes, in *occ.
template <int PREC, int THREADS, int IPT>
static cudaError_t run_one(int op, int grid, size_t smem, const StepArgs &a, cudaStream_t s, int *occ) {
  auto k = step_kernel<PREC, THREADS, IPT>;
  if (op == kSetSmem)
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (op == kOccupancy) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, THREADS, smem);
  k<<<grid, THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int PREC>
static cudaError_t run_prec(int op, int threads, int ipt, int grid, size_t smem, const StepArgs &a, cudaStream_t s,
                            int *occ) {
#define NB_CASE(T, I) \
  if (threads == T && ipt == I) return run_one<PREC, T, I>(op, grid, smem, a, s, occ);
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
