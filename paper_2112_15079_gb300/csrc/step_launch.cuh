// Instantiation + dispatch of force_kernel for one precision (included by
// step_fp64.cu / step_mixed.cu so the two precisions compile in parallel).
#pragma once

#include "step_kernel.cuh"

namespace nb {

enum ForceOp { kLaunch = 0, kSetSmem = 1, kOccupancy = 2 };

// kLaunch: launch on `grid` CTAs (chained: programmatic stream
// serialization).  kSetSmem: raise the kernel's dynamic shared-memory limit
// to at least `smem` (needed above 48 KB; done outside any stream capture).
// The limit belongs to the kernel instance, which every context of the
// process shares, so it is only ever raised: a context that needs less must
// not take away what another one launches with.  (The caller serialises
// kSetSmem calls.)  kOccupancy: resident CTAs per SM at `smem` bytes, in *occ.
template <int PREC, int THREADS, int IPT>
static cudaError_t run_one(int op, int grid, size_t smem, const ForceArgs &a, cudaStream_t s, bool chained,
                           int *occ) {
  auto k = force_kernel<PREC, THREADS, IPT>;
  if (op == kSetSmem) {
    cudaFuncAttributes fa;
    const cudaError_t e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    if (static_cast<size_t>(fa.maxDynamicSharedSizeBytes) >= smem) return cudaSuccess;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  }
  if (op == kOccupancy) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, THREADS, smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace nb
