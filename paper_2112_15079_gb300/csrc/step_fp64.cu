// FP64 instantiations of the fused force + Verlet step kernel.
#include "step_launch.cuh"

namespace nb {
cudaError_t launch_step_fp64(int threads, int ipt, int grid, size_t smem, const StepArgs &a, cudaStream_t s) {
  return launch_prec<0>(threads, ipt, grid, smem, a, s);
}
}  // namespace nb
