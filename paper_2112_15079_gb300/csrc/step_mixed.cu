// Mixed-precision instantiations of the fused force + Verlet step kernel.
#include "step_launch.cuh"

namespace nb {
cudaError_t launch_step_mixed(int threads, int ipt, int grid, size_t smem, const StepArgs &a, cudaStream_t s) {
  return launch_prec<1>(threads, ipt, grid, smem, a, s);
}
}  // namespace nb
