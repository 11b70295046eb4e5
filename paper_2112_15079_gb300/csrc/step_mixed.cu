// Mixed-precision instantiations of the fused force + Verlet step kernel.
#include "step_launch.cuh"

namespace nb {
cudaError_t run_step_mixed(int op, int threads, int ipt, int grid, size_t smem, const StepArgs &a, cudaStream_t s,
                           int *occ) {
  return run_prec<1>(op, threads, ipt, grid, smem, a, s, occ);
}
}  // namespace nb
