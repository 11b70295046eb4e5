// FP64 instantiations of the Eq. 1 force kernel.
#include "step_launch.cuh"

namespace nb {
bool force_fp64_supported(int threads, int ipt) {
  return (ipt == 1 && (threads == 64 || threads == 128 || threads == 256 || threads == 512)) ||
         (ipt == 2 && (threads == 128 || threads == 256));
}
cudaError_t run_force_fp64(int op, int threads, int ipt, int grid, size_t smem, const ForceArgs &a, cudaStream_t s,
                           bool chained, int *occ) {
#define NB_CASE(T, I) \
  if (threads == T && ipt == I) return run_one<0, T, I>(op, grid, smem, a, s, chained, occ);
  NB_CASE(64, 1)
  NB_CASE(128, 1)
  NB_CASE(256, 1)
  NB_CASE(512, 1)
  NB_CASE(128, 2)
  NB_CASE(256, 2)
#undef NB_CASE
  return cudaErrorInvalidConfiguration;
}
}  // namespace nb
