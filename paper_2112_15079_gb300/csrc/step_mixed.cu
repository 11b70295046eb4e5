// Mixed-precision instantiations of the Eq. 1 force kernel.
#include "step_launch.cuh"

namespace nb {
bool force_mixed_supported(int threads, int ipt) {
  return (ipt == 1 && (threads == 128 || threads == 256 || threads == 512 || threads == 1024)) ||
         (ipt == 2 && (threads == 256 || threads == 384 || threads == 512 || threads == 768)) ||
         (ipt == 4 && (threads == 128 || threads == 256));
}
cudaError_t run_force_mixed(int op, int threads, int ipt, int grid, size_t smem, const ForceArgs &a, cudaStream_t s,
                            bool chained, int *occ) {
#define NB_CASE(T, I) \
  if (threads == T && ipt == I) return run_one<1, T, I>(op, grid, smem, a, s, chained, occ);
  NB_CASE(128, 1)
  NB_CASE(256, 1)
  NB_CASE(512, 1)
  NB_CASE(1024, 1)
  NB_CASE(256, 2)
  NB_CASE(384, 2)
  NB_CASE(512, 2)
  NB_CASE(768, 2)
  NB_CASE(128, 4)
  NB_CASE(256, 4)
#undef NB_CASE
  return cudaErrorInvalidConfiguration;
}
}  // namespace nb
