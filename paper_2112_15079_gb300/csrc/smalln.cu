// Small systems (N <= kSmallMax, FP64, one system): every velocity-Verlet
// step of an nbody_step call inside ONE launch of one thread-block cluster.
//
// The Sun-plus-30-bodies model has 930 interactions per step; as separate
// launches a step costs two kernel launches for microseconds of work, and on
// a single SM GB300's 2-lane FP64 pipe needs ~4 us per step.  Here the
// cluster's CTAs (16, one per SM) each own up to kTargetsPerCta targets, one
// warp per target: the warp's 32 lanes split the sources, sum them in FP64
// and combine the lanes with a fixed-shape shuffle tree (deterministic).
// Every CTA keeps all positions in its shared memory (ping-pong); after the
// Eq. 3 drift each target's owner writes its new position into every CTA's
// copy through distributed shared memory, and one cluster barrier per step
// makes them visible.  Eq. 1 uses the same FP64 interaction as the general
// kernel (binomial-series refinement of the MUFU seed), Eqs. 3-4 the same
// kick/drift functions.
#include <cooperative_groups.h>

#include "nbody_dev.cuh"

namespace cg = cooperative_groups;

namespace nb {

namespace {

constexpr int kClusterCtas = 16;    // one CTA per SM (non-portable cluster size)
constexpr int kTargetsPerCta = 4;   // one warp each
constexpr int kSmallMax = kClusterCtas * kTargetsPerCta;

__global__ void __launch_bounds__(32 * kTargetsPerCta) smalln_kernel(const SmallArgs a) {
  __shared__ double4_32a pos[2][kSmallMax];  // (x, y, z, G m), a full copy per CTA
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = static_cast<int>(cluster.block_rank());
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.N;
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    pos[0][j] = make_double4_32a(a.x[j], a.y[j], a.z[j], a.G * a.m[j]);
  const int p = rank + kClusterCtas * warp;  // this warp's target (if < n)
  const bool own = p < n;
  double vx = 0, vy = 0, vz = 0, ax = 0, ay = 0, az = 0;
  if (own) {
    vx = a.vx[p];
    vy = a.vy[p];
    vz = a.vz[p];
    ax = a.ax[p];
    ay = a.ay[p];
    az = a.az[p];
  }
  cluster.sync();
  int b = 0;
  for (int64_t step = 0; step < a.n_steps; ++step) {
    // Eq. 3 drift of this warp's target, broadcast into every CTA's copy.
    if (own && lane < kClusterCtas) {
      const double4_32a r = pos[b][p];
      const double4_32a rn = make_double4_32a(drift(r.x, vx, ax, a.dt, a.half_dt2), drift(r.y, vy, ay, a.dt, a.half_dt2),
                                              drift(r.z, vz, az, a.dt, a.half_dt2), r.w);
      double4_32a *dst = cluster.map_shared_rank(&pos[1 - b][p], lane);
      *dst = rn;
    }
    cluster.sync();
    b ^= 1;
    // Eq. 1 at the new positions: lanes split the sources.
    double sx = 0, sy = 0, sz = 0;
    if (own) {
      const double4_32a me = pos[b][p];
      for (int j = lane; j < n; j += 32) {
        if (j == p) continue;
        interact_fp64<false>(pos[b][j], me.x, me.y, me.z, false, sx, sy, sz);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {  // fixed tree: lane l adds lane l + off
      sx += __shfl_down_sync(0xffffffffu, sx, off);
      sy += __shfl_down_sync(0xffffffffu, sy, off);
      sz += __shfl_down_sync(0xffffffffu, sz, off);
    }
    if (own) {
      sx = __shfl_sync(0xffffffffu, sx, 0);
      sy = __shfl_sync(0xffffffffu, sy, 0);
      sz = __shfl_sync(0xffffffffu, sz, 0);
      if (!finite3(sx, sy, sz) && lane == 0) atomicOr(a.flags, kFlagNonFinite);
      vx = kick(vx, ax, sx, a.half_dt);  // Eq. 4
      vy = kick(vy, ay, sy, a.half_dt);
      vz = kick(vz, az, sz, a.half_dt);
      ax = sx;
      ay = sy;
      az = sz;
    }
  }
  if (own && lane == 0) {
    const double4_32a r = pos[b][p];
    a.x[p] = r.x;
    a.y[p] = r.y;
    a.z[p] = r.z;
    a.vx[p] = vx;
    a.vy[p] = vy;
    a.vz[p] = vz;
    a.ax[p] = ax;
    a.ay[p] = ay;
    a.az[p] = az;
  }
  cluster.sync();  // no CTA leaves while others may still write into its shared memory
}

}  // namespace

int small_max_bodies() { return kSmallMax; }

cudaError_t small_prepare() {
  return cudaFuncSetAttribute(smalln_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

cudaError_t launch_small(const SmallArgs &a, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kClusterCtas);
  cfg.blockDim = dim3(32 * kTargetsPerCta);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, smalln_kernel, a);
}

}  // namespace nb
