// Small systems (N <= kSmallMax, FP64, one system): every velocity-Verlet
// step of an nbody_step call inside ONE launch of one thread-block cluster.
//
// The Sun-plus-30-bodies model has 930 interactions per step; as separate
// launches a step costs two kernel launches for microseconds of work.  Here
// the cluster's CTAs (8 for N <= 32, else 16; one per SM) own the targets,
// one warp per target (4 warps per CTA up to 64 bodies, then ceil(N / 16), at
// most kMaxWarps): the warp's 32 lanes split the sources and sum them in
// FP64.  Up to kSmallMax = 256 bodies this beats the general two-kernel path,
// which spreads the pairs over every SM but pays two launches and the
// partial-row sums per step (measured: 8.5x at 31 bodies, 2.7x at 131, 1.3x
// at 256).  Every CTA keeps all positions in its shared
// memory (ping-pong buffers pos[0], pos[1]).  Eq. 1 uses the same FP64
// interaction as the general kernel (binomial-series refinement of the MUFU
// seed), Eqs. 3-4 the same kick/drift functions.
//
// Exchange.  After the Eq. 3 drift each target's owner pushes its new
// position into the copy of every CTA that owns a target, with st.async,
// each store completing 8 bytes of a transaction on the receiving CTA's
// mbarrier for that buffer; a CTA reads the buffer once the barrier's phase
// completes (24 N bytes: every component of every target).  There is no
// cluster-wide barrier per step: a store is one-way.  Only warps that own a
// target take part, and every one of them is waited for by all the others.
// Reuse is then safe: a warp writes a peer's buffer for step k+2 only after
// its own wait for step k+1 completed, which needs every owner's step-(k+1)
// stores, issued after that owner finished reading its buffer at step k
// (the stored values depend on those reads).  For the same reason no owner
// can be two phases behind another, so a wait on the phase parity
// (step / 2) mod 2 is unambiguous.  Waits are bounded (kWaitPolls); a wait
// that runs out sets kFlagTimeout and the kernel winds down.
//
// At this size a step is a chain of dependent FP64 instructions, and GB300's
// FP64 pipe takes 64 cycles for every warp instruction whatever its active
// mask; the step is therefore written to issue as few as possible.  The
// three components share instructions: the 32 lane sums are combined by a
// butterfly reduce-scatter that leaves component c in lanes 8c..8c+7 (six
// FP64 additions for all three components instead of fifteen), and those
// lanes then apply Eqs. 3-4 to their component alone (two instructions each
// instead of six).  The butterfly pairs the same lane sets at each level as a
// plain shuffle tree (l with l ^ 16, then ^ 8, ^ 4, ^ 2, ^ 1), so the sums
// are fixed-order and deterministic, and all eight lanes of a group hold the
// same bits.
//
// Test hook: with a.stall set, CTA 0 leaves out its arrival on the first
// step's barrier, so its wait runs out (about 2 s), the others' next wait
// too, and the host reads NBODY_ETIMEOUT.
#include <cooperative_groups.h>

#include "nbody_dev.cuh"

namespace cg = cooperative_groups;

namespace nb {

namespace {

constexpr int kMaxClusterCtas = 16;  // one CTA per SM (non-portable cluster size)
constexpr int kMaxWarps = 16;         // targets per CTA, one warp each (4 per SM sub-partition)
constexpr int kSmallMax = kMaxClusterCtas * kMaxWarps;

// Address of `p` (this CTA's shared memory) in the shared memory of CTA
// `rank` of the cluster.
__device__ __forceinline__ uint32_t rank_addr(const void *p, int rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(p)), "r"(rank));
  return out;
}

// One double into a cluster CTA's shared memory; its 8 bytes complete a
// transaction on that CTA's mbarrier `bar`.
__device__ __forceinline__ void st_async_f64(uint32_t addr, double v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(addr), "d"(v),
               "r"(bar)
               : "memory");
}

// Bounded wait for a phase of this CTA's mbarrier, acquiring at cluster
// scope what other CTAs stored into this CTA's shared memory.
__device__ __forceinline__ bool wait_cluster(uint64_t *bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitPolls; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

template <typename T>
__device__ __forceinline__ T *pick_ptr(int c, T *x, T *y, T *z) {
  return c == 0 ? x : (c == 1 ? y : z);
}

__global__ void __launch_bounds__(32 * kMaxWarps) smalln_kernel(const SmallArgs a) {
  __shared__ double4_32a pos[2][kSmallMax];  // (x, y, z, G m), a full copy per CTA
  __shared__ uint64_t bar[2];                // pos[i] is complete when bar[i]'s phase is
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = static_cast<int>(cluster.block_rank());
  const int csize = static_cast<int>(cluster.num_blocks());
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.N;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double4_32a q = make_double4_32a(a.x[j], a.y[j], a.z[j], a.G * a.m[j]);
    pos[0][j] = q;  // G m never changes: both buffers carry it from here on
    pos[1][j] = q;
  }
  const int p = rank + csize * warp;  // this warp's target (if < n)
  const bool own = p < n;
  const int c = lane >> 3;  // component of this lane in the update phase (3: padding)
  const bool upd = own && c < 3;
  double r = 0, v = 0, acc = 0;  // component c of this warp's target
  if (upd) {
    r = pick_ptr(c, a.x, a.y, a.z)[p];
    v = pick_ptr(c, a.vx, a.vy, a.vz)[p];
    acc = pick_ptr(c, a.ax, a.ay, a.az)[p];
  }
  // Only the CTAs that own a target (ranks below nact) take part in the
  // exchange.  This lane's slot of pos[0] / pos[1] and the mbarriers, in the
  // one or two of them (ranks lane % 8 and lane % 8 + 8) that it writes to.
  const int nact = min(csize, n);
  const int rk = lane & 7;
  const bool one = rk < nact, two = rk + 8 < nact;
  uint32_t pa0 = 0, pa1 = 0, pb0 = 0, pb1 = 0, ba0 = 0, ba1 = 0, bb0 = 0, bb1 = 0;
  if (upd && one) {
    const double *m0 = reinterpret_cast<const double *>(&pos[0][p]) + c;
    const double *m1 = reinterpret_cast<const double *>(&pos[1][p]) + c;
    pa0 = rank_addr(m0, rk);
    pa1 = rank_addr(m1, rk);
    ba0 = rank_addr(&bar[0], rk);
    ba1 = rank_addr(&bar[1], rk);
    if (two) {
      pb0 = rank_addr(m0, rk + 8);
      pb1 = rank_addr(m1, rk + 8);
      bb0 = rank_addr(&bar[0], rk + 8);
      bb1 = rank_addr(&bar[1], rk + 8);
    }
  }
  const uint32_t tx = 24u * static_cast<uint32_t>(n);  // bytes each active CTA receives per step
  const bool stall = a.stall != 0 && rank == 0;
  cluster.sync();
  // Warps without a target leave the step loop at once: no other warp waits
  // for them, so a waiting one could fall two phases behind and misread the
  // parity.  (Warp 0 of an active CTA owns a target, so its thread 0, which
  // announces the CTA's expected bytes, always takes part.)
  const int64_t n_steps = own ? a.n_steps : 0;
  int b = 0;
  for (int64_t step = 0; step < n_steps; ++step) {
    const int nb = 1 - b;
    if (threadIdx.x == 0 && !(stall && step == 0)) mbar_arrive_expect_tx(&bar[nb], tx);
    // Eq. 3 drift of component c; the group's 8 lanes store it into every
    // active CTA's copy, each store counted on the receiving CTA's mbarrier.
    if (upd) {
      r = drift(r, v, acc, a.dt, a.half_dt2);
      if (one) st_async_f64(nb ? pa1 : pa0, r, nb ? ba1 : ba0);
      if (two) st_async_f64(nb ? pb1 : pb0, r, nb ? bb1 : bb0);
    }
    // bar[nb] is used every other step: its phase parity is (step / 2) mod 2.
    const bool ok = __all_sync(0xffffffffu, wait_cluster(&bar[nb], static_cast<uint32_t>(step >> 1) & 1u));
    if (!ok) {
      if (lane == 0) atomicOr(a.flags, kFlagTimeout);
      break;
    }
    b = nb;
    // Eq. 1 at the new positions: lanes split the sources.
    double s0 = 0, s1 = 0, s2 = 0;
    const double4_32a me = pos[b][p];
    for (int j = lane; j < n; j += 32) {
      if (j == p) continue;
      interact_fp64<false>(pos[b][j], me.x, me.y, me.z, false, s0, s1, s2);
    }
    // Butterfly reduce-scatter over the lanes.  Level 16: lanes with bit 4
    // clear keep components (0, 1), the others (2, 3 = zero padding).
    const bool h = (lane & 16) != 0;
    const double k0 = h ? s2 : s0, k1 = h ? 0.0 : s1;
    const double g0 = h ? s0 : s2, g1 = h ? s1 : 0.0;
    const double t0 = k0 + __shfl_xor_sync(0xffffffffu, g0, 16);
    const double t1 = k1 + __shfl_xor_sync(0xffffffffu, g1, 16);
    // Level 8: bit 3 picks one of the two; the lane now holds component c.
    const bool g = (lane & 8) != 0;
    double s = (g ? t1 : t0) + __shfl_xor_sync(0xffffffffu, g ? t0 : t1, 8);
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (upd) {
      if (!isfinite(s) && (lane & 7) == 0) atomicOr(a.flags, kFlagNonFinite);
      v = kick(v, acc, s, a.half_dt);  // Eq. 4
      acc = s;
    }
  }
  if (upd && (lane & 7) == 0) {
    pick_ptr(c, a.x, a.y, a.z)[p] = r;
    pick_ptr(c, a.vx, a.vy, a.vz)[p] = v;
    pick_ptr(c, a.ax, a.ay, a.az)[p] = acc;
  }
  cluster.sync();  // no CTA leaves while others may still write into its shared memory
}

}  // namespace

int small_max_bodies() { return kSmallMax; }

cudaError_t small_prepare() {
  return cudaFuncSetAttribute(smalln_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

cudaError_t launch_small(const SmallArgs &a, cudaStream_t s) {
  const int ctas = a.N <= 32 ? 8 : kMaxClusterCtas;
  const int warps = a.N <= 64 ? 4 : (a.N + kMaxClusterCtas - 1) / kMaxClusterCtas;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(32 * warps);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, smalln_kernel, a);
}

}  // namespace nb
