// Single-launch paths for one FP64 system: every velocity-Verlet step of an
// nbody_step call inside ONE launch, of one thread-block cluster (small
// systems, smalln_kernel) or of a cooperative grid (mid-size systems,
// gridn_kernel, further below).  The host picks the cluster up to 96 bodies
// and the grid from 97 to 4,096, where each is the fastest path measured.
//
// The Sun-plus-30-bodies model has 930 interactions per step; as separate
// launches a step costs two kernel launches for microseconds of work.  Here
// the cluster's CTAs (8 for N <= 32, else 16; one per SM) own the targets,
// one warp per target (4 warps per CTA up to 64 bodies, then ceil(N / 16), at
// most kMaxWarps): the warp's 32 lanes split the sources and sum them in
// FP64 (up to kSmallMax = 256 bodies; beyond 96 the grid kernel is faster).
// Against the general two-kernel path, which spreads the pairs over every SM
// but pays two launches and the partial-row sums per step: 8.7x at 31
// bodies, 4.8x at 96.  Every CTA keeps all positions in its shared memory
// (ping-pong buffers pos[0], pos[1]).  Eq. 1 uses the same FP64 interaction
// as the general kernel (binomial-series refinement of the MUFU seed),
// Eqs. 3-4 the same kick/drift functions.
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
#include <algorithm>

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

// Eq. 1 for target p by one warp: the lanes split the sources (positions
// and G m in shared memory), then a butterfly reduce-scatter over the lanes
// leaves component lane / 8 of a_p in every lane of that group (lanes 24..31:
// a zero padding component).  Level 16: lanes with bit 4 clear keep
// components (0, 1), the others (2, 3); level 8: bit 3 picks one of the two;
// levels 4, 2, 1 finish the sum.  Fixed order, so deterministic.
__device__ __forceinline__ double warp_accel(const double4_32a *pos, int n, int p, int lane) {
  double s0 = 0, s1 = 0, s2 = 0;
  const double4_32a me = pos[p];
  for (int j = lane; j < n; j += 32) {
    if (j == p) continue;
    interact_fp64<false>(pos[j], me.x, me.y, me.z, false, s0, s1, s2);
  }
  const bool h = (lane & 16) != 0;
  const double k0 = h ? s2 : s0, k1 = h ? 0.0 : s1;
  const double g0 = h ? s0 : s2, g1 = h ? s1 : 0.0;
  const double t0 = k0 + __shfl_xor_sync(0xffffffffu, g0, 16);
  const double t1 = k1 + __shfl_xor_sync(0xffffffffu, g1, 16);
  const bool g = (lane & 8) != 0;
  double s = (g ? t1 : t0) + __shfl_xor_sync(0xffffffffu, g ? t0 : t1, 8);
#pragma unroll
  for (int off = 4; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  return s;
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
    // Eq. 1 at the new positions.
    const double s = warp_accel(pos[b], n, p, lane);
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

// ---------------------------------------------------------------------------
// Mid-size systems: the same per-warp step over a cooperative grid.
//
// The cluster kernel above uses 16 SMs; from about a hundred bodies the FP64
// chain of its warps (one target each, ceil(N/32) sources per lane) grows
// long, while the general path pays two launches and the partial-row sums
// per step.  This kernel keeps one warp per target but spreads the targets
// over as many CTAs as the GPU holds at once (a cooperative launch, so all
// are resident): each step the owners store their drifted coordinates into
// a global exchange buffer (double-buffered by step parity), one grid-wide
// barrier publishes them, and every CTA loads all positions from L2 into
// shared memory.  The barrier is a counter of arrivals: arrival k + 1 of
// every CTA means all step-k stores are visible (fence before the arrival,
// acquire load of the counter after).  Buffer reuse needs no second
// barrier: a CTA stores into buffer b at step k + 2 only after barrier
// k + 1, which every CTA reaches only after loading buffer b at step k.
// Waits are bounded (kGridPolls); a wait that runs out sets kFlagTimeout and
// the CTA leaves, so the others' waits run out too.
// ---------------------------------------------------------------------------
constexpr int kGridMax = 4096;                // bodies (a full copy of the positions per CTA)
constexpr uint32_t kGridPolls = 1u << 21;  // an L2 round trip plus a 64 ns back-off each: about a second

__device__ __forceinline__ uint32_t ld_acquire_gpu(const unsigned *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded barrier of the whole cooperative grid; false if it ran out.
__device__ __forceinline__ bool grid_barrier(unsigned *ctr, uint32_t target, bool arrive, int *s_abort) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (arrive) atomicAdd(ctr, 1u);
    for (uint32_t i = 0; ld_acquire_gpu(ctr) < target; ++i) {
      if (i == kGridPolls) {
        *s_abort = 1;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
  return *s_abort == 0;
}

__global__ void __launch_bounds__(1024) gridn_kernel(const SmallArgs a) {
  extern __shared__ __align__(32) unsigned char gsm[];
  double4_32a *pos = reinterpret_cast<double4_32a *>(gsm);  // [N]: (x, y, z, G m)
  __shared__ int s_abort;
  const int warps = static_cast<int>(blockDim.x >> 5);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.N;
  const size_t N = static_cast<size_t>(n);
  const int p = static_cast<int>(blockIdx.x) * warps + warp;  // this warp's target (if < n)
  const bool own = p < n;
  const int c = lane >> 3;
  const bool upd = own && c < 3;
  for (int j = threadIdx.x; j < n; j += blockDim.x) pos[j].w = a.G * a.m[j];
  double r = 0, v = 0, acc = 0;
  if (upd) {
    r = pick_ptr(c, a.x, a.y, a.z)[p];
    v = pick_ptr(c, a.vx, a.vy, a.vz)[p];
    acc = pick_ptr(c, a.ax, a.ay, a.az)[p];
  }
  if (threadIdx.x == 0) s_abort = 0;
  const bool stall = a.stall != 0 && blockIdx.x == 0;
  for (int64_t step = 0; step < a.n_steps; ++step) {  // every thread of every CTA runs every step
    double *xb = a.xg + static_cast<size_t>(step & 1) * 3 * N;
    if (upd) {
      r = drift(r, v, acc, a.dt, a.half_dt2);  // Eq. 3
      if ((lane & 7) == 0) xb[c * N + p] = r;
    }
    const uint32_t target = static_cast<uint32_t>(step + 1) * gridDim.x;
    if (!grid_barrier(a.gbar, target, !(stall && step == 0), &s_abort)) {
      if (threadIdx.x == 0) atomicOr(a.flags, kFlagTimeout);
      break;
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {  // other CTAs' stores: read through L2
      pos[j].x = __ldcg(xb + j);
      pos[j].y = __ldcg(xb + N + j);
      pos[j].z = __ldcg(xb + 2 * N + j);
    }
    __syncthreads();
    if (own) {  // warp-uniform
      const double s = warp_accel(pos, n, p, lane);  // Eq. 1
      if (upd) {
        if (!isfinite(s) && (lane & 7) == 0) atomicOr(a.flags, kFlagNonFinite);
        v = kick(v, acc, s, a.half_dt);  // Eq. 4
        acc = s;
      }
    }
  }
  if (upd && (lane & 7) == 0) {
    pick_ptr(c, a.x, a.y, a.z)[p] = r;
    pick_ptr(c, a.vx, a.vy, a.vz)[p] = v;
    pick_ptr(c, a.ax, a.ay, a.az)[p] = acc;
  }
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


int grid_max_bodies() { return kGridMax; }

cudaError_t grid_shape(int N, int nsm, int *warps, int *ctas) {
  if (N < 1 || N > kGridMax) return cudaErrorInvalidValue;
  const size_t smem = 32 * static_cast<size_t>(N);
  cudaError_t e = cudaFuncSetAttribute(gridn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(32 * static_cast<size_t>(kGridMax)));
  if (e != cudaSuccess) return e;
  // One CTA per SM: ceil(N / SMs) targets per CTA, rounded up to a multiple
  // of 4 warps so the SM's four sub-partitions (each with its own share of
  // the FP64 pipe) carry equal loads.
  const int w = std::max(4, (((N + nsm - 1) / nsm) + 3) / 4 * 4);
  if (w > 32) return cudaErrorCooperativeLaunchTooLarge;
  int occ = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gridn_kernel, 32 * w, smem)) != cudaSuccess) return e;
  const int g = (N + w - 1) / w;
  if (occ >= 1 && g <= occ * nsm) {
    *warps = w;
    *ctas = g;
    return cudaSuccess;
  }
  return cudaErrorCooperativeLaunchTooLarge;
}

cudaError_t launch_grid(const SmallArgs &a, int warps, int ctas, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(32 * warps);
  cfg.dynamicSmemBytes = 32 * static_cast<size_t>(a.N);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, gridn_kernel, a);
}

}  // namespace nb
