// Device helpers shared by the force, energy and adjoint kernels:
// mbarrier + bulk-copy (TMA) PTX, bounded waits, the FP64 and mixed pair
// interactions of Eq. 1, and the Verlet kick (Eq. 4) and drift (Eq. 3).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "nbody_internal.h"

namespace nb {

// ---------------------------------------------------------------------------
// mbarrier and 1-D bulk copies global -> shared (cp.async.bulk, the TMA unit)
// ---------------------------------------------------------------------------

// Upper bound on mbarrier.try_wait polls before a wait is declared lost.
// Each poll of a phase that does not complete suspends the thread for the
// hardware's own limit (measured on GB300: ~1.9 us), so 2^20 polls are
// ~2 s, while a source tile lands in microseconds.  (An explicit timer or
// suspend-time hint in this loop cost the force kernels registers.)
constexpr uint32_t kWaitPolls = 1u << 20;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking: has the phase with the given parity completed?
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// One arrival (release semantics: this thread's earlier shared-memory
// writes are visible to a thread whose wait sees the phase complete).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Wait for the phase with the given parity to complete; false if the poll
// budget ran out (the caller records kFlagTimeout and winds down).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitPolls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned) from
// global memory into this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Programmatic dependent launch: let the next kernel in the stream start
// launching, and wait until the previous kernel has completed and its
// writes are visible (no-ops when the launch was not chained).
__device__ __forceinline__ void grid_dependency_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Mixed-path stage layout: pair blocks of two stage entries, 16 floats
//   [xh0 xh1 yh0 yh1 | zh0 zh1 mu0 mu1 | xl0 xl1 yl0 yl1 | zl0 zl1 0 0];
// float offset of field f of entry q is pair_off(q) + f.
enum PairField { kXh = 0, kYh = 2, kZh = 4, kMu = 6, kXl = 8, kYl = 10, kZl = 12 };
__device__ __forceinline__ size_t pair_off(int q) { return static_cast<size_t>(q >> 1) * 16 + (q & 1); }

// ---------------------------------------------------------------------------
// Reciprocal square-root seeds (MUFU) and their refinement
// ---------------------------------------------------------------------------

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ double rsqrt_approx(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}

// |d|^-3 = r2^{-3/2} to full FP64 accuracy from a seed y0 ~ r2^{-1/2} with
// relative error below 2^-19: with e = 1 - r2 y0^2,
//   r2^{-3/2} = y0^3 (1 - e)^{-3/2} = y0^3 (1 + 3e/2 + 15e^2/8 + O(e^3)),
// the binomial series truncated after e^2 (|e| < 2^-18, so the dropped
// 35/16 e^3 term is below 2^-52 relative).  6 FP64 operations.
__device__ __forceinline__ double inv_r3(double r2) {
  const double y0 = rsqrt_approx(r2);
  const double t = y0 * y0;
  const double e = fma(-r2, t, 1.0);
  const double y3 = t * y0;
  const double c = fma(e, 1.875, 1.5);
  return fma(y3 * e, c, y3);
}

// |d|^-1 = r2^{-1/2} = y0 (1 - e)^{-1/2} = y0 (1 + e/2 + 3e^2/8 + O(e^3)).
__device__ __forceinline__ double inv_r1(double r2) {
  const double y0 = rsqrt_approx(r2);
  const double e = fma(-r2, y0 * y0, 1.0);
  return fma(y0 * e, fma(e, 0.375, 0.5), y0);
}

// ---------------------------------------------------------------------------
// Pair interactions of Eq. 1: a_p += mu_j (r_j - r_p) |r_j - r_p|^-3,
// mu_j = G m_j.  MASK: the source may be the target itself (j == p); its
// difference is then exactly zero and r2 is replaced by 1 so the term is 0.
// ---------------------------------------------------------------------------

template <bool MASK>
__device__ __forceinline__ void interact_fp64(const double4_32a &j, double px, double py, double pz, bool self,
                                              double &ax, double &ay, double &az) {
  const double dx = j.x - px;
  const double dy = j.y - py;
  const double dz = j.z - pz;
  double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
  if (MASK) r2 = self ? 1.0 : r2;
  const double f = j.w * inv_r3(r2);
  ax = fma(f, dx, ax);
  ay = fma(f, dy, ay);
  az = fma(f, dz, az);
}

// Mixed: positions split as x = hi + lo (hi = fl32(x), lo = fl32(x - hi)).
// d = (hi_j - hi_p) + (lo_j - lo_p): the hi difference is exact whenever the
// two coordinates are within a factor 2 (Sterbenz), so close pairs keep the
// FP64 difference to about one FP32 ulp; far pairs lose nothing that FP32
// could have kept.  |d|^-3 from the MUFU rsqrt seed, products in FP32.
template <bool MASK>
__device__ __forceinline__ void interact_mixed(const float4 &hj, const float4 &lj, float hx, float hy, float hz,
                                               float lx, float ly, float lz, bool self, float &ax, float &ay,
                                               float &az) {
  const float dx = (hj.x - hx) + (lj.x - lx);
  const float dy = (hj.y - hy) + (lj.y - ly);
  const float dz = (hj.z - hz) + (lj.z - lz);
  float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  if (MASK) r2 = self ? 1.0f : r2;
  const float q = rsqrt_approx(r2);
  const float q2 = q * q;
  const float f = (hj.w * q) * q2;
  ax = fmaf(f, dx, ax);
  ay = fmaf(f, dy, ay);
  az = fmaf(f, dz, az);
}

// ---------------------------------------------------------------------------
// Bounding boxes for the mixed force kernel's far test
// ---------------------------------------------------------------------------

// Warp-wide minimum / maximum of a float through the integer reduction unit:
// ord() maps floats to unsigned integers in the same order.
__device__ __forceinline__ unsigned ord(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ float warp_min(float v) { return unord(__reduce_min_sync(0xffffffffu, ord(v))); }
__device__ __forceinline__ float warp_max(float v) { return unord(__reduce_max_sync(0xffffffffu, ord(v))); }

// Widened box of one warp's hi coordinates (mn, mx over its lanes) with lo
// parts up to (lx, ly, lz) per component: [mn - kappa l, mx + kappa l] per axis
// with l = |(lx, ly, lz)|, written by lane 0 to box[0..1].
__device__ __forceinline__ void warp_box(float mnx, float mny, float mnz, float mxx, float mxy, float mxz, float lx,
                                         float ly, float lz, float4 *box) {
  mnx = warp_min(mnx);
  mny = warp_min(mny);
  mnz = warp_min(mnz);
  mxx = warp_max(mxx);
  mxy = warp_max(mxy);
  mxz = warp_max(mxz);
  lx = warp_max(lx);
  ly = warp_max(ly);
  lz = warp_max(lz);
  const float w = kFarKappa * sqrtf(fmaf(lz, lz, fmaf(ly, ly, lx * lx)));
  if ((threadIdx.x & 31) == 0) {
    box[0] = make_float4(mnx - w, mny - w, mnz - w, 0.f);
    box[1] = make_float4(mxx + w, mxy + w, mxz + w, 0.f);
  }
}

// ---------------------------------------------------------------------------
// Velocity Verlet (Eqs. 3-4), one body, one component.  The fused step
// epilogue and the stand-alone pre-drift both call these, so a run split
// into several nbody_step calls is bitwise identical to one call.
// ---------------------------------------------------------------------------

// Eq. 4: v_{i+1} = v_i + dt/2 (a_i + a_{i+1})
__device__ __forceinline__ double kick(double v, double a_old, double a_new, double half_dt) {
  return fma(half_dt, a_old + a_new, v);
}

// Eq. 3: r_{i+1} = r_i + v_i dt + dt^2/2 a_i
__device__ __forceinline__ double drift(double r, double v, double a, double dt, double half_dt2) {
  return fma(half_dt2, a, fma(v, dt, r));
}

__device__ __forceinline__ float hi_part(double x) { return __double2float_rn(x); }
__device__ __forceinline__ float lo_part(double x, float hi) {
  return __double2float_rn(x - static_cast<double>(hi));
}

// Knuth's TwoSum: (hi, lo) += v with the rounding error of hi + v kept in lo.
// Used once per source tile, so long sums do not drop terms below half an
// ulp of a dominant term (a moon next to its planet among ~1e6 asteroids).
__device__ __forceinline__ void two_sum_acc(double &hi, double &lo, double v) {
  const double s = hi + v;
  const double bb = s - hi;
  lo += (hi - (s - bb)) + (v - bb);
  hi = s;
}

__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float v) {
  const float s = hi + v;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (v - bb);
  hi = s;
}

// ---------------------------------------------------------------------------
// Packed FP32 pairs (.f32x2, sm_100 and later): two floats in one 64-bit
// register pair.
// ---------------------------------------------------------------------------
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

__device__ __forceinline__ bool finite3(double a, double b, double c) {
  return isfinite(a) && isfinite(b) && isfinite(c);
}

}  // namespace nb
