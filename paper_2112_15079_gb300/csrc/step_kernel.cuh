// Fused Eq. 1 force + Eq. 4 kick + Eq. 3 drift, one launch per Verlet step.
//
// Work decomposition: a persistent grid (ctas_per_sm CTAs per SM) pulls
// Items from an atomic counter.  Items are sorted by cost (largest first),
// so the pull order is a longest-processing-time list schedule, which also
// balances uneven systems of a batched run.  An Item is a block of
// THREADS*IPT targets of one system against one chunk of that system's
// sources.  Targets live in registers (IPT per thread, strided by THREADS
// for coalesced access); sources stream through a kStages-deep shared-memory
// ring filled by 1-D bulk copies (cp.async.bulk, completion on mbarriers),
// issued by one thread, `tj` sources per stage.
//
// Split sources: when a target block has nsplit > 1 chunks, each chunk's CTA
// writes FP64 partial sums, then bumps the block's arrival counter; the CTA
// that arrives last sums the partials in slot order 0..nsplit-1 (fixed
// order, so results do not depend on scheduling) and runs the epilogue.
// Nothing ever spins on another CTA.
//
// Epilogue (kModeStep), per target p, FP64: Eq. 4 kick with the previous
// and the new acceleration, the caller's position array receives r_i, and
// the Eq. 3 drift r_{i+1} is staged for the next launch (ping-pong stages).
#pragma once

#include "nbody_dev.cuh"

namespace nb {

template <int PREC>
struct Prec;

template <>
struct Prec<0> {  // FP64
  static constexpr int kBytesPerSource = 32;  // double4_32a (x, y, z, mu)
};
template <>
struct Prec<1> {  // mixed
  static constexpr int kBytesPerSource = 32;  // float4 hi (x,y,z,mu) + float4 lo (x,y,z,0)
};

// Minimum resident CTAs per SM the register allocation must allow: the
// mixed kernel is latency-bound on the FP32 pipe and wants ~32 warps/SM
// (<= 64 registers); the FP64 kernel saturates GB300's narrow FP64 pipe
// with few warps, so it trades occupancy for registers.
template <int PREC, int THREADS, int IPT>
struct MinBlocks {  // mixed: 32 / 24 / 16 warps per SM for IPT 1 / 2 / 4 (64 / 85 / 128 registers)
  static constexpr int value = PREC == 1 ? ((IPT == 1 ? 1024 : IPT == 2 ? 768 : 512) / THREADS) : 1;
};

template <int PREC, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS, (MinBlocks<PREC, THREADS, IPT>::value)) step_kernel(const StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[kStages];
  __shared__ int s_item;
  __shared__ int s_flag;  // bit 0: abort (a wait ran out); bit 1: this CTA reduces the block

  const int tid = threadIdx.x;
  const int tj = a.tj;
  // Stage s holds tj sources: FP64 -> double4_32a[tj]; mixed -> float4 hi[tj], float4 lo[tj].
  auto stage_ptr = [&](int s) { return smem + static_cast<size_t>(s) * tj * Prec<PREC>::kBytesPerSource; };

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    mbar_init_fence();
    s_flag = 0;
  }
  __syncthreads();

  uint32_t phase = 0;  // bit s: parity of the next completion of stage s

  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.work_ctr, 1);
    __syncthreads();
    const int item_idx = s_item;
    if (item_idx >= a.n_items) break;
    const Item it = a.items[item_idx];

    // ---- targets into registers ---------------------------------------
    int pidx[IPT];
    bool valid[IPT];
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      const int p = it.i0 + tid + k * THREADS;
      valid[k] = p < it.i1;
      pidx[k] = valid[k] ? p : it.i1 - 1;  // duplicate a real target, result discarded
    }
    // FP64 path: (acc, cmp) is a hi/lo pair fed once per tile with the tile's
    // FP64 sub-sum through TwoSum.  Both paths leave the item's sums in acc.
    double accx[IPT], accy[IPT], accz[IPT], cmpx[IPT], cmpy[IPT], cmpz[IPT];
#pragma unroll
    for (int k = 0; k < IPT; ++k) accx[k] = accy[k] = accz[k] = cmpx[k] = cmpy[k] = cmpz[k] = 0.0;

    double px[IPT], py[IPT], pz[IPT];                               // FP64 path
    float hx[IPT], hy[IPT], hz[IPT], lx[IPT], ly[IPT], lz[IPT];     // mixed path
    // mixed path: per-target sums as unevaluated float pairs (hi + lo), fed
    // one FP32 sub-sum of kFoldEvery sources at a time through TwoSum and
    // converted to FP64 once per item, so the source loop issues no FP64
    // instruction (GB300 runs FP64 and f32<->f64 conversions at 1/64 rate).
    float shx[IPT], shy[IPT], shz[IPT], slx[IPT], sly[IPT], slz[IPT];
#pragma unroll
    for (int k = 0; k < IPT; ++k) shx[k] = shy[k] = shz[k] = slx[k] = sly[k] = slz[k] = 0.f;
    if (PREC == 0) {
      const double4_32a *cur = static_cast<const double4_32a *>(a.cur_a);
#pragma unroll
      for (int k = 0; k < IPT; ++k) {
        const double4_32a r = cur[pidx[k]];
        px[k] = r.x; py[k] = r.y; pz[k] = r.z;
      }
    } else {
      const float4 *hi = static_cast<const float4 *>(a.cur_a);
      const float4 *lo = static_cast<const float4 *>(a.cur_b);
#pragma unroll
      for (int k = 0; k < IPT; ++k) {
        const float4 h = hi[pidx[k]];
        const float4 l = lo[pidx[k]];
        hx[k] = h.x; hy[k] = h.y; hz[k] = h.z;
        lx[k] = l.x; ly[k] = l.y; lz[k] = l.z;
      }
    }

    // ---- source loop -----------------------------------------------------
    const int nsrc = it.j1 - it.j0;
    const int ntiles = (nsrc + tj - 1) / tj;
    auto issue = [&](int t) {  // tid 0 only
      const int s = t % kStages;
      const int j = it.j0 + t * tj;
      const int cnt = min(tj, it.j1 - j);
      unsigned char *dst = stage_ptr(s);
      if (PREC == 0) {
        mbar_arrive_expect_tx(&bar[s], static_cast<uint32_t>(cnt) * 32u);
        bulk_g2s(dst, static_cast<const double4_32a *>(a.cur_a) + j, static_cast<uint32_t>(cnt) * 32u, &bar[s]);
      } else {
        mbar_arrive_expect_tx(&bar[s], static_cast<uint32_t>(cnt) * 32u);
        bulk_g2s(dst, static_cast<const float4 *>(a.cur_a) + j, static_cast<uint32_t>(cnt) * 16u, &bar[s]);
        bulk_g2s(dst + static_cast<size_t>(tj) * 16, static_cast<const float4 *>(a.cur_b) + j,
                 static_cast<uint32_t>(cnt) * 16u, &bar[s]);
      }
    };
    if (tid == 0) {
      for (int t = 0; t < kStages && t < ntiles; ++t) issue(t);
    }

    bool aborted = false;
    for (int t = 0; t < ntiles; ++t) {
      const int s = t % kStages;
      if (!mbar_wait(&bar[s], (phase >> s) & 1u)) atomicOr(&s_flag, 1);
      phase ^= 1u << s;
      const int jt0 = it.j0 + t * tj;
      const int cnt = min(tj, it.j1 - jt0);
      const bool diag = jt0 < it.i1 && jt0 + cnt > it.i0;  // tile may contain a target itself

      if (PREC == 0) {
        const double4_32a *src = reinterpret_cast<const double4_32a *>(stage_ptr(s));
        double tx[IPT], ty[IPT], tz[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) tx[k] = ty[k] = tz[k] = 0.0;
        if (!diag) {
          int jj = 0;
          for (; jj + 4 <= cnt; jj += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const double4_32a sj = src[jj + u];
#pragma unroll
              for (int k = 0; k < IPT; ++k) interact_fp64<false>(sj, px[k], py[k], pz[k], false, tx[k], ty[k], tz[k]);
            }
          }
          for (; jj < cnt; ++jj) {
            const double4_32a sj = src[jj];
#pragma unroll
            for (int k = 0; k < IPT; ++k) interact_fp64<false>(sj, px[k], py[k], pz[k], false, tx[k], ty[k], tz[k]);
          }
        } else {
          for (int jj = 0; jj < cnt; ++jj) {
            const double4_32a sj = src[jj];
            const int jg = jt0 + jj;
#pragma unroll
            for (int k = 0; k < IPT; ++k)
              interact_fp64<true>(sj, px[k], py[k], pz[k], jg == pidx[k], tx[k], ty[k], tz[k]);
          }
        }
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
          two_sum_acc(accx[k], cmpx[k], tx[k]);
          two_sum_acc(accy[k], cmpy[k], ty[k]);
          two_sum_acc(accz[k], cmpz[k], tz[k]);
        }
      } else {
        const float4 *sh = reinterpret_cast<const float4 *>(stage_ptr(s));
        const float4 *sl = sh + tj;
        for (int base = 0; base < cnt; base += kFoldEvery) {
          const int lim = min(kFoldEvery, cnt - base);
          float fx[IPT], fy[IPT], fz[IPT];
#pragma unroll
          for (int k = 0; k < IPT; ++k) fx[k] = fy[k] = fz[k] = 0.f;
          if (!diag && lim == kFoldEvery) {
#pragma unroll 4
            for (int jj = 0; jj < kFoldEvery; ++jj) {
              const float4 hj = sh[base + jj];
              const float4 lj = sl[base + jj];
#pragma unroll
              for (int k = 0; k < IPT; ++k)
                interact_mixed<false>(hj, lj, hx[k], hy[k], hz[k], lx[k], ly[k], lz[k], false, fx[k], fy[k], fz[k]);
            }
          } else {
            for (int jj = 0; jj < lim; ++jj) {
              const float4 hj = sh[base + jj];
              const float4 lj = sl[base + jj];
              const int jg = jt0 + base + jj;
#pragma unroll
              for (int k = 0; k < IPT; ++k)
                interact_mixed<true>(hj, lj, hx[k], hy[k], hz[k], lx[k], ly[k], lz[k], jg == pidx[k], fx[k], fy[k],
                                     fz[k]);
            }
          }
#pragma unroll
          for (int k = 0; k < IPT; ++k) {  // fold the sub-sum into the two-float accumulator
            two_sum_acc(shx[k], slx[k], fx[k]);
            two_sum_acc(shy[k], sly[k], fy[k]);
            two_sum_acc(shz[k], slz[k], fz[k]);
          }
        }
      }

      __syncthreads();  // every thread is done with stage s
      if (s_flag & 1) {
        aborted = true;
        // Drain the copies this CTA may still have in flight (bounded): tile t
        // itself (its wait may be the one that ran out; parity before the flip)
        // and the tiles issued ahead of it.  Then leave.
        if (tid == 0) {
          mbar_wait(&bar[s], ((phase >> s) & 1u) ^ 1u);
          for (int u = t + 1; u < ntiles && u < t + kStages; ++u) {
            const int su = u % kStages;
            mbar_wait(&bar[su], (phase >> su) & 1u);
            phase ^= 1u << su;
          }
        }
        break;
      }
      if (tid == 0 && t + kStages < ntiles) issue(t + kStages);
    }
    if (aborted) {
      if (tid == 0) atomicOr(a.flags, kFlagTimeout);
      break;
    }

#pragma unroll
    for (int k = 0; k < IPT; ++k) {  // collapse the hi/lo pairs
      if (PREC == 0) {
        accx[k] += cmpx[k];
        accy[k] += cmpy[k];
        accz[k] += cmpz[k];
      } else {
        accx[k] = static_cast<double>(shx[k]) + static_cast<double>(slx[k]);
        accy[k] = static_cast<double>(shy[k]) + static_cast<double>(sly[k]);
        accz[k] = static_cast<double>(shz[k]) + static_cast<double>(slz[k]);
      }
    }

    // ---- split-source reduction ---------------------------------------
    // Partials: FP64 path -> 3 doubles per target and slot, summed by FP64
    // TwoSum; mixed path -> 3 float pairs (hi, lo) in the same 24 bytes,
    // summed by FP32 TwoSum (GB300's FP64 pipe is 64x narrower, and a few
    // last-arriving CTAs doing FP64 sums over many slots become the tail).
    if (it.nsplit > 1) {
      const size_t N = static_cast<size_t>(a.N);
      double *prow = a.partial + static_cast<size_t>(it.slot) * 3 * N;
#pragma unroll
      for (int k = 0; k < IPT; ++k) {
        if (!valid[k]) continue;
        if (PREC == 0) {
          __stcg(prow + pidx[k], accx[k]);
          __stcg(prow + N + pidx[k], accy[k]);
          __stcg(prow + 2 * N + pidx[k], accz[k]);
        } else {
          float2 *frow = reinterpret_cast<float2 *>(prow);
          __stcg(frow + pidx[k], make_float2(shx[k], slx[k]));
          __stcg(frow + N + pidx[k], make_float2(shy[k], sly[k]));
          __stcg(frow + 2 * N + pidx[k], make_float2(shz[k], slz[k]));
        }
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        const int old = atomicAdd(a.arrive + it.ib, 1);
        const bool last = old == it.nsplit - 1;
        if (last) {
          atomicExch(a.arrive + it.ib, 0);
          __threadfence();
          atomicOr(&s_flag, 2);
        }
      }
      __syncthreads();
      const bool last = (s_flag & 2) != 0;
      if (!last) continue;  // s_flag bit 1 is clear here; the next fetch re-syncs
#pragma unroll
      for (int k = 0; k < IPT; ++k) {
        if (PREC == 0) {
          double sx = 0.0, sy = 0.0, sz = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
          for (int c = 0; c < it.nsplit; ++c) {
            const double *row = a.partial + static_cast<size_t>(c) * 3 * N;
            two_sum_acc(sx, ex, __ldcg(row + pidx[k]));
            two_sum_acc(sy, ey, __ldcg(row + N + pidx[k]));
            two_sum_acc(sz, ez, __ldcg(row + 2 * N + pidx[k]));
          }
          accx[k] = sx + ex;
          accy[k] = sy + ey;
          accz[k] = sz + ez;
        } else {
          float sx = 0.f, sy = 0.f, sz = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;
          for (int c = 0; c < it.nsplit; ++c) {
            const float2 *row = reinterpret_cast<const float2 *>(a.partial + static_cast<size_t>(c) * 3 * N);
            const float2 vx = __ldcg(row + pidx[k]);
            const float2 vy = __ldcg(row + N + pidx[k]);
            const float2 vz = __ldcg(row + 2 * N + pidx[k]);
            two_sum_acc(sx, ex, vx.x);
            two_sum_acc(sy, ey, vy.x);
            two_sum_acc(sz, ez, vz.x);
            ex += vx.y;
            ey += vy.y;
            ez += vz.y;
          }
          accx[k] = static_cast<double>(sx) + static_cast<double>(ex);
          accy[k] = static_cast<double>(sy) + static_cast<double>(ey);
          accz[k] = static_cast<double>(sz) + static_cast<double>(ez);
        }
      }
      __syncthreads();
      if (tid == 0) s_flag &= ~2;
    }

    // ---- epilogue --------------------------------------------------------
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      if (!valid[k]) continue;
      const int p = pidx[k];
      const double anx = accx[k], any = accy[k], anz = accz[k];
      if (!finite3(anx, any, anz)) atomicOr(a.flags, kFlagNonFinite);
      if (a.mode == kModeStep) {
        const double vx = kick(a.vx[p], a.ax[p], anx, a.half_dt);
        const double vy = kick(a.vy[p], a.ay[p], any, a.half_dt);
        const double vz = kick(a.vz[p], a.az[p], anz, a.half_dt);
        double rx, ry, rz;
        if (PREC == 0) {
          const double4_32a r = static_cast<const double4_32a *>(a.cur_a)[p];
          rx = r.x; ry = r.y; rz = r.z;
          const double4_32a rn = make_double4_32a(drift(rx, vx, anx, a.dt, a.half_dt2), drift(ry, vy, any, a.dt, a.half_dt2),
                                          drift(rz, vz, anz, a.dt, a.half_dt2), r.w);
          static_cast<double4_32a *>(a.nxt_a)[p] = rn;
        } else {
          rx = a.Rx[p]; ry = a.Ry[p]; rz = a.Rz[p];
          const double nx = drift(rx, vx, anx, a.dt, a.half_dt2);
          const double ny = drift(ry, vy, any, a.dt, a.half_dt2);
          const double nz = drift(rz, vz, anz, a.dt, a.half_dt2);
          a.Rx[p] = nx; a.Ry[p] = ny; a.Rz[p] = nz;
          const float hxn = hi_part(nx), hyn = hi_part(ny), hzn = hi_part(nz);
          const float mu = static_cast<const float4 *>(a.cur_a)[p].w;
          static_cast<float4 *>(a.nxt_a)[p] = make_float4(hxn, hyn, hzn, mu);
          static_cast<float4 *>(a.nxt_b)[p] = make_float4(lo_part(nx, hxn), lo_part(ny, hyn), lo_part(nz, hzn), 0.f);
        }
        a.x[p] = rx; a.y[p] = ry; a.z[p] = rz;
        a.vx[p] = vx; a.vy[p] = vy; a.vz[p] = vz;
      }
      a.ax[p] = anx; a.ay[p] = any; a.az[p] = anz;
    }
    // The next iteration's fetch is preceded by __syncthreads() inside the
    // loop head, so s_item is not overwritten while still being read.
    __syncthreads();
  }

  // ---- persistent-grid bookkeeping: the last CTA out resets the counters --
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const int done = atomicAdd(a.exit_ctr, 1);
    if (done == static_cast<int>(gridDim.x) - 1) {
      atomicExch(a.work_ctr, 0);
      atomicExch(a.exit_ctr, 0);
    }
  }
}

}  // namespace nb
