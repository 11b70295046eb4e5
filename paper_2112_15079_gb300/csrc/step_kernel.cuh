// Eq. 1 force kernel (one launch per Verlet step, followed by the per-body
// Verlet kernel in kernels_misc.cu that sums its partials and applies
// Eqs. 4 and 3).
//
// Work decomposition (hybrid stream-K): the force work of a step is the list
// of target blocks (at most THREADS*IPT consecutive bodies of one system,
// sizes balanced within a system) times the sources of their system, laid
// end to end and weighted by the warps a block keeps busy.  The host cuts
// most of that line into gridDim.x equal static shares (CTA c takes share
// c) and the rest into small chunks that free CTAs pull from a counter.
// Every segment writes one partial sum per target: FP64 for the FP64 path,
// a float pair (hi, lo) for the mixed path, in its fixed row `slot` of the
// partial array.  The Verlet kernel adds a body's rows in slot order (fixed
// order, so results do not depend on scheduling).  No CTA ever waits for
// another.
//
// Sources stream through a ring of 2-4 shared-memory stages (as deep as the
// CTAs per SM allow) filled by 1-D bulk copies (cp.async.bulk) that thread
// 0 issues, `tj` sources per stage.  Each stage has two mbarriers: `full`
// completes when its tile has landed, `empty` when every warp has released
// it.  The tiles of all the CTA's segments and pieces form one sequence, each
// stage carrying a small header (segment, source range), so the next
// segment's tiles load while the current one finishes and the warps never
// meet at a CTA-wide barrier inside the loop.  Targets live in registers,
// IPT per thread: warp w holds the block's 32 IPT consecutive entries from
// 32 IPT w, lane l entry 32 (IPT w + k) + l for k < IPT, so the loads
// coalesce and a warp's targets sit together in the stage (on the mixed
// path, near each other in space); warps without a valid target skip the
// arithmetic.
//
// FP64 path: sources as double4 (x, y, z, G m), one per body.
// Mixed path: sources as pair blocks of 64 bytes holding two consecutive
// stage entries field by field,
//     [xh0 xh1 yh0 yh1 | zh0 zh1 mu0 mu1 | xl0 xl1 yl0 yl1 | zl0 zl1 0 0],
// so one 16-byte shared load yields two packed f32x2 operands; the pair
// arithmetic then runs two sources per packed instruction (add/mul/fma
// .f32x2), halving the issued FP32 instructions.  Systems are padded to an
// even length with inert sources (far away, massless: their term is 0).
//
// Mixed path, far source groups: the stage of each system is in a spatial
// (Morton) order fixed by the host, and a warp's targets are consecutive
// stage entries, so they sit close together.  The stage is cut into groups
// of kBoxPairs pairs (64 sources); before each force launch box_kernel
// computes each group's bounding box of the hi parts, widened on every side
// by kFarKappa times the largest lo part of the group (as a vector), and
// every warp keeps the same box for its targets.  Where the two widened boxes are
// disjoint along some axis, every pair between them is at least kFarKappa
// (lo_j + lo_p) apart, and the difference of the hi parts alone,
// d' = hi_j - hi_p, moves the term mu_j d / |d|^3 by at most
// 2 |lo_j - lo_p| / |d| <= kFarEps relative (the derivative of d / |d|^3 has
// norm 2 / |d|^3): such a group takes the hi-only path, 12 FP32 lane
// operations per interaction instead of 18.  A target's own source is never
// in a far group (its box contains the target), so that path needs no self
// test.
//
// Launch chaining: griddepcontrol.wait before the first read of data the
// previous kernels wrote (staged sources), then griddepcontrol.
// launch_dependents, so the Verlet kernel's launch overlaps our work; it
// prefetches what this kernel does not write.
#pragma once

#include "nbody_dev.cuh"

namespace nb {

// Eq. 1 for one target (negated hi/lo coordinates duplicated in both halves)
// against a pair of sources, accumulating both terms into one packed pair.
// d = (hi_j - hi_p) + (lo_j - lo_p) per component: the hi difference is exact
// for close pairs (Sterbenz), so close pairs keep the FP64 difference to
// about one FP32 ulp.  MASK: replace r2 by 1 where the source is the target.
template <bool MASK>
__device__ __forceinline__ void interact_pair(const ulonglong2 &v0, const ulonglong2 &v1, const ulonglong2 &v2,
                                              const ulonglong2 &v3, f2 nxh, f2 nyh, f2 nzh, f2 nxl, f2 nyl,
                                              f2 nzl, bool self_a, bool self_b, f2 &ax, f2 &ay, f2 &az) {
  // v0 = (xh, yh), v1 = (zh, mu), v2 = (xl, yl), v3 = (zl, -)
  const f2 dx = add2(add2(v0.x, nxh), add2(v2.x, nxl));
  const f2 dy = add2(add2(v0.y, nyh), add2(v2.y, nyl));
  const f2 dz = add2(add2(v1.x, nzh), add2(v3.x, nzl));
  f2 r2 = mul2(dx, dx);
  r2 = fma2(dy, dy, r2);
  r2 = fma2(dz, dz, r2);
  float ra, rb;
  upk(r2, ra, rb);
  if (MASK) {
    ra = self_a ? 1.0f : ra;
    rb = self_b ? 1.0f : rb;
  }
  const f2 q = pk(rsqrt_approx(ra), rsqrt_approx(rb));
  const f2 f = mul2(mul2(v1.y, q), mul2(q, q));
  ax = fma2(f, dx, ax);
  ay = fma2(f, dy, ay);
  az = fma2(f, dz, az);
}

// The far-group form of interact_pair: d = hi_j - hi_p only (the lo parts
// are dropped; the caller has checked that this moves each term by at most
// kFarEps relative), no self test.  v0 = (xh, yh), v1 = (zh, mu).
__device__ __forceinline__ void interact_pair_hi(const ulonglong2 &v0, const ulonglong2 &v1, f2 nxh, f2 nyh, f2 nzh,
                                                 f2 &ax, f2 &ay, f2 &az) {
  const f2 dx = add2(v0.x, nxh);
  const f2 dy = add2(v0.y, nyh);
  const f2 dz = add2(v1.x, nzh);
  f2 r2 = mul2(dx, dx);
  r2 = fma2(dy, dy, r2);
  r2 = fma2(dz, dz, r2);
  float ra, rb;
  upk(r2, ra, rb);
  const f2 q = pk(rsqrt_approx(ra), rsqrt_approx(rb));
  const f2 f = mul2(mul2(v1.y, q), mul2(q, q));
  ax = fma2(f, dx, ax);
  ay = fma2(f, dy, ay);
  az = fma2(f, dz, az);
}

// Register budget: the mixed kernel wants many warps per SM (64 registers
// at 1024 threads per SM for IPT 1, 85 for IPT 2 at 768, up to 255 for
// IPT 4 at 256); the FP64 kernel
// saturates GB300's narrow FP64 pipe with few warps and takes what it needs.
template <int PREC, int THREADS, int IPT>
struct MinBlocks {
  static constexpr int raw = PREC == 1 ? ((IPT == 1 ? 1024 : IPT == 2 ? 768 : 256) / THREADS) : 1;
  static constexpr int value = raw < 1 ? 1 : raw;
};

template <int PREC, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS, (MinBlocks<PREC, THREADS, IPT>::value)) force_kernel(const ForceArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  // Ring of a.stages stages: full[s] completes when tile data (or the end
  // marker) is in stage s, empty[s] when every warp has released it.
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
  // Tile in stage s: (segment, first source, sources); segment -1 = no more work.
  __shared__ int4 s_hdr[kMaxStages];
  __shared__ int s_flag;              // bit 0: abort (a wait ran out)
  // The producer's cursor (thread 0 only): the next tile to issue.
  __shared__ struct {
    int piece, si, se, t, nt, s0, s1, issued, state;  // state: 0 issuing, 1 end marker out, 2 stopped
  } s_pc;
  // Mixed: the widened box of each warp's targets (low corner, high corner);
  // per target, its negated lo parts (read by the near path only) and its
  // running sums as float pairs (touched once per kFoldPairs pairs) -- kept
  // in shared memory so the source loop has the registers for more pairs in
  // flight.  Index [field][k * THREADS + tid].  All of it belongs to one
  // warp (or thread), so no CTA-wide barrier guards it.
  __shared__ __align__(16) float4 s_wbox[PREC == 1 ? 2 * (THREADS / 32) : 1];
  constexpr int kT = PREC == 1 ? THREADS * IPT : 1;
  __shared__ float s_tlo[3][kT];
  __shared__ float s_sum[6][kT];  // x hi, x lo, y hi, y lo, z hi, z lo

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tj = a.tj;  // sources per stage; both layouts take 32 bytes per source
  const int K = a.stages;
  // Stage s: tj sources (32 bytes each), then (mixed) the boxes of the
  // source groups the tile touches (at most tj / 64 + 2 groups, 32 bytes each).
  const size_t stage_bytes = static_cast<size_t>(tj) * 32 + (PREC == 1 ? (tj / 64 + 2) * 32 : 0);
  auto stage_ptr = [&](int s) { return smem + static_cast<size_t>(s) * stage_bytes; };
  auto box_ptr = [&](int s) { return reinterpret_cast<const float4 *>(stage_ptr(s) + static_cast<size_t>(tj) * 32); };
  const size_t N = static_cast<size_t>(a.N);
  const int n_static = static_cast<int>(gridDim.x);

  // ---- producer (thread 0) ---------------------------------------------
  // The work of this CTA is its static piece (blockIdx.x), then dynamic
  // pieces pulled from the counter while any is left; each piece is a run
  // of segments, each segment a run of tiles.  seek() moves the cursor to
  // the first tile of segment si or, past the piece's end, of the next
  // piece that has a segment (piece -1: none left).
  auto seek = [&]() {
    while (s_pc.si >= s_pc.se) {
      const int next = n_static + atomicAdd(a.dyn_ctr, 1);
      if (next >= n_static + a.n_dyn) {
        s_pc.piece = -1;
        return;
      }
      s_pc.piece = next;
      s_pc.si = a.seg_off[next];
      s_pc.se = a.seg_off[next + 1];
    }
    const Seg sg = a.segs[s_pc.si];
    s_pc.s0 = sg.s0;
    s_pc.s1 = sg.s1;
    s_pc.t = 0;
    s_pc.nt = (sg.s1 - sg.s0 + tj - 1) / tj;
  };
  // Issue tiles while the ring has room: at most K tiles ahead of tile c
  // (the next one warp 0 consumes), each into a stage every warp has
  // released.  A stage still held is left for a later call, except for
  // tile c itself, which must be out before anyone waits for it: for that
  // one the wait is (bounded) blocking.  Other warps never wait for warp 0
  // beyond that: the tiles before c were issued when warp 0 reached them.
  auto pump = [&](int c) {
    while (s_pc.state == 0 && s_pc.issued < c + K) {
      const int u = s_pc.issued, s = u % K, n = u / K;
      if (n > 0) {  // stage s last held tile u - K: released by every warp?
        const uint32_t par = static_cast<uint32_t>(n - 1) & 1u;
        if (u == c) {
          if (!mbar_wait(&empty[s], par)) {
            s_pc.state = 2;
            atomicOr(&s_flag, 1);
            return;
          }
        } else if (!mbar_test_wait(&empty[s], par)) {
          return;
        }
      }
      if (s_pc.piece < 0) {  // no more work: the end marker
        s_hdr[s] = make_int4(-1, 0, 0, 0);
        mbar_arrive(&full[s]);
        s_pc.state = 1;
        s_pc.issued = u + 1;
        return;
      }
      const int j = s_pc.s0 + s_pc.t * tj;
      const int nb = min(tj, s_pc.s1 - j);
      s_hdr[s] = make_int4(s_pc.si, j, nb, 0);
      const uint32_t bytes = static_cast<uint32_t>(nb) * 32u;
      // mixed: the boxes of groups (j / 2) / 32 .. ((j + nb) / 2 - 1) / 32, 32 bytes each
      const int g0 = (j >> 1) / kBoxPairs, g1 = (((j + nb) >> 1) - 1) / kBoxPairs;
      const uint32_t bbytes = PREC == 1 ? static_cast<uint32_t>(g1 - g0 + 1) * 32u : 0u;
      mbar_arrive_expect_tx(&full[s], bytes + bbytes);
      bulk_g2s(stage_ptr(s), static_cast<const unsigned char *>(a.cur) + static_cast<size_t>(j) * 32, bytes,
               &full[s]);
      if (PREC == 1)
        bulk_g2s(stage_ptr(s) + static_cast<size_t>(tj) * 32, a.boxes + 2 * static_cast<size_t>(g0), bbytes,
                 &full[s]);
      s_pc.issued = u + 1;
      if (++s_pc.t == s_pc.nt) {
        ++s_pc.si;
        seek();
      }
    }
  };

  if (tid == 0) {
    for (int s = 0; s < K; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], THREADS / 32);
      s_hdr[s] = make_int4(-1, 0, 0, 0);
    }
    mbar_init_fence();
    s_flag = 0;
  }
  grid_dependency_wait();    // staged sources of this step are complete (and the
                             // previous Verlet kernel has finished)
  grid_dependency_launch();  // so the Verlet kernel may start launching
  if (tid == 0) {
    s_pc.piece = blockIdx.x;
    s_pc.si = a.seg_off[blockIdx.x];
    s_pc.se = a.seg_off[blockIdx.x + 1];
    s_pc.issued = 0;
    s_pc.state = 0;
    seek();
    pump(0);  // the first tiles go out before the targets are loaded
  }
  __syncthreads();

  // ---- consumers (every warp): tiles in issue order ---------------------
  // A warp sets up a segment's targets when its first tile arrives and
  // writes their partial sums when the next segment's first tile (or the
  // end marker) arrives; between tiles it only releases the stage, so warps
  // drift apart by up to K tiles instead of meeting at a barrier per tile.
  bool aborted = false;
  int cur = -1;  // segment in progress
  int q0 = 0, q_end = 0;  // stage indices of its block's targets: [q0, q_end)
  int pidx[IPT], tq[IPT];
  bool valid[IPT];
  bool warp_busy = false;
  // FP64 path: (acc, cmp) is a hi/lo pair fed once per tile with the tile's
  // FP64 sub-sum through TwoSum.
  double accx[IPT], accy[IPT], accz[IPT], cmpx[IPT], cmpy[IPT], cmpz[IPT];
  double px[IPT], py[IPT], pz[IPT];
  // Mixed path: packed partial sums (even / odd sources) and the running
  // sums as unevaluated float pairs (hi + lo), fed one packed sub-sum of
  // kFoldPairs source pairs at a time through TwoSum, so the source loop
  // issues no FP64 instruction (GB300 runs FP64 and f32<->f64 conversions
  // at 1/64 of the FP32 rate).
  f2 nxh[IPT], nyh[IPT], nzh[IPT], pax[IPT], pay[IPT], paz[IPT];
  int mlo[IPT], mhi[IPT];

  // The partial sums of segment `cur`, row `slot`.
  auto flush = [&]() {
    double *prow = a.partial + static_cast<size_t>(a.segs[cur].slot) * 3 * N;
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      if (!valid[k]) continue;
      if (PREC == 0) {
        prow[pidx[k]] = accx[k] + cmpx[k];
        prow[N + pidx[k]] = accy[k] + cmpy[k];
        prow[2 * N + pidx[k]] = accz[k] + cmpz[k];
      } else {
        float2 *frow = reinterpret_cast<float2 *>(prow);
        const int i = k * THREADS + tid;
        frow[pidx[k]] = make_float2(s_sum[0][i], s_sum[1][i]);
        frow[N + pidx[k]] = make_float2(s_sum[2][i], s_sum[3][i]);
        frow[2 * N + pidx[k]] = make_float2(s_sum[4][i], s_sum[5][i]);
      }
    }
  };

  // The targets of segment `cur` (this warp's share of its block): target k
  // of this thread is stage entry tq (the block's entries are consecutive),
  // body pidx (the same index, or perm[tq] in a spatially ordered stage).
  auto setup = [&]() {
    const Blk bk = a.blks[a.segs[cur].blk];
    q0 = bk.q0;
    q_end = bk.q0 + (bk.i1 - bk.i0);
    bool any_valid = false;
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      const int r = (warp * IPT + k) * 32 + lane, cnt_b = bk.i1 - bk.i0;
      valid[k] = r < cnt_b;
      any_valid |= valid[k];
      const int rr = valid[k] ? r : cnt_b - 1;  // duplicate a real target, result discarded
      tq[k] = bk.q0 + rr;
      pidx[k] = a.perm ? a.perm[tq[k]] : bk.i0 + rr;
    }
    warp_busy = __any_sync(0xffffffffu, any_valid);  // warp-uniform
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      accx[k] = accy[k] = accz[k] = cmpx[k] = cmpy[k] = cmpz[k] = 0.0;
      pax[k] = pay[k] = paz[k] = 0ull;
      if (PREC == 0) {
        const double4_32a r = static_cast<const double4_32a *>(a.cur)[tq[k]];
        px[k] = r.x;
        py[k] = r.y;
        pz[k] = r.z;
      } else {
        const float *e = static_cast<const float *>(a.cur) + pair_off(tq[k]);
        nxh[k] = pk(-e[kXh], -e[kXh]);
        nyh[k] = pk(-e[kYh], -e[kYh]);
        nzh[k] = pk(-e[kZh], -e[kZh]);
        const int i = k * THREADS + tid;
        s_tlo[0][i] = -e[kXl];
        s_tlo[1][i] = -e[kYl];
        s_tlo[2][i] = -e[kZl];
#pragma unroll
        for (int f = 0; f < 6; ++f) s_sum[f][i] = 0.f;
      }
    }
    if constexpr (PREC == 1) {  // the widened box of this warp's targets
      float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, lo[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < IPT; ++k) {
        const float *e = static_cast<const float *>(a.cur) + pair_off(tq[k]);
        const float h[3] = {e[kXh], e[kYh], e[kZh]}, l[3] = {e[kXl], e[kYl], e[kZl]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          mn[d] = fminf(mn[d], h[d]);
          mx[d] = fmaxf(mx[d], h[d]);
          lo[d] = fmaxf(lo[d], fabsf(l[d]));
        }
      }
      warp_box(mn[0], mn[1], mn[2], mx[0], mx[1], mx[2], lo[0], lo[1], lo[2], &s_wbox[2 * warp]);
      __syncwarp();  // lane 0 wrote the box the whole warp reads
    }
    // Mixed path: the source pairs that may hold one of this warp's own
    // targets (for each k, the warp's 32 consecutive targets span <= 17
    // pairs).  Only those pairs take the masked path.
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      mlo[k] = static_cast<int>(__reduce_min_sync(0xffffffffu, static_cast<unsigned>(tq[k]))) >> 1;
      mhi[k] = static_cast<int>(__reduce_max_sync(0xffffffffu, static_cast<unsigned>(tq[k]))) >> 1;
    }
  };

  int ct = 0;               // tiles this warp has consumed
  int s = 0;                // their stage: ct mod K
  uint32_t par = 0;         // and the parity of that stage's next phase: (ct / K) mod 2
  for (;; ++ct) {
    if (tid == 0) pump(ct);
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&full[s], par));
    if (!ok) {  // a wait ran out: this warp winds down (the others run out on theirs)
      if (lane == 0) atomicOr(&s_flag, 1);
      aborted = true;
      break;
    }
    const int4 h = s_hdr[s];
    if (h.x < 0) break;  // no more work
    if (h.x != cur) {
      if (cur >= 0) flush();
      cur = h.x;
      setup();
    }
    {
      const int jt0 = h.y, cnt = h.z;  // the tile's sources [jt0, jt0 + cnt)

      if (warp_busy && PREC == 0) {
        const bool diag = jt0 < q_end && jt0 + cnt > q0;  // tile may contain a target itself
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
              interact_fp64<true>(sj, px[k], py[k], pz[k], jg == tq[k], tx[k], ty[k], tz[k]);
          }
        }
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
          two_sum_acc(accx[k], cmpx[k], tx[k]);
          two_sum_acc(accy[k], cmpy[k], ty[k]);
          two_sum_acc(accz[k], cmpz[k], tz[k]);
        }
      } else if (warp_busy) {
        const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(stage_ptr(s));  // 4 per pair block
        const float4 *gbox = box_ptr(s);  // the boxes of groups Pt / kBoxPairs ..
        const int Pt = jt0 >> 1, Pe = (jt0 + cnt) >> 1;  // the tile's stage pairs [Pt, Pe)
        const int gt = Pt / kBoxPairs;
        auto fold = [&]() {  // the packed sub-sums into the float pairs
#pragma unroll
          for (int k = 0; k < IPT; ++k) {
            const int i = k * THREADS + tid;
            const f2 p3[3] = {pax[k], pay[k], paz[k]};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              float e, o, h = s_sum[2 * c][i], l = s_sum[2 * c + 1][i];
              upk(p3[c], e, o);
              two_sum_acc(h, l, e + o);
              s_sum[2 * c][i] = h;
              s_sum[2 * c + 1][i] = l;
            }
            pax[k] = pay[k] = paz[k] = 0ull;
          }
        };
        // Near groups read the targets' lo parts from shared memory.
        f2 nxl[IPT], nyl[IPT], nzl[IPT];
        auto load_lo = [&]() {
#pragma unroll
          for (int k = 0; k < IPT; ++k) {
            const int i = k * THREADS + tid;
            nxl[k] = pk(s_tlo[0][i], s_tlo[0][i]);
            nyl[k] = pk(s_tlo[1][i], s_tlo[1][i]);
            nzl[k] = pk(s_tlo[2][i], s_tlo[2][i]);
          }
        };
        // Pairs [b0, b1) (stage pair indices): unmasked, with the self test,
        // or hi-only (far groups).  All visit the pairs in ascending order.
        auto unmasked = [&](int b0, int b1) {
          // (IPT 1 is capped at 64 registers: unrolling this rarer path
          // would spill.)
#pragma unroll(IPT == 1 ? 1 : 4)
          for (int b = b0; b < b1; ++b) {
            const ulonglong2 *pb = src + 4 * (b - Pt);
            const ulonglong2 v0 = pb[0], v1 = pb[1], v2 = pb[2], v3 = pb[3];
#pragma unroll
            for (int k = 0; k < IPT; ++k)
              interact_pair<false>(v0, v1, v2, v3, nxh[k], nyh[k], nzh[k], nxl[k], nyl[k], nzl[k], false, false,
                                   pax[k], pay[k], paz[k]);
          }
        };
        auto masked = [&](int b0, int b1) {
          for (int b = b0; b < b1; ++b) {
            const ulonglong2 *pb = src + 4 * (b - Pt);
            const ulonglong2 v0 = pb[0], v1 = pb[1], v2 = pb[2], v3 = pb[3];
#pragma unroll
            for (int k = 0; k < IPT; ++k)
              interact_pair<true>(v0, v1, v2, v3, nxh[k], nyh[k], nzh[k], nxl[k], nyl[k], nzl[k], 2 * b == tq[k],
                                  2 * b + 1 == tq[k], pax[k], pay[k], paz[k]);
          }
        };
        int since_fold = 0;  // pairs in the packed sub-sums
        // The tile in box groups (stage pairs [32 g, 32 g + 32), cut at the
        // tile's ends): far groups take the hi-only path.
        for (int P = Pt; P < Pe;) {
          const int g = P / kBoxPairs;
          const int P1 = min((g + 1) * kBoxPairs, Pe);
          const float4 glo = gbox[2 * (g - gt)], ghi = gbox[2 * (g - gt) + 1];
          const float4 wlo = s_wbox[2 * warp], whi = s_wbox[2 * warp + 1];
          const bool far = glo.x > whi.x || glo.y > whi.y || glo.z > whi.z || wlo.x > ghi.x || wlo.y > ghi.y ||
                           wlo.z > ghi.z;
          if (far) {
            if (P1 - P == kBoxPairs) {
#pragma unroll 4
              for (int b = P; b < P + kBoxPairs; ++b) {
                const ulonglong2 *pb = src + 4 * (b - Pt);
                const ulonglong2 v0 = pb[0], v1 = pb[1];
#pragma unroll
                for (int k = 0; k < IPT; ++k) interact_pair_hi(v0, v1, nxh[k], nyh[k], nzh[k], pax[k], pay[k], paz[k]);
              }
            } else {
              for (int b = P; b < P1; ++b) {
                const ulonglong2 *pb = src + 4 * (b - Pt);
                const ulonglong2 v0 = pb[0], v1 = pb[1];
#pragma unroll
                for (int k = 0; k < IPT; ++k) interact_pair_hi(v0, v1, nxh[k], nyh[k], nzh[k], pax[k], pay[k], paz[k]);
              }
            }
          } else {
            load_lo();
            bool need_mask = false;
#pragma unroll
            for (int k = 0; k < IPT; ++k) need_mask |= mlo[k] < P1 && mhi[k] >= P;
            if (!need_mask && P1 - P == kBoxPairs) {
#pragma unroll 4
              for (int b = P; b < P + kBoxPairs; ++b) {
                const ulonglong2 *pb = src + 4 * (b - Pt);
                const ulonglong2 v0 = pb[0], v1 = pb[1], v2 = pb[2], v3 = pb[3];
#pragma unroll
                for (int k = 0; k < IPT; ++k)
                  interact_pair<false>(v0, v1, v2, v3, nxh[k], nyh[k], nzh[k], nxl[k], nyl[k], nzl[k], false, false,
                                       pax[k], pay[k], paz[k]);
              }
            } else {
              // Only the pairs that may hold one of this warp's own targets
              // (per k an ascending, warp-uniform range) take the self test.
              int cur = P;
#pragma unroll
              for (int k = 0; k < IPT; ++k) {
                const int r0 = max(mlo[k], cur), r1 = min(mhi[k] + 1, P1);
                if (r0 < r1) {
                  unmasked(cur, r0);
                  masked(r0, r1);
                  cur = r1;
                }
              }
              unmasked(cur, P1);
            }
          }
          since_fold += P1 - P;
          if (since_fold >= kFoldPairs) {
            fold();
            since_fold = 0;
          }
          P = P1;
        }
        fold();
      }

    }
    __syncwarp();  // every lane is done with stage s
    if (lane == 0) mbar_arrive(&empty[s]);
    if (++s == K) {
      s = 0;
      par ^= 1u;
    }
  }
  if (!aborted && cur >= 0) flush();

  // No copy into this CTA's shared memory may outlive it: thread 0 waits
  // (bounded) for every tile it issued from the one warp 0 stopped at (after
  // the end marker there is none; after a wait that ran out, at most K).
  if (tid == 0)
    for (int u = ct; u < s_pc.issued; ++u) mbar_wait(&full[u % K], static_cast<uint32_t>(u / K) & 1u);
  __syncthreads();
  // The last CTA out resets the chunk counter for the next launch.
  if (tid == 0) {
    if (s_flag & 1) atomicOr(a.flags, kFlagTimeout);
    __threadfence();
    if (atomicAdd(a.dyn_ctr + 1, 1) == n_static - 1) {
      atomicExch(a.dyn_ctr, 0);
      atomicExch(a.dyn_ctr + 1, 0);
    }
  }
}

}  // namespace nb
