// Eq. 1 force kernel of the mixed path, each pair once (Newton's third law).
//
// One pair (p, j) gives the term on p, mu_j |d|^-3 d, and the reaction on
// j, -mu_p |d|^-3 d, from one difference d = r_j - r_p, one |d|^2 and one
// |d|^-3: 16 FP32 lane operations for the two interactions of a far pair
// (hi-only difference) instead of 24, 22 instead of 36 for a near pair
// (hi/lo difference).  The arithmetic of each term is that of the
// every-ordered-pair kernel (step_kernel.cuh): the same hi/lo split, the
// same far test, MUFU rsqrt.
//
// Decomposition: each system's stage (spatial order) is cut into blocks of
// B = 32 T entries; the work items are the block pairs (I, J), I <= J,
// handed out by a counter.  A CTA of W = T / 4 warps takes an item: warp p
// holds block I's entries [128 p, 128 p + 128) in registers, four per lane
// (slot a: entry 128 p + 32 a + lane).  Block J is cut into chunks of 64
// entries; in phase t the warp takes chunk c = (2 p + t) mod (T / 2).  The
// chunk's 32 stage pair blocks (two entries each, 64 B) are copied
// (cp.async) into the warp's shared memory a phase ahead, the four 16-byte
// pieces of each block into four arrays, so that at step k lane l reads
// pair block (l + k) mod 32 without bank conflicts, its two entries already
// packed as f32x2 operands: in 32 steps every source meets every target
// once, eight pairs per lane and step, the two sources of a lane in one
// packed instruction.  The sources' reaction sums rotate around the warp
// with shuffles, one lane per step; a CTA barrier closes each phase, and
// within a phase the warps' chunks differ, so each chunk belongs to one
// warp and its sums in shared memory take their terms in phase order.
//
// Sums, all float pairs (hi, lo) fed through TwoSum: a target's packed
// per-slot sums every two phases (64 terms per half), a source's reaction
// sums twice per phase (after 16 steps, when the sums of the sources of pair
// block l sit in lane l - 16, and at the end; 64 terms per half).
// Off-diagonal items: block I's sums go to row J of its bodies, block J's to
// row I.  Diagonal items (I == J) take each pair (target entry e, source
// entry f) with e < f, by weights on the two chunks that meet the warp's
// own entries (the others are wholly above or below them); each warp adds
// its targets' sums into the block's shared sums after the last phase, and
// the total goes to row I.  Entries past the end of a system's stage are
// inert (massless, far away, distinct).
//
// Far test: a chunk takes the hi-only difference when the union of the
// widened boxes (box_kernel) of the 64-entry stage groups holding the
// warp's targets and the one of the groups holding the chunk are disjoint
// (the bound of step_kernel.cuh holds for either term of the pair).
#include "nbody_dev.cuh"

namespace nb {

namespace {

// Per-warp shared scratch: two chunk buffers, the targets' negated lo parts
// (duplicated in both halves, read by the near path) and their running
// float-pair sums.
struct MsymWarp {
  // [buffer][piece][pair block]: the 16-byte pieces (xh0 xh1 yh0 yh1),
  // (zh0 zh1 mu0 mu1), (xl0 xl1 yl0 yl1), (zl0 zl1 - -) of a chunk's pair blocks
  float4 src[2][4][32];
  f2 tlo[4][3][32];     // [slot a][component][lane]
  float sum[4][6][32];  // [slot a][x hi, x lo, y hi, y lo, z hi, z lo][lane]
  float4 box[2];        // the union of the widened boxes of the targets' groups
};

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Union of the widened boxes of the stage groups that hold entries [e0, e1).
__device__ __forceinline__ void box_union(const float4 *boxes, int e0, int e1, float4 &lo, float4 &hi) {
  lo = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
  hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
  for (int g = (e0 >> 1) / kBoxPairs; g <= ((e1 - 1) >> 1) / kBoxPairs; ++g) {
    const float4 l = boxes[2 * g], h = boxes[2 * g + 1];
    lo.x = fminf(lo.x, l.x);
    lo.y = fminf(lo.y, l.y);
    lo.z = fminf(lo.z, l.z);
    hi.x = fmaxf(hi.x, h.x);
    hi.y = fmaxf(hi.y, h.y);
    hi.z = fmaxf(hi.z, h.z);
  }
}

__device__ __forceinline__ bool boxes_apart(const float4 &alo, const float4 &ahi, const float4 &blo,
                                            const float4 &bhi) {
  return alo.x > bhi.x || alo.y > bhi.y || alo.z > bhi.z || blo.x > ahi.x || blo.y > ahi.y || blo.z > ahi.z;
}

// Position (hi) and mu of local entry e of a system's stage (first stage
// entry s0, nst entries); past the end an inert entry: massless, far away,
// at a position of its own.
__device__ __forceinline__ float4 msym_hi(const float *cur, int s0, int e, int nst) {
  if (e < nst) {
    const float *q = cur + pair_off(s0 + e);
    return make_float4(q[kXh], q[kYh], q[kZh], q[kMu]);
  }
  const float x = 2.f * kPadCoord + 1e12f * static_cast<float>(e - nst);
  return make_float4(x, x, x, 0.f);
}

__device__ __forceinline__ float4 msym_lo(const float *cur, int s0, int e, int nst) {
  if (e < nst) {
    const float *q = cur + pair_off(s0 + e);
    return make_float4(q[kXl], q[kYl], q[kZl], 0.f);
  }
  return make_float4(0.f, 0.f, 0.f, 0.f);
}

// One chunk: 32 rotation steps of the chunk's sources past the lane's four
// targets; at step k lane l takes the two entries of pair block
// (l + k) mod 32 from the chunk buffer cb.  Reaction sums fold into the
// chunk's shared sums s_j (local chunk entries jc + 2 m + h for pair block
// m) half way and at the end.  MASKED (a diagonal item): a pair counts only
// if the target's entry, et0 + 32 a, precedes the source's, jc + 2 m + h.
// MU_SMEM: the targets' mu come from wmu ([slot a][lane], shared memory)
// instead of registers.
template <bool NEAR, bool MASKED, bool MU_SMEM>
__device__ __forceinline__ void msym_chunk(const float4 (*cb)[32], const f2 (&nxh)[4], const f2 (&nyh)[4],
                                           const f2 (&nzh)[4], const f2 (&tmu)[4], const f2 (*wmu)[32],
                                           const MsymWarp &ws, int lane,
                                           int et0, f2 (&ax)[4], f2 (&ay)[4], f2 (&az)[4], float *s_j, int BT,
                                           int jc) {
  f2 bx = 0ull, by = 0ull, bz = 0ull;
  // the reaction sums held here belong to the sources of pair block m
  auto fold = [&](int m) {
    const f2 b[3] = {bx, by, bz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float b0, b1;
      upk(b[d], b0, b1);
      const int e0 = jc + 2 * m;
      two_sum_acc(s_j[(2 * d) * BT + e0], s_j[(2 * d + 1) * BT + e0], -b0);
      two_sum_acc(s_j[(2 * d) * BT + e0 + 1], s_j[(2 * d + 1) * BT + e0 + 1], -b1);
    }
  };
  auto step = [&](int k) {
    const int m = (lane + k) & 31;
    const float4 A = cb[0][m], B = cb[1][m];
    const f2 sx = pk(A.x, A.y), sy = pk(A.z, A.w), sz = pk(B.x, B.y), sm = pk(B.z, B.w);
    f2 sxl = 0ull, syl = 0ull, szl = 0ull;
    if (NEAR) {
      const float4 C = cb[2][m];
      const float2 D = *reinterpret_cast<const float2 *>(&cb[3][m]);  // (zl0, zl1)
      sxl = pk(C.x, C.y);
      syl = pk(C.z, C.w);
      szl = pk(D.x, D.y);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      f2 dx = add2(sx, nxh[a]), dy = add2(sy, nyh[a]), dz = add2(sz, nzh[a]);
      if (NEAR) {
        dx = add2(dx, add2(sxl, ws.tlo[a][0][lane]));
        dy = add2(dy, add2(syl, ws.tlo[a][1][lane]));
        dz = add2(dz, add2(szl, ws.tlo[a][2][lane]));
      }
      f2 r2 = mul2(dx, dx);
      r2 = fma2(dy, dy, r2);
      r2 = fma2(dz, dz, r2);
      float ra, rb;
      upk(r2, ra, rb);
      float w0 = 1.f, w1 = 1.f;
      if (MASKED) {
        const int et = et0 + 32 * a, es = jc + 2 * m;
        w0 = et < es ? 1.f : 0.f;
        w1 = et < es + 1 ? 1.f : 0.f;
        ra = w0 != 0.f ? ra : 1.f;  // (a target with itself: r2 = 0)
        rb = w1 != 0.f ? rb : 1.f;
      }
      const f2 q = pk(rsqrt_approx(ra), rsqrt_approx(rb));
      const f2 q3 = mul2(mul2(q, q), q);
      f2 fi = mul2(sm, q3), fj = mul2(MU_SMEM ? wmu[a][lane] : tmu[a], q3);
      if (MASKED) {
        const f2 wgt = pk(w0, w1);
        fi = mul2(fi, wgt);
        fj = mul2(fj, wgt);
      }
      ax[a] = fma2(fi, dx, ax[a]);
      ay[a] = fma2(fi, dy, ay[a]);
      az[a] = fma2(fi, dz, az[a]);
      bx = fma2(fj, dx, bx);
      by = fma2(fj, dy, by);
      bz = fma2(fj, dz, bz);
    }
    const int src = (lane + 1) & 31;  // the sums follow their sources to the next lane's step
    bx = __shfl_sync(0xffffffffu, bx, src);
    by = __shfl_sync(0xffffffffu, by, src);
    bz = __shfl_sync(0xffffffffu, bz, src);
  };
#pragma unroll 1
  for (int k = 0; k < 16; ++k) step(k);
  fold((lane + 16) & 31);
  bx = by = bz = 0ull;
#pragma unroll 1
  for (int k = 16; k < 32; ++k) step(k);
  fold(lane);
}

}  // namespace

// MU_SMEM: the targets' mu in shared memory, which frees 8 registers in the
// rotation loop.  Used with 2,048-entry blocks (16-warp CTAs, one per SM),
// where it measured faster on GB300 (1,048,576 bodies: 395 against 403 ms
// per step); with 512-entry blocks its 4 KB per CTA cost an SM its fourth
// CTA (65,536 bodies: 1.71 against 1.64 ms), so they keep mu in registers.
template <bool MU_SMEM>
__global__ void __launch_bounds__(32 * kMsymMaxWarps, 1) force_msym_kernel(const MsymArgs a) {
  extern __shared__ __align__(16) unsigned char msym_smem[];
  __shared__ int s_item;
  grid_dependency_wait();    // staged sources and boxes of this step are complete
  grid_dependency_launch();  // the Verlet kernel may start launching
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int W = a.warps, T = a.tiles, BT = 32 * T, NC = T / 2;
  MsymWarp &ws = reinterpret_cast<MsymWarp *>(msym_smem)[w];
  // block J's sums of the item: [x hi, x lo, y hi, y lo, z hi, z lo][BT]
  float *s_j = reinterpret_cast<float *>(msym_smem + static_cast<size_t>(W) * sizeof(MsymWarp));
  // MU_SMEM: this warp's targets' mu, after the sums
  f2 (*wmu)[32] = reinterpret_cast<f2 (*)[32]>(s_j + 6 * BT) + 4 * w;
  const size_t N = static_cast<size_t>(a.N);
  const float *cur = a.cur;
  for (;;) {
    __syncthreads();  // the previous item's shared sums are consumed
    if (tid == 0) s_item = atomicAdd(a.ctr, 1);
    for (int k = tid; k < 6 * BT; k += 32 * W) s_j[k] = 0.f;
    __syncthreads();
    const int item = s_item;
    if (item >= a.n_pairs) break;
    const int4 pr = a.pairs[item];  // (first stage entry of the system, its bodies, block I, block J)
    const int s0 = pr.x, ns = pr.y, I = pr.z, J = pr.w;
    const int nst = (ns + 1) & ~1;  // the system's stage entries (padded to even)
    const bool diag = I == J;
    const int i0 = I * BT, j0 = J * BT;
    {
      const int p = w;               // one round: W = T / 4 warps cover block I
      const int ib = i0 + 128 * p;   // this warp's targets: local entries [ib, ib + 128)
      const bool p_live = ib < nst;  // warp-uniform
      // chunk cc into buffer bb: lane l copies pair block l (its four
      // pieces) if it lies inside the system, else writes two inert entries
      auto stage_chunk = [&](int cc, int bb) {
        const int jb = j0 + 64 * cc;
        const int e0 = jb + 2 * lane;  // the block's first local entry
        if (e0 < nst) {
          const float4 *src = reinterpret_cast<const float4 *>(cur) + static_cast<size_t>((s0 + e0) >> 1) * 4;
#pragma unroll
          for (int q = 0; q < 4; ++q) cp_async16(&ws.src[bb][q][lane], src + q);
        } else {
          const float x0 = 2.f * kPadCoord + 1e12f * static_cast<float>(e0 - nst), x1 = x0 + 1e12f;
          ws.src[bb][0][lane] = make_float4(x0, x1, x0, x1);
          ws.src[bb][1][lane] = make_float4(x0, x1, 0.f, 0.f);
          ws.src[bb][2][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
          ws.src[bb][3][lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cp_async_commit();
      };
      int c = (2 * p) % NC;
      if (p_live) stage_chunk(c, 0);
      f2 nxh[4], nyh[4], nzh[4], tmu[4], ax[4], ay[4], az[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int e = ib + 32 * s + lane;
        const float4 h = msym_hi(cur, s0, e, nst), l = msym_lo(cur, s0, e, nst);
        nxh[s] = pk(-h.x, -h.x);
        nyh[s] = pk(-h.y, -h.y);
        nzh[s] = pk(-h.z, -h.z);
        tmu[s] = pk(h.w, h.w);
        if (MU_SMEM) wmu[s][lane] = tmu[s];
        ws.tlo[s][0][lane] = pk(-l.x, -l.x);
        ws.tlo[s][1][lane] = pk(-l.y, -l.y);
        ws.tlo[s][2][lane] = pk(-l.z, -l.z);
#pragma unroll
        for (int f = 0; f < 6; ++f) ws.sum[s][f][lane] = 0.f;
        ax[s] = ay[s] = az[s] = 0ull;
      }
      if (p_live && lane == 0) box_union(a.boxes, s0 + ib, s0 + min(ib + 128, nst), ws.box[0], ws.box[1]);
      __syncwarp();
      // the targets' packed sums into their float pairs
      auto fold_targets = [&]() {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const f2 v[3] = {ax[s], ay[s], az[s]};
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            float v0, v1;
            upk(v[d], v0, v1);
            two_sum_acc(ws.sum[s][2 * d][lane], ws.sum[s][2 * d + 1][lane], v0);
            two_sum_acc(ws.sum[s][2 * d][lane], ws.sum[s][2 * d + 1][lane], v1);
          }
          ax[s] = ay[s] = az[s] = 0ull;
        }
      };
      for (int t = 0; t < NC; ++t) {
        const int cc = c;
        c = (2 * p + t + 1) % NC;
        const int jb = j0 + 64 * cc;  // the chunk: local entries [jb, jb + 64)
        // diagonal item: chunk tiles 2 cc, 2 cc + 1 against the warp's 4 p .. 4 p + 3
        const bool skip = diag && 2 * cc + 1 < 4 * p;
        const bool masked = diag && 2 * cc <= 4 * p + 3;
        if (p_live) {
          cp_async_wait_all();
          __syncwarp();  // every lane's copies (and inert entries) are in buffer t & 1
          // the next chunk into the other buffer, read last in the previous phase
          if (t + 1 < NC) stage_chunk(c, (t + 1) & 1);
          if (jb < nst && !skip) {
            float4 jlo, jhi;
            box_union(a.boxes, s0 + jb, s0 + min(jb + 64, nst), jlo, jhi);
            const bool far = boxes_apart(ws.box[0], ws.box[1], jlo, jhi);
            const float4(*cb)[32] = ws.src[t & 1];
            const int jc = 64 * cc, et0 = 128 * p + lane;
            if (far && !masked)
              msym_chunk<false, false, MU_SMEM>(cb, nxh, nyh, nzh, tmu, wmu, ws, lane, et0, ax, ay, az, s_j, BT, jc);
            else if (masked)
              msym_chunk<true, true, MU_SMEM>(cb, nxh, nyh, nzh, tmu, wmu, ws, lane, et0, ax, ay, az, s_j, BT, jc);
            else
              msym_chunk<true, false, MU_SMEM>(cb, nxh, nyh, nzh, tmu, wmu, ws, lane, et0, ax, ay, az, s_j, BT, jc);
          }
        }
        if ((t & 1) || t + 1 == NC) fold_targets();
        __syncthreads();  // phase done: the chunks change hands
      }
      if (p_live) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int e = ib + 32 * s + lane;
          if (diag) {  // into the block's shared sums (no warp takes these entries until the next barrier)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              const int k = 128 * p + 32 * s + lane;
              two_sum_acc(s_j[(2 * d) * BT + k], s_j[(2 * d + 1) * BT + k], ws.sum[s][2 * d][lane]);
              s_j[(2 * d + 1) * BT + k] += ws.sum[s][2 * d + 1][lane];
            }
          } else if (e < ns) {
            float2 *row = reinterpret_cast<float2 *>(a.partial) + static_cast<size_t>(J) * 3 * N;
            const int b = a.perm[s0 + e];
            row[b] = make_float2(ws.sum[s][0][lane], ws.sum[s][1][lane]);
            row[N + b] = make_float2(ws.sum[s][2][lane], ws.sum[s][3][lane]);
            row[2 * N + b] = make_float2(ws.sum[s][4][lane], ws.sum[s][5][lane]);
          }
        }
      }
    }
    __syncthreads();
    // block J's sums (on a diagonal item, the block's whole sums) to row I
    float2 *row = reinterpret_cast<float2 *>(a.partial) + static_cast<size_t>(I) * 3 * N;
    for (int k = tid; k < BT && j0 + k < ns; k += 32 * W) {
      const int b = a.perm[s0 + j0 + k];
      row[b] = make_float2(s_j[k], s_j[BT + k]);
      row[N + b] = make_float2(s_j[2 * BT + k], s_j[3 * BT + k]);
      row[2 * N + b] = make_float2(s_j[4 * BT + k], s_j[5 * BT + k]);
    }
  }
  // The last CTA out resets the item counter for the next launch.
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(a.ctr + 1, 1) == static_cast<int>(gridDim.x) - 1) {
      atomicExch(a.ctr, 0);
      atomicExch(a.ctr + 1, 0);
    }
  }
}

namespace {
bool msym_mu_smem(int tiles) { return tiles == kMsymMaxTiles; }
}  // namespace

size_t force_msym_smem_bytes(int tiles, int warps) {
  return static_cast<size_t>(warps) * sizeof(MsymWarp) + sizeof(float) * 6 * 32 * static_cast<size_t>(tiles) +
         (msym_mu_smem(tiles) ? sizeof(f2) * 4 * 32 * static_cast<size_t>(warps) : 0);
}

cudaError_t launch_force_msym(const MsymArgs &a, int grid, cudaStream_t s, bool chained) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(32 * a.warps);
  cfg.dynamicSmemBytes = force_msym_smem_bytes(a.tiles, a.warps);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  if (msym_mu_smem(a.tiles)) return cudaLaunchKernelEx(&cfg, force_msym_kernel<true>, a);
  return cudaLaunchKernelEx(&cfg, force_msym_kernel<false>, a);
}

int force_msym_ctas_per_sm(int tiles, int warps) {
  int occ = 0;
  const int max_smem = static_cast<int>(force_msym_smem_bytes(kMsymMaxTiles, kMsymMaxWarps));
  cudaError_t e = cudaFuncSetAttribute(force_msym_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(force_msym_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, msym_mu_smem(tiles) ? force_msym_kernel<true>
                                                                               : force_msym_kernel<false>,
                                                      32 * warps, force_msym_smem_bytes(tiles, warps));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

}  // namespace nb
