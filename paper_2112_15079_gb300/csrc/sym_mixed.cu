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
// entries; in phase t the warp takes chunk c = (2 p + t) mod (T / 2), two
// entries per lane (slot h: entry 64 c + 32 h + lane, packed in one f32x2
// register pair), and rotates them around the warp with shuffles: in 32
// steps every source meets every target once, eight pairs per lane and
// step, the two sources of a lane in one packed instruction.  The chunk's
// 2 KB of stage pair blocks are copied (cp.async) into the warp's shared
// memory a phase ahead.  The sources' reaction sums rotate with them; a
// CTA barrier closes each phase, and within a phase the warps' chunks
// differ, so each chunk belongs to one warp and its sums in shared memory
// take their terms in phase order.
//
// Sums, all float pairs (hi, lo) fed through TwoSum: a target's packed
// per-slot sums every two phases (64 terms per half), a source's reaction
// sums twice per phase (after 16 steps, when the sources that started in
// lane l sit in lane l - 16, and at the end; 64 terms per half).
// Off-diagonal items: block I's sums go to row J of its bodies, block J's to
// row I.  Diagonal items (I == J) take the 32-entry tile pairs (i, j) with
// i <= j once, i == j as the half rotation (offsets 1..16 for the target,
// 1..15 for the reaction), by weights on the two chunks that meet the
// warp's own tiles; each warp adds its targets' sums into the block's
// shared sums after the last phase, and the total goes to row I.  Entries past
// the end of a system's stage are inert (massless, far away, distinct).
//
// Far test: a chunk takes the hi-only difference when the union of the
// widened boxes (box_kernel) of the 64-entry stage groups holding the
// warp's targets and the one of the groups holding the chunk are disjoint
// (the bound of step_kernel.cuh holds for either term of the pair).
#include "nbody_dev.cuh"

namespace nb {

namespace {

// Per-warp shared scratch: the targets' negated lo parts (duplicated in both
// halves, read by the near path) and their running float-pair sums.
struct MsymWarp {
  float chunk[32 * 16];  // the next chunk's 32 stage pair blocks (cp.async, a phase ahead)
  f2 tlo[4][3][32];      // [slot a][component][lane]
  f2 clo[3][32];         // the chunk's lo parts [component][home lane] (slots packed), for the near path
  float sum[4][6][32];   // [slot a][x hi, x lo, y hi, y lo, z hi, z lo][lane]
  float4 box[2];         // the union of the widened boxes of the targets' groups
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

// Entry u (0..63) of a staged chunk whose first entry is local entry jb:
// hi and mu into h, lo into l (inert past the system's nst entries).
__device__ __forceinline__ void chunk_entry(const float *chunk, int jb, int u, int nst, float4 &h, float4 &l) {
  if (jb + u < nst) {
    const float *q = chunk + pair_off(u);
    h = make_float4(q[kXh], q[kYh], q[kZh], q[kMu]);
    l = make_float4(q[kXl], q[kYl], q[kZl], 0.f);
  } else {
    const float x = 2.f * kPadCoord + 1e12f * static_cast<float>(jb + u - nst);
    h = make_float4(x, x, x, 0.f);
    l = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Diagonal items: the class of the tile pair (target tile it, source tile
// jt), 2 bits: tile pairs i < j in full (1), i == j as the half rotation
// (2), i > j not at all (0: that pair is the warp holding tile j's).
__device__ __forceinline__ int diag_class(int it, int jt) { return it < jt ? 1 : it == jt ? 2 : 0; }

// The target weight and the reaction weight of a pair of class cls at
// rotation offset k (half rotation: offsets 1..16 for the target, 1..15 for
// the reaction).
__device__ __forceinline__ void diag_weights(int cls, int k, float &wt, float &wr) {
  wt = (cls == 1 || (cls == 2 && k >= 1 && k <= 16)) ? 1.f : 0.f;
  wr = (cls == 1 || (cls == 2 && k >= 1 && k <= 15)) ? 1.f : 0.f;
}

// One chunk: 32 rotation steps of the lane's two packed sources past its
// four targets.  Reaction sums fold into the chunk's shared sums s_j (local
// chunk entry jc + 32 h + lane) half way and at the end.  NEAR: the sources'
// lo parts come from ws.clo (at step k the lane holds the sources of lane
// lane + k).  MASKED: diagonal weights, from the class of the tile pair of
// target slot a and source slot h in bits 2 (2 a + h) of codes.
template <bool NEAR, bool MASKED>
__device__ __forceinline__ void msym_chunk(f2 sx, f2 sy, f2 sz, f2 sm, const f2 (&nxh)[4],
                                           const f2 (&nyh)[4], const f2 (&nzh)[4], const f2 (&tmu)[4],
                                           const MsymWarp &ws, int lane, int codes, f2 (&ax)[4],
                                           f2 (&ay)[4], f2 (&az)[4], float *s_j, int BT, int jc) {
  f2 bx = 0ull, by = 0ull, bz = 0ull;
  // the reaction sums held here belong to the sources that started in lane `home`
  auto fold = [&](int home) {
    const f2 b[3] = {bx, by, bz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float b0, b1;
      upk(b[d], b0, b1);
      const int e0 = jc + home, e1 = jc + 32 + home;
      two_sum_acc(s_j[(2 * d) * BT + e0], s_j[(2 * d + 1) * BT + e0], -b0);
      two_sum_acc(s_j[(2 * d) * BT + e1], s_j[(2 * d + 1) * BT + e1], -b1);
    }
  };
  auto step = [&](int k) {
    f2 sxl = 0ull, syl = 0ull, szl = 0ull;
    if (NEAR) {
      const int hl = (lane + k) & 31;
      sxl = ws.clo[0][hl];
      syl = ws.clo[1][hl];
      szl = ws.clo[2][hl];
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
      float wt0 = 1.f, wr0 = 1.f, wt1 = 1.f, wr1 = 1.f;
      if (MASKED) {
        diag_weights((codes >> (4 * a)) & 3, k, wt0, wr0);
        diag_weights((codes >> (4 * a + 2)) & 3, k, wt1, wr1);
        ra = (wt0 != 0.f || wr0 != 0.f) ? ra : 1.f;  // a target with itself: r2 = 0
        rb = (wt1 != 0.f || wr1 != 0.f) ? rb : 1.f;
      }
      const f2 q = pk(rsqrt_approx(ra), rsqrt_approx(rb));
      const f2 q3 = mul2(mul2(q, q), q);
      f2 fi = mul2(sm, q3), fj = mul2(tmu[a], q3);
      if (MASKED) {
        fi = mul2(fi, pk(wt0, wt1));
        fj = mul2(fj, pk(wr0, wr1));
      }
      ax[a] = fma2(fi, dx, ax[a]);
      ay[a] = fma2(fi, dy, ay[a]);
      az[a] = fma2(fi, dz, az[a]);
      bx = fma2(fj, dx, bx);
      by = fma2(fj, dy, by);
      bz = fma2(fj, dz, bz);
    }
    const int src = (lane + 1) & 31;
    sx = __shfl_sync(0xffffffffu, sx, src);
    sy = __shfl_sync(0xffffffffu, sy, src);
    sz = __shfl_sync(0xffffffffu, sz, src);
    sm = __shfl_sync(0xffffffffu, sm, src);
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
      // copy chunk cc's stage pair blocks (those inside the system) into ws.chunk
      auto stage_chunk = [&](int cc) {
        const int jb = j0 + 64 * cc;
        const int npb = min(32, (nst - jb) / 2);
        const float *src = cur + static_cast<size_t>((s0 + jb) >> 1) * 16;
        for (int q = lane; q < 4 * npb; q += 32) cp_async16(&ws.chunk[4 * q], src + 4 * q);
        cp_async_commit();
      };
      int c = (2 * p) % NC;
      if (p_live) stage_chunk(c);
      f2 nxh[4], nyh[4], nzh[4], tmu[4], ax[4], ay[4], az[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int e = ib + 32 * s + lane;
        const float4 h = msym_hi(cur, s0, e, nst), l = msym_lo(cur, s0, e, nst);
        nxh[s] = pk(-h.x, -h.x);
        nyh[s] = pk(-h.y, -h.y);
        nzh[s] = pk(-h.z, -h.z);
        tmu[s] = pk(h.w, h.w);
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
          __syncwarp();  // every lane's copies have landed
          float4 h0, l0, h1, l1;
          chunk_entry(ws.chunk, jb, lane, nst, h0, l0);
          chunk_entry(ws.chunk, jb, 32 + lane, nst, h1, l1);
          ws.clo[0][lane] = pk(l0.x, l1.x);
          ws.clo[1][lane] = pk(l0.y, l1.y);
          ws.clo[2][lane] = pk(l0.z, l1.z);
          __syncwarp();  // the chunk is read: the next one may land over it
          if (t + 1 < NC) stage_chunk(c);
          if (jb < nst && !skip) {
            float4 jlo, jhi;
            box_union(a.boxes, s0 + jb, s0 + min(jb + 64, nst), jlo, jhi);
            const bool far = boxes_apart(ws.box[0], ws.box[1], jlo, jhi);
            const f2 sx = pk(h0.x, h1.x), sy = pk(h0.y, h1.y), sz = pk(h0.z, h1.z), sm = pk(h0.w, h1.w);
            const int jc = 64 * cc;
            if (far && !masked)
              msym_chunk<false, false>(sx, sy, sz, sm, nxh, nyh, nzh, tmu, ws, lane, 0, ax, ay, az, s_j, BT, jc);
            else if (masked) {
              int codes = 0;
              for (int u = 0; u < 8; ++u) codes |= diag_class(4 * p + (u >> 1), 2 * cc + (u & 1)) << (2 * u);
              msym_chunk<true, true>(sx, sy, sz, sm, nxh, nyh, nzh, tmu, ws, lane, codes, ax, ay, az, s_j, BT, jc);
            } else {
              msym_chunk<true, false>(sx, sy, sz, sm, nxh, nyh, nzh, tmu, ws, lane, 0, ax, ay, az, s_j, BT, jc);
            }
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

size_t force_msym_smem_bytes(int tiles, int warps) {
  return static_cast<size_t>(warps) * sizeof(MsymWarp) + sizeof(float) * 6 * 32 * static_cast<size_t>(tiles);
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
  return cudaLaunchKernelEx(&cfg, force_msym_kernel, a);
}

int force_msym_ctas_per_sm(int tiles, int warps) {
  int occ = 0;
  cudaError_t e = cudaFuncSetAttribute(force_msym_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(force_msym_smem_bytes(kMsymMaxTiles, kMsymMaxWarps)));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, force_msym_kernel, 32 * warps,
                                                      force_msym_smem_bytes(tiles, warps));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

}  // namespace nb
