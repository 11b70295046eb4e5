// Eq. 1 force kernel of the FP64 path, each pair once (Newton's third law).
//
// The FP64 pipe bounds this path, and one interaction of Eq. 1 takes 16 FP64
// operations (3 differences, 3 for |d|^2, 6 for |d|^-3 from the MUFU seed and
// its series, the product with mu_j, 3 accumulations).  The pair (p, j) and
// its reaction share the first 12 of them: evaluating each unordered pair
// once and accumulating both terms -- a_p += mu_j |d|^-3 d and
// a_j -= mu_p |d|^-3 d -- takes 20 operations for two interactions.
//
// Decomposition: each system's bodies are cut into blocks of 64 (two warp
// tiles of 32); the work items are the block pairs (I, J), I <= J, handed
// out by a counter (off-diagonal pairs first, the cheaper diagonal ones
// last).  A CTA of two warps takes an item: warp w keeps the 32 bodies of
// tile w of block I in registers and, for each tile t of block J, loads its
// 32 bodies as the "sources" and rotates them (positions, masses and their
// reaction sums) once around the warp with shuffles: after 32 steps every
// source has met every target once and its reaction sum is back in its own
// lane, with no FP64 reduction.  A tile paired with itself (diagonal items)
// rotates 16 steps (the 16th for the target side only: lanes L and L + 16
// meet twice).  The two warps' reaction sums for a J tile are added in a
// fixed order in shared memory.
//
// Output: block I's sums go to partial row J of its bodies, block J's to row
// I (a diagonal item adds both into row I); the Verlet kernel adds a body's
// rows 0 .. blocks-1 in order, so the result does not depend on which CTA
// took which item.
#include "nbody_dev.cuh"

namespace nb {

namespace {

__device__ __forceinline__ double4_32a sym_load(const double4_32a *cur, int64_t sb, int il, int ns, double pad) {
  if (il < ns) return cur[sb + il];
  // outside the system: inert (massless, far away, distinct per lane)
  return make_double4_32a(pad, 0.0, 0.0, 0.0);
}

__device__ __forceinline__ void sym_pair(double xi, double yi, double zi, double mi, double xj, double yj, double zj,
                                         double mj, double &ax, double &ay, double &az, double &bx, double &by,
                                         double &bz, bool react) {
  const double dx = xj - xi, dy = yj - yi, dz = zj - zi;
  const double s3 = inv_r3(fma(dz, dz, fma(dy, dy, dx * dx)));
  const double fi = mj * s3;
  ax = fma(fi, dx, ax);
  ay = fma(fi, dy, ay);
  az = fma(fi, dz, az);
  if (react) {
    const double fj = mi * s3;
    bx = fma(-fj, dx, bx);
    by = fma(-fj, dy, by);
    bz = fma(-fj, dz, bz);
  }
}

}  // namespace

__global__ void __launch_bounds__(kSymThreads) force_sym_kernel(const SymArgs a) {
  __shared__ double s_b[2][2][3][32];  // reaction sums [warp][J tile][component][lane]
  __shared__ int s_item;
  grid_dependency_wait();    // staged sources of this step are complete
  grid_dependency_launch();  // the Verlet kernel may start launching
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const size_t N = static_cast<size_t>(a.N);
  for (;;) {
    __syncthreads();  // the previous item's shared sums are consumed
    if (tid == 0) s_item = atomicAdd(a.ctr, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= a.n_pairs) break;
    const int4 pr = a.pairs[item];  // (first body of the system, its bodies, block I, block J)
    const int64_t sb = pr.x;
    const int ns = pr.y, I = pr.z, J = pr.w;
    const double4_32a pi = sym_load(a.cur, sb, I * kSymBlock + w * 32 + lane, ns, 1e15 * (lane + 1));
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int t = 0; t < 2; ++t) {
      double bx = 0.0, by = 0.0, bz = 0.0;
      if (!(I == J && t < w)) {  // tile pair (w, t) with t < w of a diagonal item is (t, w), warp t's
        const double4_32a pj0 = sym_load(a.cur, sb, J * kSymBlock + t * 32 + lane, ns, 1e15 * (lane + 1) + 5e14);
        double xj = pj0.x, yj = pj0.y, zj = pj0.z, mj = pj0.w;
        auto rotate = [&]() {
          const int src = (lane + 1) & 31;
          xj = __shfl_sync(0xffffffffu, xj, src);
          yj = __shfl_sync(0xffffffffu, yj, src);
          zj = __shfl_sync(0xffffffffu, zj, src);
          mj = __shfl_sync(0xffffffffu, mj, src);
          bx = __shfl_sync(0xffffffffu, bx, src);
          by = __shfl_sync(0xffffffffu, by, src);
          bz = __shfl_sync(0xffffffffu, bz, src);
        };
        if (I == J && t == w) {  // a tile with itself: offsets 1..15 both ways, 16 one way
#pragma unroll 4
          for (int k = 1; k <= 16; ++k) {
            rotate();
            sym_pair(pi.x, pi.y, pi.z, pi.w, xj, yj, zj, mj, ax, ay, az, bx, by, bz, k < 16);
          }
          // lane L holds the sums of lane L + 16: hand them back
          const int back = (lane + 16) & 31;
          bx = __shfl_sync(0xffffffffu, bx, back);
          by = __shfl_sync(0xffffffffu, by, back);
          bz = __shfl_sync(0xffffffffu, bz, back);
        } else {
#pragma unroll 4
          for (int k = 0; k < 32; ++k) {
            sym_pair(pi.x, pi.y, pi.z, pi.w, xj, yj, zj, mj, ax, ay, az, bx, by, bz, true);
            rotate();
          }
        }
      }
      s_b[w][t][0][lane] = bx;
      s_b[w][t][1][lane] = by;
      s_b[w][t][2][lane] = bz;
    }
    __syncthreads();
    // thread (w, lane): body J*64 + tid of block J (reaction sums of both
    // warps, warp 0 first) and body I*64 + tid of block I (its own sums)
    const int jl = J * kSymBlock + tid, il = I * kSymBlock + tid;
    double rj[3];
    for (int d = 0; d < 3; ++d) rj[d] = s_b[0][w][d][lane] + s_b[1][w][d][lane];
    if (I == J) {
      if (il < ns) {
        double *row = a.partial + static_cast<size_t>(I) * 3 * N;
        row[sb + il] = ax + rj[0];
        row[N + sb + il] = ay + rj[1];
        row[2 * N + sb + il] = az + rj[2];
      }
    } else {
      if (il < ns) {
        double *row = a.partial + static_cast<size_t>(J) * 3 * N;
        row[sb + il] = ax;
        row[N + sb + il] = ay;
        row[2 * N + sb + il] = az;
      }
      if (jl < ns) {
        double *row = a.partial + static_cast<size_t>(I) * 3 * N;
        row[sb + jl] = rj[0];
        row[N + sb + jl] = rj[1];
        row[2 * N + sb + jl] = rj[2];
      }
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

// Wide blocks, for systems whose 64-body blocks would need too many partial
// rows (one per block): blocks of B = 32 T bodies (T tiles, a power of two,
// kSymWideMinTiles .. kSymWideMaxTiles), so a body has one row per B bodies
// of its system.  A CTA of kSymWideWarps warps takes an item (I, J).  In
// round r warp w holds tile p = r W + w of block I in registers; in phase
// t = 0 .. T-1 it rotates tile q = (p + t) mod T of block J past it, as
// force_sym_kernel does, and adds the tile's reaction sums into block J's
// sums in shared memory.  A CTA barrier closes each phase, and within a
// phase the warps' q differ, so each tile's shared sums take their terms in
// phase order, whichever warp runs first.  Block I's sums of a tile are
// added per tile pair, in phase order.  Off-diagonal items: block I's sums
// go to row J, block J's shared sums to row I.  A diagonal item takes the
// tile pairs q >= p only (q == p as the 16-step half rotation); each warp
// adds its tile's own sums into the shared sums after its round, and the
// total goes to row I.  Tiles past the end of the system are skipped.
__global__ void __launch_bounds__(kSymWideThreads) force_sym_wide_kernel(const SymArgs a) {
  extern __shared__ double s_acc[];  // [3][32 T]: block J's reaction sums of the item
  __shared__ int s_item;
  grid_dependency_wait();    // staged sources of this step are complete
  grid_dependency_launch();  // the Verlet kernel may start launching
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int T = a.tiles, BT = 32 * T;
  const size_t N = static_cast<size_t>(a.N);
  for (;;) {
    __syncthreads();  // the previous item's shared sums are consumed
    if (tid == 0) s_item = atomicAdd(a.ctr, 1);
    for (int k = tid; k < 3 * BT; k += kSymWideThreads) s_acc[k] = 0.0;
    __syncthreads();
    const int item = s_item;
    if (item >= a.n_pairs) break;
    const int4 pr = a.pairs[item];  // (first body of the system, its bodies, block I, block J)
    const int64_t sb = pr.x;
    const int ns = pr.y, I = pr.z, J = pr.w;
    const bool diag = I == J;
    const int i0 = I * BT, j0 = J * BT;  // first body of each block within the system
    for (int r = 0; r < T; r += kSymWideWarps) {
      const int p = r + w;
      const bool p_live = i0 + p * 32 < ns;  // warp-uniform
      const double4_32a pi = sym_load(a.cur, sb, i0 + p * 32 + lane, ns, 1e15 * (lane + 1));
      double ax = 0.0, ay = 0.0, az = 0.0;
      // the next phase's J tile, loaded a phase ahead
      int q = p;
      double4_32a pn = sym_load(a.cur, sb, j0 + q * 32 + lane, ns, 1e15 * (lane + 1) + 5e14);
      for (int t = 0; t < T; ++t) {
        const double4_32a pj0 = pn;
        const int qn = (p + t + 1) & (T - 1);
        if (t + 1 < T) pn = sym_load(a.cur, sb, j0 + qn * 32 + lane, ns, 1e15 * (lane + 1) + 5e14);
        if (p_live && j0 + q * 32 < ns && !(diag && q < p)) {  // (q < p on a diagonal item: tile q's warp's pair)
          double xj = pj0.x, yj = pj0.y, zj = pj0.z, mj = pj0.w;
          double tx = 0.0, ty = 0.0, tz = 0.0, bx = 0.0, by = 0.0, bz = 0.0;
          auto rotate = [&]() {
            const int src = (lane + 1) & 31;
            xj = __shfl_sync(0xffffffffu, xj, src);
            yj = __shfl_sync(0xffffffffu, yj, src);
            zj = __shfl_sync(0xffffffffu, zj, src);
            mj = __shfl_sync(0xffffffffu, mj, src);
            bx = __shfl_sync(0xffffffffu, bx, src);
            by = __shfl_sync(0xffffffffu, by, src);
            bz = __shfl_sync(0xffffffffu, bz, src);
          };
          if (diag && q == p) {  // a tile with itself: offsets 1..15 both ways, 16 one way
#pragma unroll 4
            for (int k = 1; k <= 16; ++k) {
              rotate();
              sym_pair(pi.x, pi.y, pi.z, pi.w, xj, yj, zj, mj, tx, ty, tz, bx, by, bz, k < 16);
            }
            const int back = (lane + 16) & 31;
            bx = __shfl_sync(0xffffffffu, bx, back);
            by = __shfl_sync(0xffffffffu, by, back);
            bz = __shfl_sync(0xffffffffu, bz, back);
          } else {
#pragma unroll 4
            for (int k = 0; k < 32; ++k) {
              sym_pair(pi.x, pi.y, pi.z, pi.w, xj, yj, zj, mj, tx, ty, tz, bx, by, bz, true);
              rotate();
            }
          }
          ax += tx;
          ay += ty;
          az += tz;
          double *acc = s_acc + q * 32 + lane;
          acc[0] += bx;
          acc[BT] += by;
          acc[2 * BT] += bz;
        }
        q = qn;
        __syncthreads();  // phase done: the J tiles change hands
      }
      if (p_live) {
        const int il = i0 + p * 32 + lane;
        if (diag) {  // tile p's own sums join its shared sums (no warp takes tile p until the next barrier)
          double *acc = s_acc + p * 32 + lane;
          acc[0] += ax;
          acc[BT] += ay;
          acc[2 * BT] += az;
        } else if (il < ns) {
          double *row = a.partial + static_cast<size_t>(J) * 3 * N;
          row[sb + il] = ax;
          row[N + sb + il] = ay;
          row[2 * N + sb + il] = az;
        }
      }
    }
    __syncthreads();
    // block J's sums (on a diagonal item, the block's whole sums) to row I
    double *row = a.partial + static_cast<size_t>(I) * 3 * N;
    for (int k = tid; k < BT && j0 + k < ns; k += kSymWideThreads) {
      row[sb + j0 + k] = s_acc[k];
      row[N + sb + j0 + k] = s_acc[BT + k];
      row[2 * N + sb + j0 + k] = s_acc[2 * BT + k];
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

// The adjoint's vector-Jacobian product of Eq. 1 (see vjp.cu), each pair
// once.  For the pair (q, j), d = r_j - r_q, s3 = |d|^-3, s5 = |d|^-5 and
// u = mu_q w_j - mu_j w_q, the q term s3 u - 3 s5 (d.u) d changes sign
// under q <-> j (K(d) is even in d, u is odd), and the mass terms are
// s3 (w_j . d) for q and -s3 (w_q . d) for j.  Rows hold 4 values per body
// (the three components and the mass sum), block I's sums in row J, block
// J's in row I, as in force_sym_kernel.
__global__ void __launch_bounds__(kSymThreads) vjp_sym_kernel(const VjpSymArgs a) {
  __shared__ double s_b[2][2][4][32];  // reaction sums [warp][J tile][component][lane]
  __shared__ int s_item;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const size_t N = static_cast<size_t>(a.N);
  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(a.ctr, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= a.n_pairs) break;
    const int4 pr = a.pairs[item];
    const int64_t sb = pr.x;
    const int ns = pr.y, I = pr.z, J = pr.w;
    const int iq = I * kSymBlock + w * 32 + lane;
    const double4_32a pq = sym_load(a.pos, sb, iq, ns, 1e15 * (lane + 1));
    const double4_32a wq = iq < ns ? a.w[sb + iq] : make_double4_32a(0.0, 0.0, 0.0, 0.0);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int t = 0; t < 2; ++t) {
      double b[4] = {0.0, 0.0, 0.0, 0.0};
      if (!(I == J && t < w)) {  // tile pair (w, t) with t < w of a diagonal item is (t, w), warp t's
        const int ij = J * kSymBlock + t * 32 + lane;
        const double4_32a pj0 = sym_load(a.pos, sb, ij, ns, 1e15 * (lane + 1) + 5e14);
        const double4_32a wj0 = ij < ns ? a.w[sb + ij] : make_double4_32a(0.0, 0.0, 0.0, 0.0);
        double xj = pj0.x, yj = pj0.y, zj = pj0.z, mj = pj0.w, wjx = wj0.x, wjy = wj0.y, wjz = wj0.z;
        auto rotate = [&]() {
          const int src = (lane + 1) & 31;
          xj = __shfl_sync(0xffffffffu, xj, src);
          yj = __shfl_sync(0xffffffffu, yj, src);
          zj = __shfl_sync(0xffffffffu, zj, src);
          mj = __shfl_sync(0xffffffffu, mj, src);
          wjx = __shfl_sync(0xffffffffu, wjx, src);
          wjy = __shfl_sync(0xffffffffu, wjy, src);
          wjz = __shfl_sync(0xffffffffu, wjz, src);
#pragma unroll
          for (int c = 0; c < 4; ++c) b[c] = __shfl_sync(0xffffffffu, b[c], src);
        };
        auto pair = [&](bool react) {
          const double dx = xj - pq.x, dy = yj - pq.y, dz = zj - pq.z;
          const double y = inv_r1(fma(dz, dz, fma(dy, dy, dx * dx)));
          const double y2 = y * y;
          const double s3 = y * y2;
          const double s5 = s3 * y2;
          const double ux = fma(-mj, wq.x, pq.w * wjx);
          const double uy = fma(-mj, wq.y, pq.w * wjy);
          const double uz = fma(-mj, wq.z, pq.w * wjz);
          const double t3 = 3.0 * s5 * fma(dz, uz, fma(dy, uy, dx * ux));
          const double tx = fma(-t3, dx, s3 * ux), ty = fma(-t3, dy, s3 * uy), tz = fma(-t3, dz, s3 * uz);
          acc[0] += tx;
          acc[1] += ty;
          acc[2] += tz;
          acc[3] = fma(s3, fma(wjz, dz, fma(wjy, dy, wjx * dx)), acc[3]);
          if (react) {
            b[0] -= tx;
            b[1] -= ty;
            b[2] -= tz;
            b[3] = fma(-s3, fma(wq.z, dz, fma(wq.y, dy, wq.x * dx)), b[3]);
          }
        };
        if (I == J && t == w) {
#pragma unroll 2
          for (int k = 1; k <= 16; ++k) {
            rotate();
            pair(k < 16);
          }
          const int back = (lane + 16) & 31;
#pragma unroll
          for (int c = 0; c < 4; ++c) b[c] = __shfl_sync(0xffffffffu, b[c], back);
        } else {
#pragma unroll 2
          for (int k = 0; k < 32; ++k) {
            pair(true);
            rotate();
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) s_b[w][t][c][lane] = b[c];
    }
    __syncthreads();
    const int jl = J * kSymBlock + tid, il = I * kSymBlock + tid;
    double rj[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) rj[c] = s_b[0][w][c][lane] + s_b[1][w][c][lane];
    if (I == J) {
      if (il < ns) {
        double *row = a.partial + static_cast<size_t>(I) * 4 * N;
#pragma unroll
        for (int c = 0; c < 4; ++c) row[c * N + sb + il] = acc[c] + rj[c];
      }
    } else {
      if (il < ns) {
        double *row = a.partial + static_cast<size_t>(J) * 4 * N;
#pragma unroll
        for (int c = 0; c < 4; ++c) row[c * N + sb + il] = acc[c];
      }
      if (jl < ns) {
        double *row = a.partial + static_cast<size_t>(I) * 4 * N;
#pragma unroll
        for (int c = 0; c < 4; ++c) row[c * N + sb + jl] = rj[c];
      }
    }
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(a.ctr + 1, 1) == static_cast<int>(gridDim.x) - 1) {
      atomicExch(a.ctr, 0);
      atomicExch(a.ctr + 1, 0);
    }
  }
}

cudaError_t launch_vjp_sym(const VjpSymArgs &a, int grid, cudaStream_t s) {
  vjp_sym_kernel<<<grid, kSymThreads, 0, s>>>(a);
  return cudaGetLastError();
}

size_t force_sym_smem_bytes(int tiles) {
  return tiles == 2 ? 0 : sizeof(double) * 3 * 32 * static_cast<size_t>(tiles);
}

cudaError_t launch_force_sym(const SymArgs &a, int grid, cudaStream_t s, bool chained) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(a.tiles == 2 ? kSymThreads : kSymWideThreads);
  cfg.dynamicSmemBytes = force_sym_smem_bytes(a.tiles);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  if (a.tiles == 2) return cudaLaunchKernelEx(&cfg, force_sym_kernel, a);
  return cudaLaunchKernelEx(&cfg, force_sym_wide_kernel, a);
}

int force_sym_ctas_per_sm(int tiles) {
  int occ = 0;
  cudaError_t e;
  if (tiles == 2) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, force_sym_kernel, kSymThreads, 0);
  } else {
    const size_t smem = force_sym_smem_bytes(tiles);
    e = cudaFuncSetAttribute(force_sym_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(force_sym_smem_bytes(kSymWideMaxTiles)));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, force_sym_wide_kernel, kSymWideThreads, smem);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

}  // namespace nb
