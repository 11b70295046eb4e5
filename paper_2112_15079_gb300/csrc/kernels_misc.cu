// Per-body kernels around the Eq. 1 force launches: the Verlet step
// completion (Eqs. 4 and 3), the RK4 stage completion and stage-1 prep, the
// staging / pre-drift kernel, the energy kernels, and the force-launch
// dispatcher.
#include <mutex>
#include <type_traits>

#include "nbody_dev.cuh"

namespace nb {

bool force_fp64_supported(int threads, int ipt);
bool force_mixed_supported(int threads, int ipt);
cudaError_t run_force_fp64(int op, int threads, int ipt, int grid, size_t smem, const ForceArgs &a, cudaStream_t s,
                           bool chained, int *occ);
cudaError_t run_force_mixed(int op, int threads, int ipt, int grid, size_t smem, const ForceArgs &a, cudaStream_t s,
                            bool chained, int *occ);

static cudaError_t run_force(int precision, int op, int threads, int ipt, int grid, size_t smem, const ForceArgs &a,
                             cudaStream_t s, bool chained, int *occ) {
  return precision == 0 ? run_force_fp64(op, threads, ipt, grid, smem, a, s, chained, occ)
                        : run_force_mixed(op, threads, ipt, grid, smem, a, s, chained, occ);
}

cudaError_t launch_force(int precision, int threads, int ipt, int grid, size_t smem, const ForceArgs &a,
                         cudaStream_t s, bool chained) {
  return run_force(precision, 0, threads, ipt, grid, smem, a, s, chained, nullptr);
}

cudaError_t force_set_smem(int precision, int threads, int ipt, size_t smem) {
  // Read-and-raise of a limit shared by every context (and host thread).
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  return run_force(precision, 1, threads, ipt, 0, smem, ForceArgs{}, nullptr, false, nullptr);
}

int force_max_ctas_per_sm(int precision, int threads, int ipt, size_t smem) {
  int occ = 0;
  if (run_force(precision, 2, threads, ipt, 0, smem, ForceArgs{}, nullptr, false, &occ) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

bool force_config_supported(int precision, int threads, int ipt) {
  return precision == 0 ? force_fp64_supported(threads, ipt) : force_mixed_supported(threads, ipt);
}

size_t force_smem_bytes(int precision, int tj, int stages) {
  // 32 bytes per staged source in both layouts; the mixed stage also holds
  // the boxes of the source groups its tile touches
  return static_cast<size_t>(stages) * (static_cast<size_t>(tj) * 32 + (precision == 1 ? (tj / 64 + 2) * 32 : 0));
}

// ---------------------------------------------------------------------------
// Widened boxes of the mixed stage's source groups for the next force launch:
// group g = stage pairs [kBoxPairs g, kBoxPairs (g + 1)), one warp per group,
// lane l reading pairs kBoxPairs g + l + 32 i.  The box of the hi parts is widened on
// every side by kFarKappa times the largest lo part (see step_kernel.cuh).
// Padding sources (coordinate kPadCoord, mu = 0) stay out of the box; a group
// of padding only gets an empty box (low corner +inf, high corner -inf),
// which the far test finds far from every warp.
// ---------------------------------------------------------------------------
constexpr int kBoxWarps = 8;  // groups per CTA

__global__ void __launch_bounds__(32 * kBoxWarps) box_kernel(const float4 *stage, int64_t n_pairs, float4 *boxes) {
  grid_dependency_wait();  // the stage was written by the previous kernel
  grid_dependency_launch();
  const int64_t g = static_cast<int64_t>(blockIdx.x) * kBoxWarps + threadIdx.x / 32;
  const int64_t n_groups = (n_pairs + kBoxPairs - 1) / kBoxPairs;
  if (g >= n_groups) return;  // warp-uniform
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY}, lo[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < kBoxPairs / 32; ++i) {
    const int64_t b = g * kBoxPairs + (threadIdx.x & 31) + 32 * i;
    if (b >= n_pairs) break;
    // (xh0 xh1 yh0 yh1) (zh0 zh1 mu0 mu1) (xl0 xl1 yl0 yl1) (zl0 zl1 - -)
    const float4 A = stage[4 * b], B = stage[4 * b + 1], C = stage[4 * b + 2], D = stage[4 * b + 3];
    const float hx[2] = {A.x, A.y}, hy[2] = {A.z, A.w}, hz[2] = {B.x, B.y}, mu[2] = {B.z, B.w};
    const float lx[2] = {C.x, C.y}, ly[2] = {C.z, C.w}, lz[2] = {D.x, D.y};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      if (hx[e] == kPadCoord && mu[e] == 0.f) continue;
      mn[0] = fminf(mn[0], hx[e]);
      mn[1] = fminf(mn[1], hy[e]);
      mn[2] = fminf(mn[2], hz[e]);
      mx[0] = fmaxf(mx[0], hx[e]);
      mx[1] = fmaxf(mx[1], hy[e]);
      mx[2] = fmaxf(mx[2], hz[e]);
      lo[0] = fmaxf(lo[0], fabsf(lx[e]));
      lo[1] = fmaxf(lo[1], fabsf(ly[e]));
      lo[2] = fmaxf(lo[2], fabsf(lz[e]));
    }
  }
  warp_box(mn[0], mn[1], mn[2], mx[0], mx[1], mx[2], lo[0], lo[1], lo[2], boxes + 2 * g);
}

cudaError_t launch_boxes(const void *stage, int64_t n_pairs, float4 *boxes, cudaStream_t s, bool chained) {
  const int64_t n_groups = (n_pairs + kBoxPairs - 1) / kBoxPairs;
  if (n_groups <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>((n_groups + kBoxWarps - 1) / kBoxWarps));
  cfg.blockDim = dim3(32 * kBoxWarps);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, box_kernel, static_cast<const float4 *>(stage), n_pairs, boxes);
}

// ---------------------------------------------------------------------------
// Completes a step for VerletShape<PREC>::kBodies consecutive bodies per CTA.
//   Phase A (kLanes threads per body): a_new = the sum of the body's force
//   partials in a fixed order.  Lane l takes rows l, l + kLanes, ... (TwoSum:
//   FP64 pairs for the FP64 path, float pairs for the mixed path), its loads
//   issued kUnroll rows at a time; for kLanes > 1 a fixed-shape shuffle tree
//   then combines the lanes, so the summation order never changes.
//   Phase B (one body per thread): for kModeStep,
//     Eq. 4  v_{i+1} = v_i + dt/2 (a_i + a_{i+1}),
//     the caller's position receives r_{i+1} (the staged positions),
//     Eq. 3  r_{i+2} = r_{i+1} + v_{i+1} dt + dt^2/2 a_{i+1} -> next stage.
// GB300 runs FP64 at 1/64 of the FP32 rate and charges a warp instruction
// for all 32 lanes whatever the active mask, so FP64 work runs one body per
// lane: the mixed path sums its float-pair rows 8 lanes per body (short
// latency) and hands the sums to warp 0 for phase B; the FP64 path, whose
// row sums are FP64 themselves, sums one body per lane.
// ---------------------------------------------------------------------------
template <int PREC>
struct VerletShape {
  // FP64: one lane per body and 64 bodies per CTA, so the FP64 work spreads
  // over ~N/64 CTAs (every SM at N = 10k); mixed: 8 lanes per body, 32 bodies.
  static constexpr int kBlock = PREC == 0 ? 64 : 256;
  static constexpr int kLanes = PREC == 0 ? 1 : 8;   // threads per body in phase A
  static constexpr int kUnroll = PREC == 0 ? 8 : 4;  // rows per lane whose loads go out together
  static constexpr int kBodies = kBlock / kLanes;
};

// (hi, lo) pair sums: FP64 pairs for the FP64 path, float pairs for mixed.
template <typename T>
__device__ __forceinline__ void pair_add(T &hi, T &lo, T vhi, T vlo) {
  two_sum_acc(hi, lo, vhi);
  lo += vlo;
}

// Phase A of the per-body kernels: body p's force partials (rows 0..rows-1)
// summed in a fixed order by L = VerletShape<PREC>::kLanes threads; the sum,
// an unevaluated (hi, lo) pair per component, ends in lane 0.  FP64 adds
// each group of U rows plainly before it enters the pair (see below); the
// mixed path feeds every row through the pair.
template <int PREC, typename T>
__device__ __forceinline__ void sum_partial_rows(const double *partial, int rows, size_t N, int p, int lane, T &sx,
                                                 T &ex, T &sy, T &ey, T &sz, T &ez) {
  typedef typename std::conditional<PREC == 0, double, float2>::type E;  // one partial-row entry
  constexpr int L = VerletShape<PREC>::kLanes, U = VerletShape<PREC>::kUnroll;
  sx = sy = sz = ex = ey = ez = 0;
  const E *part = reinterpret_cast<const E *>(partial);  // row c of body p: part[c*3N + k*N + p]
  auto add = [&](T &s, T &e, const E &v) {
    if constexpr (PREC == 0) {
      two_sum_acc(s, e, v);
    } else {
      pair_add<T>(s, e, v.x, v.y);
    }
  };
  for (int c0 = lane; c0 < rows; c0 += U * L) {
    E vx_[U], vy_[U], vz_[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {  // all loads first, then the sums in row order
      const int c = c0 + u * L;
      if (c < rows) {
        const E *row = part + static_cast<size_t>(c) * 3 * N;
        vx_[u] = __ldg(row + p);
        vy_[u] = __ldg(row + N + p);
        vz_[u] = __ldg(row + 2 * N + p);
      }
    }
    if constexpr (PREC == 0) {
      // FP64: the (up to) U loaded rows added plainly in row order, then the
      // group sum into the (hi, lo) pair: one TwoSum per U rows (the
      // pair-once kernel leaves a row per 64-body block, ~160 per body at
      // N = 10,425; each row is a sum of at most 128 terms).
      E gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (c0 + u * L < rows) {
          gx += vx_[u];
          gy += vy_[u];
          gz += vz_[u];
        }
      }
      add(sx, ex, gx);
      add(sy, ey, gy);
      add(sz, ez, gz);
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (c0 + u * L < rows) {
          add(sx, ex, vx_[u]);
          add(sy, ey, vy_[u]);
          add(sz, ez, vz_[u]);
        }
      }
    }
  }
  if constexpr (L > 1) {
#pragma unroll
    for (int off = 1; off < L; off <<= 1) {
      const T hx = __shfl_down_sync(0xffffffffu, sx, off), lx = __shfl_down_sync(0xffffffffu, ex, off);
      const T hy = __shfl_down_sync(0xffffffffu, sy, off), ly = __shfl_down_sync(0xffffffffu, ey, off);
      const T hz = __shfl_down_sync(0xffffffffu, sz, off), lz = __shfl_down_sync(0xffffffffu, ez, off);
      if ((lane & (2 * off - 1)) == 0) {
        pair_add<T>(sx, ex, hx, lx);
        pair_add<T>(sy, ey, hy, ly);
        pair_add<T>(sz, ez, hz, lz);
      }
    }
  }
}

// One component of the per-body update after a force evaluation `an` at the
// staged position r (from velocity v, previous acceleration ao):
//   Verlet (Eqs. 4, 3): v' = v + dt/2 (ao + an); the state position is r;
//     the next staged position is r + v' dt + dt^2/2 an.
//   Leapfrog, drift-kick-drift (r is the half-step position r_{n+1/2}):
//     v' = v + dt an; the state position is r + dt/2 v'; the next staged
//     position is that plus dt/2 v' (the next half step).
// Returns the state position; v becomes v', *next the next staged position.
__device__ __forceinline__ double step_component(bool leap, double r, double &v, double ao, double an, double dt,
                                                 double half_dt, double half_dt2, double *next) {
  if (leap) {
    v = fma(dt, an, v);
    const double x = fma(half_dt, v, r);
    *next = fma(half_dt, v, x);
    return x;
  }
  v = kick(v, ao, an, half_dt);
  *next = drift(r, v, an, dt, half_dt2);
  return r;
}

// Stage position (rx, ry, rz) of body q for the next force launch, with mu
// copied from the current stage: FP64 double4 at q, or the mixed hi/lo pair
// block at qidx[q] (mixed: *o is the pair offset, *muf the staged mu).
template <int PREC>
__device__ __forceinline__ void stage_position(void *nxt, int q, size_t o, double rx, double ry, double rz, double mu,
                                               float muf) {
  if (PREC == 0) {
    static_cast<double4_32a *>(nxt)[q] = make_double4_32a(rx, ry, rz, mu);
  } else {
    float *w = static_cast<float *>(nxt) + o;
    const float hx = hi_part(rx), hy = hi_part(ry), hz = hi_part(rz);
    w[kXh] = hx;
    w[kYh] = hy;
    w[kZh] = hz;
    w[kMu] = muf;
    w[kXl] = lo_part(rx, hx);
    w[kYl] = lo_part(ry, hy);
    w[kZl] = lo_part(rz, hz);
  }
}

template <int PREC, int MODE>  // MODE: kModeForce, kModeStep or kModeLeapfrog (a.mode)
__global__ void __launch_bounds__(VerletShape<PREC>::kBlock) verlet_kernel(const VerletArgs a) {
  // When at most one force CTA fits on an SM, the next force grid can only
  // land one CTA per SM, however early it launches: let it launch now, so its
  // launch overlaps this kernel (its own griddepcontrol.wait still waits for
  // our completion).  Otherwise release only at the end (below).
  if (a.release_early) grid_dependency_launch();
  typedef typename std::conditional<PREC == 0, double, float>::type T;
  constexpr int L = VerletShape<PREC>::kLanes, NB = VerletShape<PREC>::kBodies;
  // Phase B: FP64 path one thread per body (all three components); mixed
  // path warp c < 3 takes component c of the CTA's 32 bodies, lane = body,
  // so each warp issues a third of the FP64 instructions (GB300's FP64 pipe
  // spends 64 cycles on every warp instruction, so this is the latency).
  constexpr bool kSplit = PREC == 1;
  __shared__ T s_hi[3][NB], s_lo[3][NB];
  const int p0 = a.p_begin + blockIdx.x * NB;  // bodies [p_begin, p_end) (a row shard, or all)
  const int b = threadIdx.x / L, lane = threadIdx.x % L;
  const int p = p0 + b;  // phase A body
  const bool live = p < a.p_end;
  const size_t N = static_cast<size_t>(a.N);
  const int warp = threadIdx.x >> 5;
  const int k = kSplit ? (threadIdx.x & 31) : threadIdx.x;  // phase B body within the CTA
  const int q = p0 + k;
  const int comp = kSplit ? warp : 0;
  const bool own = (kSplit ? warp < 3 : threadIdx.x < NB) && q < a.p_end;
  constexpr bool step = MODE != kModeForce;
  constexpr bool leap = MODE == kModeLeapfrog;
  // This thread's component arrays (mixed split; the FP64 path uses all three).
  auto pick = [&](double *x, double *y, double *z) { return comp == 0 ? x : comp == 1 ? y : z; };
  double *const Xc = pick(a.x, a.y, a.z), *const Vc = pick(a.vx, a.vy, a.vz), *const Ac = pick(a.ax, a.ay, a.az);
  double *const Rc = pick(a.Rx, a.Ry, a.Rz);

  // Before the wait: everything this step's force kernel does not write (it
  // writes only the partial rows), so these loads overlap its tail.
  const int rows = live ? a.nsl[p] : 0;
  double v[3] = {0, 0, 0}, ao[3] = {0, 0, 0}, r[3] = {0, 0, 0}, mu = 0.0;
  float muf = 0.f;
  size_t o = 0;
  if (own && step) {
    if (kSplit) {
      v[0] = Vc[q];
      ao[0] = Ac[q];
      r[0] = Rc[q];
      o = pair_off(a.qidx[q]);
      if (comp == 0) muf = static_cast<const float *>(a.cur)[o + kMu];
    } else {
      v[0] = a.vx[q];
      v[1] = a.vy[q];
      v[2] = a.vz[q];
      ao[0] = a.ax[q];
      ao[1] = a.ay[q];
      ao[2] = a.az[q];
      const double4_32a rr = static_cast<const double4_32a *>(a.cur)[q];
      r[0] = rr.x;
      r[1] = rr.y;
      r[2] = rr.z;
      mu = rr.w;
    }
  }
  grid_dependency_wait();  // the force partials of this step are complete

  // ---- phase A: the partial rows of body p --------------------------------
  T sx, sy, sz, ex, ey, ez;
  sum_partial_rows<PREC, T>(a.partial, rows, N, p, lane, sx, ex, sy, ey, sz, ez);
  if (lane == 0) {
    s_hi[0][b] = sx;
    s_lo[0][b] = ex;
    s_hi[1][b] = sy;
    s_lo[1][b] = ey;
    s_hi[2][b] = sz;
    s_lo[2][b] = ez;
  }
  __syncthreads();
  if (!own) {
    if (!a.release_early) grid_dependency_launch();
    return;
  }

  // ---- phase B: Eqs. 4 and 3 ---------------------------------------------------
  if (kSplit) {  // component `comp` of body q
    const double an = static_cast<double>(s_hi[comp][k]) + static_cast<double>(s_lo[comp][k]);
    if (!isfinite(an)) atomicOr(a.flags, kFlagNonFinite);
    if (step) {
      double vn = v[0], nr;
      const double x = step_component(leap, r[0], vn, ao[0], an, a.dt, a.half_dt, a.half_dt2, &nr);
      Rc[q] = nr;
      float *w = static_cast<float *>(a.nxt) + o;
      const float h = hi_part(nr);
      w[kXh + 2 * comp] = h;
      w[kXl + 2 * comp] = lo_part(nr, h);
      if (comp == 0) w[kMu] = muf;
      Xc[q] = x;
      Vc[q] = vn;
    }
    Ac[q] = an;
  } else {  // body q, all three components
    double an[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) an[c] = static_cast<double>(s_hi[c][k]) + static_cast<double>(s_lo[c][k]);
    if (!finite3(an[0], an[1], an[2])) atomicOr(a.flags, kFlagNonFinite);
    if (step) {
      double nr[3], x[3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        x[c] = step_component(leap, r[c], v[c], ao[c], an[c], a.dt, a.half_dt, a.half_dt2, &nr[c]);
      stage_position<PREC>(a.nxt, q, o, nr[0], nr[1], nr[2], mu, muf);
      a.x[q] = x[0];
      a.y[q] = x[1];
      a.z[q] = x[2];
      a.vx[q] = v[0];
      a.vy[q] = v[1];
      a.vz[q] = v[2];
    }
    a.ax[q] = an[0];
    a.ay[q] = an[1];
    a.az[q] = an[2];
  }
  // Otherwise only now may the next force launch be placed: its CTAs then
  // land on an idle GPU, one share per slot, as the equal-share decomposition
  // assumes (an early launch let several CTAs pile onto the SMs that freed
  // first).
  if (!a.release_early) grid_dependency_launch();
}

cudaError_t launch_verlet(int precision, const VerletArgs &a, cudaStream_t s, bool chained) {
  if (a.p_end <= a.p_begin) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  const int64_t nb = precision == 0 ? VerletShape<0>::kBodies : VerletShape<1>::kBodies;
  cfg.gridDim = dim3(static_cast<unsigned>((static_cast<int64_t>(a.p_end - a.p_begin) + nb - 1) / nb));
  cfg.blockDim = dim3(precision == 0 ? VerletShape<0>::kBlock : VerletShape<1>::kBlock);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
#define NB_VERLET(P, M) \
  if (precision == P && a.mode == M) return cudaLaunchKernelEx(&cfg, verlet_kernel<P, M>, a);
  NB_VERLET(0, kModeForce)
  NB_VERLET(0, kModeStep)
  NB_VERLET(0, kModeLeapfrog)
  NB_VERLET(1, kModeForce)
  NB_VERLET(1, kModeStep)
  NB_VERLET(1, kModeLeapfrog)
#undef NB_VERLET
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Classical RK4 (the higher-order method Section 2 names) on y = (r, v),
// y' = (v, A(r)): stage completion, s = 2..5 (stage 1 is rk_prep or the end
// of s = 5).  Phase A as in the Verlet kernel; phase B, one body per thread:
//   s = 2, 3: AR += 2 v_s, AV += 2 a_s; r_{s+1} = r + c v_s, v_{s+1} = v + c a_s
//             (c = dt/2 at s = 2, dt at s = 3);
//   s = 4:    r <- r + dt/6 (AR + v_4), v <- v + dt/6 (AV + a_4), stage r;
//   s = 5:    a <- a_5 = A(r); then stage 1 of the next step:
//             AR = v, AV = a, v_2 = v + dt/2 a, stage r_2 = r + dt/2 v.
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(VerletShape<PREC>::kBlock) rk_stage_kernel(const RkArgs a) {
  if (a.release_early) grid_dependency_launch();
  typedef typename std::conditional<PREC == 0, double, float>::type T;
  constexpr int L = VerletShape<PREC>::kLanes, NB = VerletShape<PREC>::kBodies;
  constexpr bool kSplit = PREC == 1;  // mixed: warp c < 3 takes component c (as the Verlet kernel)
  __shared__ T s_hi[3][NB], s_lo[3][NB];
  const int p0 = blockIdx.x * NB;
  const int b = threadIdx.x / L, lane = threadIdx.x % L;
  const int p = p0 + b;
  const bool live = p < a.N;
  const size_t N = static_cast<size_t>(a.N);
  const int warp = threadIdx.x >> 5;
  const int k0 = kSplit ? (threadIdx.x & 31) : threadIdx.x;
  const int q = p0 + k0;
  const int comp = kSplit ? warp : 0;
  const bool own = (kSplit ? warp < 3 : threadIdx.x < NB) && q < a.N;
  const int rows = live ? a.nsl[p] : 0;
  auto sel = [](int c, double *x, double *y, double *z) { return c == 0 ? x : c == 1 ? y : z; };
  // Prefetch what the force launch does not write (the state, the RK sums):
  // component comp (mixed) or all three (FP64).
  constexpr int NC = kSplit ? 1 : 3;
  double rn[NC], vn[NC], vs[NC], ar[NC], av[NC], mu = 0.0;
  float muf = 0.f;
  size_t o = 0;
#pragma unroll
  for (int j = 0; j < NC; ++j) rn[j] = vn[j] = vs[j] = ar[j] = av[j] = 0.0;
  if (own) {
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const int c = kSplit ? comp : j;
      rn[j] = sel(c, a.x, a.y, a.z)[q];
      vn[j] = sel(c, a.vx, a.vy, a.vz)[q];
      if (a.stage <= 4) {
        vs[j] = a.V[c * N + q];
        ar[j] = a.AR[c * N + q];
        av[j] = a.AV[c * N + q];
      }
    }
    if (PREC == 0) {
      mu = static_cast<const double4_32a *>(a.cur)[q].w;
    } else {
      o = pair_off(a.qidx[q]);
      if (comp == 0) muf = static_cast<const float *>(a.cur)[o + kMu];
    }
  }
  grid_dependency_wait();  // the force partials of this stage are complete
  T sx, sy, sz, ex, ey, ez;
  sum_partial_rows<PREC, T>(a.partial, rows, N, p, lane, sx, ex, sy, ey, sz, ez);
  if (lane == 0) {
    s_hi[0][b] = sx;
    s_lo[0][b] = ex;
    s_hi[1][b] = sy;
    s_lo[1][b] = ey;
    s_hi[2][b] = sz;
    s_lo[2][b] = ez;
  }
  __syncthreads();
  if (!own) {
    if (!a.release_early) grid_dependency_launch();
    return;
  }
  bool finite = true;
  double rnext[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const int c = kSplit ? comp : j;
    const size_t i = c * N + q;
    const double as = static_cast<double>(s_hi[c][k0]) + static_cast<double>(s_lo[c][k0]);
    finite = finite && isfinite(as);
    if (a.stage == 2 || a.stage == 3) {
      const double cc = a.stage == 2 ? 0.5 * a.dt : a.dt;
      a.AR[i] = ar[j] + 2.0 * vs[j];
      a.AV[i] = av[j] + 2.0 * as;
      rnext[j] = rn[j] + cc * vs[j];
      a.V[i] = vn[j] + cc * as;
    } else if (a.stage == 4) {
      const double h = a.dt / 6.0;
      rnext[j] = rn[j] + h * (ar[j] + vs[j]);
      sel(c, a.x, a.y, a.z)[q] = rnext[j];
      sel(c, a.vx, a.vy, a.vz)[q] = vn[j] + h * (av[j] + as);
    } else {  // s = 5: A at the new state, then stage 1 of the next step
      sel(c, a.ax, a.ay, a.az)[q] = as;
      const double cc = 0.5 * a.dt;
      a.AR[i] = vn[j];
      a.AV[i] = as;
      rnext[j] = rn[j] + cc * vn[j];
      a.V[i] = vn[j] + cc * as;
    }
  }
  if (!finite) atomicOr(a.flags, kFlagNonFinite);
  if (kSplit) {
    float *w = static_cast<float *>(a.nxt) + o;
    const float h = hi_part(rnext[0]);
    w[kXh + 2 * comp] = h;
    w[kXl + 2 * comp] = lo_part(rnext[0], h);
    if (comp == 0) w[kMu] = muf;
  } else {
    stage_position<PREC>(a.nxt, q, o, rnext[0], rnext[NC > 1 ? 1 : 0], rnext[NC > 2 ? 2 : 0], mu, muf);
  }
  if (!a.release_early) grid_dependency_launch();
}

cudaError_t launch_rk_stage(int precision, const RkArgs &a, cudaStream_t s, bool chained) {
  if (a.N <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  const int64_t nb = precision == 0 ? VerletShape<0>::kBodies : VerletShape<1>::kBodies;
  cfg.gridDim = dim3(static_cast<unsigned>((static_cast<int64_t>(a.N) + nb - 1) / nb));
  cfg.blockDim = dim3(precision == 0 ? VerletShape<0>::kBlock : VerletShape<1>::kBlock);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  return precision == 0 ? cudaLaunchKernelEx(&cfg, rk_stage_kernel<0>, a)
                        : cudaLaunchKernelEx(&cfg, rk_stage_kernel<1>, a);
}

// RK4 stage 1 from the state (r, v, a = A(r)): AR = v, AV = a,
// V = v + dt/2 a, and the staged sources r_2 = r + dt/2 v with mu = G m.
template <int PREC>
__global__ void rk_prep_kernel(const RkArgs a) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.N) return;
  const size_t N = static_cast<size_t>(a.N);
  const double rn[3] = {a.x[q], a.y[q], a.z[q]}, vn[3] = {a.vx[q], a.vy[q], a.vz[q]};
  const double an[3] = {a.ax[q], a.ay[q], a.az[q]};
  const double c = 0.5 * a.dt;
  double r2[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    a.AR[k * N + q] = vn[k];
    a.AV[k * N + q] = an[k];
    r2[k] = rn[k] + c * vn[k];
    a.V[k * N + q] = vn[k] + c * an[k];
  }
  const double mu = a.G * a.m[q];
  const size_t o = PREC == 0 ? 0 : pair_off(a.qidx[q]);
  stage_position<PREC>(a.nxt, q, o, r2[0], r2[1], r2[2], mu, static_cast<float>(mu));
}

cudaError_t launch_rk_prep(int precision, const RkArgs &a, cudaStream_t s) {
  if (a.N <= 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>((static_cast<int64_t>(a.N) + 255) / 256);
  if (precision == 0)
    rk_prep_kernel<0><<<grid, 256, 0, s>>>(a);
  else
    rk_prep_kernel<1><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Stage the sources of the next force launch: r (drift == 0) or the Eq. 3
// drift of (r, v, a) (drift == 1), with mu = G m.
//   FP64: double4 (x, y, z, mu) at index p.
//   Mixed: FP64 positions R[p], and hi = fl32(r), lo = fl32(r - hi), mu into
//   the pair block of stage entry q = qidx[p] (layout in step_kernel.cuh).
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void prep_kernel(const PrepArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.N) return;
  double rx = a.x[p], ry = a.y[p], rz = a.z[p];
  const double m = a.m[p];
  if (a.check) {
    const bool ok = finite3(rx, ry, rz) && finite3(a.vx[p], a.vy[p], a.vz[p]) && isfinite(m) && m >= 0.0;
    if (!ok) atomicOr(a.flags, kFlagBadInput);
  }
  if (a.drift == 1) {  // Eq. 3
    rx = drift(rx, a.vx[p], a.ax[p], a.dt, a.half_dt2);
    ry = drift(ry, a.vy[p], a.ay[p], a.dt, a.half_dt2);
    rz = drift(rz, a.vz[p], a.az[p], a.dt, a.half_dt2);
  } else if (a.drift == 2) {  // leapfrog: the first half-step drift
    const double h = 0.5 * a.dt;
    rx = fma(h, a.vx[p], rx);
    ry = fma(h, a.vy[p], ry);
    rz = fma(h, a.vz[p], rz);
  }
  const double mu = a.G * m;
  if (PREC == 0) {
    static_cast<double4_32a *>(a.stage)[p] = make_double4_32a(rx, ry, rz, mu);
  } else {
    a.Rx[p] = rx;
    a.Ry[p] = ry;
    a.Rz[p] = rz;
    const int q = a.qidx[p];
    float *w = static_cast<float *>(a.stage) + pair_off(q);
    const float hx = hi_part(rx), hy = hi_part(ry), hz = hi_part(rz);
    w[kXh] = hx;
    w[kYh] = hy;
    w[kZh] = hz;
    w[kMu] = static_cast<float>(mu);
    w[kXl] = lo_part(rx, hx);
    w[kYl] = lo_part(ry, hy);
    w[kZl] = lo_part(rz, hz);
    w[14] = 0.f;
  }
}

cudaError_t launch_prep(int precision, const PrepArgs &a, cudaStream_t s) {
  if (a.N <= 0) return cudaSuccess;
  const int grid = (a.N + 255) / 256;
  if (precision == 0)
    prep_kernel<0><<<grid, 256, 0, s>>>(a);
  else
    prep_kernel<1><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

// Padding sources of the mixed layout: hi = (kPadCoord, kPadCoord,
// kPadCoord), mu = 0, lo = 0.  Against any real target r2 ~ 3e30 stays
// finite in FP32, q = r2^{-1/2} is tiny and mu = 0 makes the term exactly 0.
__global__ void pad_fill_kernel(float *stage, int64_t n_pairs) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_pairs * 16) return;
  const int f = static_cast<int>(i & 15);
  stage[i] = f < 6 ? kPadCoord : 0.f;
}

// Padding sources of the FP64 layout (row shards pad the stage to equal
// chunks): (kPadCoord, kPadCoord, kPadCoord, mu = 0); the term of each is
// exactly 0 against any real target.
__global__ void pad_fill_fp64_kernel(double4_32a *stage, int64_t n) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) stage[i] = make_double4_32a(kPadCoord, kPadCoord, kPadCoord, 0.0);
}

cudaError_t launch_pad_fill_fp64(void *stage, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  pad_fill_fp64_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(static_cast<double4_32a *>(stage), n);
  return cudaGetLastError();
}

cudaError_t launch_pad_fill(void *stage, int64_t n_pairs, cudaStream_t s) {
  if (n_pairs <= 0) return cudaSuccess;
  const int64_t n = n_pairs * 16;
  pad_fill_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(static_cast<float *>(stage), n_pairs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Energy (Sections 2 and 4): per body p,
//   e_kin[p] = (1/2) m_p |v_p|^2,   e_pot[p] = -(1/2) m_p sum_{j != p} G m_j / |r_j - r_p|,
// so that sum_p e_pot[p] = -sum_{p<j} G m_p m_j / |r_j - r_p|.  FP64, one
// CTA per block of kEnergyBlock targets, sources staged through shared memory.
// Each body's potential is compensated as the force is: the terms of one
// source tile are summed plainly, and each tile's sub-sum enters a (hi, lo)
// pair through TwoSum, so the many small asteroid terms of a moon's sum are
// not lost below half an ulp of its host's term.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEnergyBlock) energy_kernel(const EnergyArgs a) {
  __shared__ double4_32a tile[kEnergyBlock];
  const Item it = a.items[blockIdx.x];
  const int p = it.i0 + threadIdx.x;
  const bool valid = p < it.i1;
  const int pp = valid ? p : it.i0;
  const double px = a.x[pp], py = a.y[pp], pz = a.z[pp];
  double phi = 0.0, phi_lo = 0.0;
  for (int j0 = it.j0; j0 < it.j1; j0 += kEnergyBlock) {
    const int j = j0 + threadIdx.x;
    __syncthreads();
    if (j < it.j1) tile[threadIdx.x] = make_double4_32a(a.x[j], a.y[j], a.z[j], a.G * a.m[j]);
    __syncthreads();
    const int cnt = min(kEnergyBlock, it.j1 - j0);
    double t = 0.0;
    for (int u = 0; u < cnt; ++u) {
      const double4_32a s = tile[u];
      const double dx = s.x - px, dy = s.y - py, dz = s.z - pz;
      double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      const bool self = (j0 + u) == pp;
      r2 = self ? 1.0 : r2;
      t += self ? 0.0 : s.w * inv_r1(r2);
    }
    two_sum_acc(phi, phi_lo, t);
  }
  if (valid) {
    const double m = a.m[p];
    const double v2 = fma(a.vz[p], a.vz[p], fma(a.vy[p], a.vy[p], a.vx[p] * a.vx[p]));
    a.e_kin[p] = 0.5 * m * v2;
    a.e_pot[p] = -0.5 * m * (phi + phi_lo);
  }
}

cudaError_t launch_energy(const EnergyArgs &a, cudaStream_t s) {
  if (a.n_items <= 0) return cudaSuccess;
  energy_kernel<<<a.n_items, kEnergyBlock, 0, s>>>(a);
  return cudaGetLastError();
}

// Double-double accumulation: Knuth's TwoSum for the error-free sum of two
// doubles, and Dekker's Fast2Sum to renormalise.
struct DD {
  double hi, lo;
};
__device__ __forceinline__ DD two_sum(double a, double b) {
  const double s = a + b;
  const double bb = s - a;
  const double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ DD dd_add(DD a, DD b) {
  DD s = two_sum(a.hi, b.hi);
  const double e = s.lo + (a.lo + b.lo);
  const double hi = s.hi + e;
  return {hi, e - (hi - s.hi)};
}

// One CTA per system: strided double-double partial sums per thread, then a
// fixed-shape tree in shared memory (deterministic).
__global__ void __launch_bounds__(256) energy_reduce_kernel(const ReduceArgs a) {
  __shared__ DD sk[256], sp[256];
  const int s = blockIdx.x;
  const int64_t b = a.offsets[s], e = a.offsets[s + 1];
  DD k = {0.0, 0.0}, q = {0.0, 0.0};
  for (int64_t i = b + threadIdx.x; i < e; i += 256) {
    k = dd_add(k, DD{a.e_kin[i], 0.0});
    q = dd_add(q, DD{a.e_pot[i], 0.0});
  }
  sk[threadIdx.x] = k;
  sp[threadIdx.x] = q;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sk[threadIdx.x] = dd_add(sk[threadIdx.x], sk[threadIdx.x + w]);
      sp[threadIdx.x] = dd_add(sp[threadIdx.x], sp[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.out[s] = sk[0].hi + sk[0].lo;
    a.out[a.n_systems + s] = sp[0].hi + sp[0].lo;
  }
}

cudaError_t launch_energy_reduce(const ReduceArgs &a, cudaStream_t s) {
  if (a.n_systems <= 0) return cudaSuccess;
  energy_reduce_kernel<<<a.n_systems, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace nb
