// Adjoint of the Verlet trajectory: the vector-Jacobian product (VJP) of
// Eq. 1 and the per-body reverse-sweep update.
//
// With d = r_j - r_q, s3 = |d|^-3, s5 = |d|^-5 and mu = G m, the Jacobian of
// the pair term d |d|^-3 is K(d) = I s3 - 3 d d^T s5 (symmetric, K(-d) = K(d)),
// so for an adjoint vector w on the accelerations
//   (J^T w)_q = sum_{j != q} K(d) (mu_q w_j - mu_j w_q)
//             = sum_j [ s3 u - 3 s5 (d.u) d ],  u = mu_q w_j - mu_j w_q,
//   (dA/dm)^T w at q = -G sum_{j != q} s3 (w_j . d).
// vjp_kernel evaluates both sums for every target q, using the same
// stream-K work tables as the force kernel (segments of sources per target
// block, one partial row per segment, here 4 values: the three components of
// J^T w and the mass sum).  adjoint_kernel then sums a body's rows in a fixed
// order and applies one step of the reverse sweep of Eqs. 3-4:
//   rho += J^T w;  g_m += (dA/dm)^T w;
//   nu' = nu + dt rho;  alpha' = dt/2 nu + dt^2/2 rho;  nu = nu';
//   next w = alpha' + dt/2 nu'  (w = alpha' before the last product, at r_0).
#include "step_kernel.cuh"  // packed f32x2 helpers (f2, pk, upk, add2, mul2, fma2)

namespace nb {

namespace {

// Mixed path: w is staged in pair blocks like the positions, 32 bytes per two
// consecutive stage entries, [wx0 wx1 wy0 wy1 | wz0 wz1 0 0], so one 16-byte
// shared load yields packed (f32x2) operands for a source pair.
__device__ __forceinline__ void w_pair_store(void *w, int q, float wx, float wy, float wz) {
  float *b = static_cast<float *>(w) + 8 * static_cast<size_t>(q >> 1) + (q & 1);
  b[0] = wx;
  b[2] = wy;
  b[4] = wz;
}
__device__ __forceinline__ float3 w_pair_load(const void *w, int q) {
  const float *b = static_cast<const float *>(w) + 8 * static_cast<size_t>(q >> 1) + (q & 1);
  return make_float3(b[0], b[2], b[4]);
}

// The VJP terms of one target against a source pair (mixed path), both terms
// accumulated into packed pairs: with d = r_j - r_q from the hi/lo split,
// s3 = |d|^-3, s5 = |d|^-5, u = mu_q w_j - mu_j w_q,
//   acc_xyz += s3 u - 3 s5 (d.u) d,   acc_m += s3 (w_j . d).
// v0..v3: the pair's position block; w0 = (wx, wy), w1 = (wz, 0) of the pair.
// MASK: a source that is the target itself gets r2 = 1 and |d|^-1 = 0, so
// all of its terms are exactly 0.
template <bool MASK>
__device__ __forceinline__ void vjp_pair(const ulonglong2 &v0, const ulonglong2 &v1, const ulonglong2 &v2,
                                         const ulonglong2 &v3, const ulonglong2 &w0, const ulonglong2 &w1, f2 nxh,
                                         f2 nyh, f2 nzh, f2 nxl, f2 nyl, f2 nzl, f2 muq, f2 nwqx, f2 nwqy, f2 nwqz,
                                         f2 m3, bool self_a, bool self_b, f2 (&acc)[4]) {
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
  float ya = rsqrt_approx(ra), yb = rsqrt_approx(rb);
  if (MASK) {
    ya = self_a ? 0.0f : ya;
    yb = self_b ? 0.0f : yb;
  }
  const f2 y = pk(ya, yb);
  const f2 y2 = mul2(y, y);
  const f2 s3 = mul2(y, y2);
  const f2 s5 = mul2(s3, y2);
  const f2 mu = v1.y;  // (mu_j0, mu_j1)
  const f2 ux = fma2(mu, nwqx, mul2(muq, w0.x));
  const f2 uy = fma2(mu, nwqy, mul2(muq, w0.y));
  const f2 uz = fma2(mu, nwqz, mul2(muq, w1.x));
  f2 du = mul2(dx, ux);
  du = fma2(dy, uy, du);
  du = fma2(dz, uz, du);
  const f2 t3 = mul2(mul2(s5, du), m3);  // -3 s5 (d.u)
  acc[0] = fma2(t3, dx, fma2(s3, ux, acc[0]));
  acc[1] = fma2(t3, dy, fma2(s3, uy, acc[1]));
  acc[2] = fma2(t3, dz, fma2(s3, uz, acc[2]));
  f2 dw = mul2(w0.x, dx);
  dw = fma2(w0.y, dy, dw);
  dw = fma2(w1.x, dz, dw);
  acc[3] = fma2(s3, dw, acc[3]);
}

// Source tile: positions as staged by the forward pass (FP64 double4 or
// mixed pair blocks, 32 B per source) followed by w (FP64 double4; mixed pair
// blocks of 16 B per source).
template <int PREC>
struct VjpLayout {
  static constexpr int kWBytes = PREC == 0 ? 32 : 16;
  static constexpr int kBytesPerSource = 32 + kWBytes;
};

template <int PREC, int THREADS>
__global__ void __launch_bounds__(THREADS) vjp_kernel(const VjpArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[kStages];
  __shared__ int s_flag;
  const int tid = threadIdx.x;
  const int tj = a.tj;
  constexpr int kW = VjpLayout<PREC>::kWBytes;
  auto pos_ptr = [&](int s) { return smem + static_cast<size_t>(s) * tj * VjpLayout<PREC>::kBytesPerSource; };
  auto w_ptr = [&](int s) { return pos_ptr(s) + static_cast<size_t>(tj) * 32; };

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    mbar_init_fence();
    s_flag = 0;
  }
  __syncthreads();
  uint32_t phase = 0;
  bool aborted = false;
  bool stall = a.stall != 0 && blockIdx.x == 0;
  const size_t N = static_cast<size_t>(a.N);
  const int seg_end = a.seg_off[blockIdx.x + 1];

  for (int si = a.seg_off[blockIdx.x]; si < seg_end && !aborted; ++si) {
    const Seg sg = a.segs[si];
    const Blk bk = a.blks[sg.blk];
    const int q_end = bk.q0 + (bk.i1 - bk.i0);
    // target: stage entry tq (consecutive within the block), body p (the
    // same index, or perm[tq] in a spatially ordered stage)
    const bool valid = tid < bk.i1 - bk.i0;
    const int tq = bk.q0 + (valid ? tid : bk.i1 - bk.i0 - 1);
    const int p = a.perm ? a.perm[tq] : bk.i0 + (tq - bk.q0);
    // Mixed path: the stage pairs that may hold one of this warp's targets.
    const int mlo = static_cast<int>(__reduce_min_sync(0xffffffffu, static_cast<unsigned>(tq))) >> 1;
    const int mhi = static_cast<int>(__reduce_max_sync(0xffffffffu, static_cast<unsigned>(tq))) >> 1;

    // target q: position, mu_q, w_q
    double qx = 0, qy = 0, qz = 0, qmu = 0, wqx = 0, wqy = 0, wqz = 0;
    float hx = 0, hy = 0, hz = 0, lx = 0, ly = 0, lz = 0, fmu = 0, fwx = 0, fwy = 0, fwz = 0;
    if (PREC == 0) {
      const double4_32a r = static_cast<const double4_32a *>(a.pos)[tq];
      qx = r.x;
      qy = r.y;
      qz = r.z;
      qmu = r.w;
      const double4_32a w = static_cast<const double4_32a *>(a.w)[tq];
      wqx = w.x;
      wqy = w.y;
      wqz = w.z;
    } else {
      const float *e = static_cast<const float *>(a.pos) + pair_off(tq);
      hx = e[kXh];
      hy = e[kYh];
      hz = e[kZh];
      lx = e[kXl];
      ly = e[kYl];
      lz = e[kZl];
      fmu = e[kMu];
      const float3 w = w_pair_load(a.w, tq);
      fwx = w.x;
      fwy = w.y;
      fwz = w.z;
    }
    // FP64: per-tile sub-sums folded into (acc, cmp) pairs by TwoSum.
    // Mixed: FP32 sub-sums of kFoldPairs*2 sources folded into float pairs.
    double acc[4] = {0, 0, 0, 0}, cmp[4] = {0, 0, 0, 0};
    float sh[4] = {0, 0, 0, 0}, sl[4] = {0, 0, 0, 0};

    const int ntiles = (sg.s1 - sg.s0 + tj - 1) / tj;
    auto issue = [&](int t) {
      const int s = t % kStages;
      const int j = sg.s0 + t * tj;
      const uint32_t n = static_cast<uint32_t>(min(tj, sg.s1 - j));
      mbar_arrive_expect_tx(&bar[s], n * (32u + kW));
      bulk_g2s(pos_ptr(s), static_cast<const unsigned char *>(a.pos) + static_cast<size_t>(j) * 32, n * 32u, &bar[s]);
      bulk_g2s(w_ptr(s), static_cast<const unsigned char *>(a.w) + static_cast<size_t>(j) * kW, n * kW, &bar[s]);
    };
    if (tid == 0)
      for (int t = 0; t < kStages && t < ntiles; ++t)
        if (!(stall && t == 0)) issue(t);  // (the test hook leaves tile 0 of CTA 0 unissued)
    stall = false;

    for (int t = 0; t < ntiles; ++t) {
      const int s = t % kStages;
      if (!mbar_wait(&bar[s], (phase >> s) & 1u)) atomicOr(&s_flag, 1);
      phase ^= 1u << s;
      const int jt0 = sg.s0 + t * tj;
      const int cnt = min(tj, sg.s1 - jt0);
      const bool diag = jt0 < q_end && jt0 + cnt > bk.q0;
      if (PREC == 0) {
        const double4_32a *sp = reinterpret_cast<const double4_32a *>(pos_ptr(s));
        const double4_32a *sw = reinterpret_cast<const double4_32a *>(w_ptr(s));
        double tacc[4] = {0, 0, 0, 0};
        for (int jj = 0; jj < cnt; ++jj) {
          const double4_32a r = sp[jj], w = sw[jj];
          const double dx = r.x - qx, dy = r.y - qy, dz = r.z - qz;
          double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
          // The target itself: r2 = 1 and |d|^-1 = 0, so all its terms are 0
          // (u = mu_q w_q - mu_q w_q need not round to exactly 0).
          const bool self = diag && jt0 + jj == tq;
          r2 = self ? 1.0 : r2;
          const double y = self ? 0.0 : inv_r1(r2);
          const double y2 = y * y;
          const double s3 = y * y2;
          const double s5 = s3 * y2;
          const double ux = fma(-r.w, wqx, qmu * w.x);
          const double uy = fma(-r.w, wqy, qmu * w.y);
          const double uz = fma(-r.w, wqz, qmu * w.z);
          const double t3 = 3.0 * s5 * fma(dz, uz, fma(dy, uy, dx * ux));
          tacc[0] = fma(-t3, dx, fma(s3, ux, tacc[0]));
          tacc[1] = fma(-t3, dy, fma(s3, uy, tacc[1]));
          tacc[2] = fma(-t3, dz, fma(s3, uz, tacc[2]));
          tacc[3] = fma(s3, fma(w.z, dz, fma(w.y, dy, w.x * dx)), tacc[3]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) two_sum_acc(acc[c], cmp[c], tacc[c]);
      } else {
        const ulonglong2 *sp = reinterpret_cast<const ulonglong2 *>(pos_ptr(s));  // 4 per pair block
        const ulonglong2 *sw = reinterpret_cast<const ulonglong2 *>(w_ptr(s));    // 2 per pair block
        const f2 nxh = pk(-hx, -hx), nyh = pk(-hy, -hy), nzh = pk(-hz, -hz);
        const f2 nxl = pk(-lx, -lx), nyl = pk(-ly, -ly), nzl = pk(-lz, -lz);
        const f2 muq = pk(fmu, fmu), nwqx = pk(-fwx, -fwx), nwqy = pk(-fwy, -fwy), nwqz = pk(-fwz, -fwz);
        const f2 m3 = pk(-3.0f, -3.0f);
        const int npairs = cnt >> 1;
        const int P0t = jt0 >> 1;  // stage pair index of the tile's first pair
        for (int g0 = 0; g0 < npairs; g0 += kFoldPairs) {
          const int lim = min(kFoldPairs, npairs - g0);
          f2 pacc[4] = {0ull, 0ull, 0ull, 0ull};
          // Only pairs that may hold one of this warp's own targets take the
          // self test (a warp's 32 consecutive targets span <= 17 pairs).
          const int r0 = max(mlo - P0t - g0, 0), r1 = min(mhi - P0t - g0 + 1, lim);
          auto run = [&](int b0, int b1, bool masked) {
            if (!masked) {
#pragma unroll 2
              for (int b = b0; b < b1; ++b) {
                const ulonglong2 *pb = sp + 4 * (g0 + b), *wb = sw + 2 * (g0 + b);
                vjp_pair<false>(pb[0], pb[1], pb[2], pb[3], wb[0], wb[1], nxh, nyh, nzh, nxl, nyl, nzl, muq, nwqx,
                                nwqy, nwqz, m3, false, false, pacc);
              }
            } else {
              for (int b = b0; b < b1; ++b) {
                const ulonglong2 *pb = sp + 4 * (g0 + b), *wb = sw + 2 * (g0 + b);
                const int P = P0t + g0 + b;
                vjp_pair<true>(pb[0], pb[1], pb[2], pb[3], wb[0], wb[1], nxh, nyh, nzh, nxl, nyl, nzl, muq, nwqx,
                               nwqy, nwqz, m3, 2 * P == tq, 2 * P + 1 == tq, pacc);
              }
            }
          };
          if (r0 < r1) {
            run(0, r0, false);
            run(r0, r1, true);
            run(r1, lim, false);
          } else {
            run(0, lim, false);
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {  // fold the packed sub-sums into the float pairs
            float e, o;
            upk(pacc[c], e, o);
            two_sum_acc(sh[c], sl[c], e + o);
          }
        }
      }
      __syncthreads();
      if (s_flag & 1) {
        aborted = true;
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
    if (valid) {
      double *prow = a.partial + static_cast<size_t>(sg.slot) * 4 * N;
      if (PREC == 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c) prow[c * N + p] = acc[c] + cmp[c];
      } else {
        float2 *frow = reinterpret_cast<float2 *>(prow);
#pragma unroll
        for (int c = 0; c < 4; ++c) frow[c * N + p] = make_float2(sh[c], sl[c]);
      }
    }
  }
}

// One reverse-sweep step per body (see the file comment).  mode 0: full
// update and stage w = alpha' + dt/2 nu'; mode 1: the same but stage
// w = alpha' (the next product is the last one, at r_0); mode 2: the last
// product only (rho, g_m updated, nothing staged).
template <int PREC>
__global__ void __launch_bounds__(256) adjoint_kernel(const AdjArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.N) return;
  const size_t N = static_cast<size_t>(a.N);
  const int rows = a.nsl[p];
  double s[4], e[4];
  if (PREC == 0) {
    // rows in groups of 8, added plainly in row order, each group sum then
    // through TwoSum (the pair-once VJP leaves a row per 64-body block)
#pragma unroll
    for (int c = 0; c < 4; ++c) s[c] = e[c] = 0.0;
    for (int r0 = 0; r0 < rows; r0 += 8) {
      double g[4] = {0.0, 0.0, 0.0, 0.0};
      for (int r = r0; r < min(rows, r0 + 8); ++r) {
        const double *row = a.partial + static_cast<size_t>(r) * 4 * N;
#pragma unroll
        for (int c = 0; c < 4; ++c) g[c] += row[c * N + p];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) two_sum_acc(s[c], e[c], g[c]);
    }
  } else {
    float fs[4] = {0.f, 0.f, 0.f, 0.f}, fe[4] = {0.f, 0.f, 0.f, 0.f};
    for (int r = 0; r < rows; ++r) {
      const float2 *row = reinterpret_cast<const float2 *>(a.partial + static_cast<size_t>(r) * 4 * N);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float2 v = row[c * N + p];
        two_sum_acc(fs[c], fe[c], v.x);
        fe[c] += v.y;
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      s[c] = static_cast<double>(fs[c]);
      e[c] = static_cast<double>(fe[c]);
    }
  }
  double jtw[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) jtw[c] = s[c] + e[c];
  const double gsum = s[3] + e[3];
  if (!finite3(jtw[0], jtw[1], jtw[2]) || !isfinite(gsum)) atomicOr(a.flags, kFlagNonFinite);
  a.gm[p] += -a.G * gsum;
  double rho[3], nu[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    rho[c] = a.rho[c * N + p] + jtw[c];
    a.rho[c * N + p] = rho[c];
    nu[c] = a.nu[c * N + p];
  }
  if (a.mode == 2) return;
  double w[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double nun = fma(a.dt, rho[c], nu[c]);               // nu' = nu + dt rho
    const double al = fma(a.half_dt2, rho[c], a.half_dt * nu[c]);  // alpha' = dt/2 nu + dt^2/2 rho
    a.nu[c * N + p] = nun;
    w[c] = a.mode == 0 ? fma(a.half_dt, nun, al) : al;         // next w
  }
  const int q = a.qidx ? a.qidx[p] : p;
  if (PREC == 0)
    static_cast<double4_32a *>(a.w)[q] = make_double4_32a(w[0], w[1], w[2], 0.0);
  else
    w_pair_store(a.w, q, static_cast<float>(w[0]), static_cast<float>(w[1]), static_cast<float>(w[2]));
}

// rho = dL/dr_T, nu = dL/dv_T (or 0), g_m = 0, and the first w = dt/2 nu
// (mode 0) or 0 (mode 1: no step, the only product is at r_0 with w = 0).
template <int PREC>
__global__ void adjoint_init_kernel(const AdjArgs a, const double *dr, const double *dv) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.N) return;
  const size_t N = static_cast<size_t>(a.N);
  double w[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    a.rho[c * N + p] = dr[c * N + p];
    const double nu = dv ? dv[c * N + p] : 0.0;
    a.nu[c * N + p] = nu;
    w[c] = a.mode == 0 ? a.half_dt * nu : 0.0;
  }
  a.gm[p] = 0.0;
  const int q = a.qidx ? a.qidx[p] : p;
  if (PREC == 0)
    static_cast<double4_32a *>(a.w)[q] = make_double4_32a(w[0], w[1], w[2], 0.0);
  else
    w_pair_store(a.w, q, static_cast<float>(w[0]), static_cast<float>(w[1]), static_cast<float>(w[2]));
}

}  // namespace

size_t vjp_smem_bytes(int precision, int tj) {
  return static_cast<size_t>(kStages) * tj * (precision == 0 ? VjpLayout<0>::kBytesPerSource : VjpLayout<1>::kBytesPerSource);
}

// The VJP runs with fixed tiles: FP64 128 threads, mixed 256 threads, IPT 1.
int vjp_threads(int precision) { return precision == 0 ? 128 : 256; }

cudaError_t vjp_prepare(int precision, size_t smem, int *occ) {
  cudaError_t e;
  if (precision == 0) {
    e = cudaFuncSetAttribute(vjp_kernel<0, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, vjp_kernel<0, 128>, 128, smem);
  } else {
    e = cudaFuncSetAttribute(vjp_kernel<1, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, vjp_kernel<1, 256>, 256, smem);
  }
  return e;
}

cudaError_t launch_vjp(int precision, int grid, size_t smem, const VjpArgs &a, cudaStream_t s) {
  if (precision == 0)
    vjp_kernel<0, 128><<<grid, 128, smem, s>>>(a);
  else
    vjp_kernel<1, 256><<<grid, 256, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(int precision, const AdjArgs &a, cudaStream_t s) {
  if (a.N <= 0) return cudaSuccess;
  const int grid = (a.N + 255) / 256;
  if (precision == 0)
    adjoint_kernel<0><<<grid, 256, 0, s>>>(a);
  else
    adjoint_kernel<1><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_init(int precision, const AdjArgs &a, const double *dr, const double *dv, cudaStream_t s) {
  if (a.N <= 0) return cudaSuccess;
  const int grid = (a.N + 255) / 256;
  if (precision == 0)
    adjoint_init_kernel<0><<<grid, 256, 0, s>>>(a, dr, dv);
  else
    adjoint_init_kernel<1><<<grid, 256, 0, s>>>(a, dr, dv);
  return cudaGetLastError();
}

}  // namespace nb
