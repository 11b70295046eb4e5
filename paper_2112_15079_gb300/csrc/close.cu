// Close-encounter handling: impulse multiple time stepping of close pairs
// (Tuckerman, Berne and Martyna 1992), FP64, for the members of clusters of
// close pairs (close_pairs.h).
//
// Per Verlet step the force launch evaluates Eq. 1 at the staged positions
// and the per-body Verlet kernel closes the step for every body (bodies in
// no cluster are then done: with no near force the scheme is Verlet).  Two
// kernels then correct the cluster members and start their next step:
//   close_far_kernel: A_far of each member at its position -- Eq. 1 over
//     every source of its system except itself and its close partners,
//     summed directly (not as A - A_near, which would carry the rounding of
//     the dominant near term into a far force many orders smaller);
//   close_kernel, per cluster:
//     complete: v <- vh + dt/2 A_far       (vh saved by the previous sub-cycle)
//     start:    vh <- v + dt/2 A_far
//               k times, h = dt/k:  vh += h/2 a_near; r += h vh;
//                                   a_near <- A_near(r); vh += h/2 a_near
//               stage r for the next force launch; save vh, a_near.
// A_near(r)_p = sum over p's close pairs (p, j), j ascending, of
// mu_j (r_j - r_p) |r_j - r_p|^-3 (mu_j = G m_j), in the force kernel's FP64
// pair arithmetic.  At the start of an nbody_step call (start only) a_near
// is computed from the state.
#include "nbody_dev.cuh"

namespace nb {

constexpr int kFarThreads = 256;

// One CTA per chunk: the chunk's share of its member's far force, reduced in
// a fixed order (a tree over the threads' sums) into far_part.
__global__ void __launch_bounds__(kFarThreads) close_far_kernel(const CloseArgs a) {
  __shared__ double s_red[3][kFarThreads];
  __shared__ int32_t s_part[kFarPartners];
  grid_dependency_wait();    // positions written by the Verlet kernel
  grid_dependency_launch();  // the cluster kernel may start launching (it waits for us)
  const int g = blockIdx.x, t = threadIdx.x;
  const int mi = a.fc_mem[g], j0 = a.fc_j0[g], j1 = a.fc_j1[g];
  const int p = a.mem_body[mi];
  const double px = a.x[p], py = a.y[p], pz = a.z[p];
  // this member's close partners (at most kFarPartners, checked at init)
  const int e0 = a.mp_off[mi], ne = a.mp_off[mi + 1] - e0;
  if (t < ne) {
    const int q = a.mp_pair[e0 + t];
    const int ba = a.mem_body[a.pr_a[q]], bb = a.mem_body[a.pr_b[q]];
    s_part[t] = ba == p ? bb : ba;
  }
  __syncthreads();
  double sx = 0.0, sy = 0.0, sz = 0.0;
  for (int j = j0 + t; j < j1; j += kFarThreads) {
    if (j == p) continue;
    bool partner = false;
    for (int u = 0; u < ne; ++u) partner |= s_part[u] == j;
    if (partner) continue;
    const double dx = a.x[j] - px, dy = a.y[j] - py, dz = a.z[j] - pz;
    const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
    const double f = (a.G * a.m[j]) * inv_r3(r2);
    sx = fma(f, dx, sx);
    sy = fma(f, dy, sy);
    sz = fma(f, dz, sz);
  }
  s_red[0][t] = sx;
  s_red[1][t] = sy;
  s_red[2][t] = sz;
  for (int w = kFarThreads / 2; w > 0; w >>= 1) {
    __syncthreads();
    if (t < w)
      for (int d = 0; d < 3; ++d) s_red[d][t] += s_red[d][t + w];
  }
  if (t == 0)
    for (int d = 0; d < 3; ++d) a.far_part[static_cast<size_t>(d) * a.n_chunks + g] = s_red[d][0];
}

__global__ void __launch_bounds__(kCloseThreads) close_kernel(const CloseArgs a) {
  __shared__ double s_r[3][kCloseThreads], s_mu[kCloseThreads];
  // per pair (a, b): the term on a (mu_b s d) and on b (-mu_a s d), d = r_b - r_a
  __shared__ double s_ua[3][kCloseMaxPairs], s_ub[3][kCloseMaxPairs];
  grid_dependency_wait();    // the far forces, and the state and stage the Verlet kernel wrote
  grid_dependency_launch();  // the next kernel may start launching (it waits for us)
  const int c = blockIdx.x, t = threadIdx.x;
  const int m0 = a.cl_off[c], nm = a.cl_off[c + 1] - m0;
  const int p0 = a.pr_off[c], np = a.pr_off[c + 1] - p0;
  const int k = a.cl_k[c];
  const double h = a.dt / k, hh = 0.5 * h;
  const bool own = t < nm;
  const int mi = m0 + t;  // this thread's member
  const int b = own ? a.mem_body[mi] : 0;
  const size_t M = static_cast<size_t>(a.n_mem);
  double v[3] = {0.0, 0.0, 0.0}, an[3] = {0.0, 0.0, 0.0}, af[3] = {0.0, 0.0, 0.0};
  if (own) {
    s_r[0][t] = a.x[b];
    s_r[1][t] = a.y[b];
    s_r[2][t] = a.z[b];
    s_mu[t] = a.G * a.m[b];
    for (int g = a.mch_off[mi]; g < a.mch_off[mi + 1]; ++g)  // chunks in order
      for (int d = 0; d < 3; ++d) af[d] += a.far_part[static_cast<size_t>(d) * a.n_chunks + g];
    if (a.complete) {
      for (int d = 0; d < 3; ++d) {
        an[d] = a.an[d * M + mi];
        v[d] = fma(a.half_dt, af[d], a.vh[d * M + mi]);
      }
      a.vx[b] = v[0];
      a.vy[b] = v[1];
      a.vz[b] = v[2];
    } else {
      v[0] = a.vx[b];
      v[1] = a.vy[b];
      v[2] = a.vz[b];
    }
  }
  // A_near at the positions in s_r, into an (members only).
  auto near = [&]() {
    __syncthreads();  // positions written
    for (int q = t; q < np; q += kCloseThreads) {
      const int ia = a.pr_a[p0 + q] - m0, ib = a.pr_b[p0 + q] - m0;
      const double d[3] = {s_r[0][ib] - s_r[0][ia], s_r[1][ib] - s_r[1][ia], s_r[2][ib] - s_r[2][ia]};
      const double sq = inv_r3(fma(d[2], d[2], fma(d[1], d[1], d[0] * d[0])));
      const double fa = s_mu[ib] * sq, fb = s_mu[ia] * sq;  // as the force kernel: mu_j |d|^-3
      for (int u = 0; u < 3; ++u) {
        s_ua[u][q] = fa * d[u];
        s_ub[u][q] = fb * -d[u];
      }
    }
    __syncthreads();  // pair terms written (and every read of the positions done)
    if (own) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      for (int e = a.mp_off[mi]; e < a.mp_off[mi + 1]; ++e) {  // partners in ascending body order
        const int q = a.mp_pair[e] - p0;
        const bool first = a.pr_a[p0 + q] - m0 == t;  // this member is the pair's lower body
        s0 += first ? s_ua[0][q] : s_ub[0][q];
        s1 += first ? s_ua[1][q] : s_ub[1][q];
        s2 += first ? s_ua[2][q] : s_ub[2][q];
      }
      an[0] = s0;
      an[1] = s1;
      an[2] = s2;
    }
  };
  if (!a.complete) near();
  double vh[3];
  for (int d = 0; d < 3; ++d) vh[d] = fma(a.half_dt, af[d], v[d]);
  for (int sub = 0; sub < k; ++sub) {
    // (the previous near() ended with a barrier after its last read of the
    // positions, so they may be overwritten now)
    if (own)
      for (int d = 0; d < 3; ++d) {
        vh[d] = fma(hh, an[d], vh[d]);
        s_r[d][t] = fma(h, vh[d], s_r[d][t]);
      }
    near();
    for (int d = 0; d < 3; ++d) vh[d] = fma(hh, an[d], vh[d]);
  }
  if (!own) return;
  if (!(isfinite(an[0]) && isfinite(an[1]) && isfinite(an[2]) && isfinite(vh[0]) && isfinite(vh[1]) &&
        isfinite(vh[2])))
    atomicOr(a.flags, kFlagNonFinite);
  for (int d = 0; d < 3; ++d) {
    a.vh[d * M + mi] = vh[d];
    a.an[d * M + mi] = an[d];
  }
  const double rx = s_r[0][t], ry = s_r[1][t], rz = s_r[2][t];
  if (a.precision == 0) {
    static_cast<double4_32a *>(a.stage)[b] = make_double4_32a(rx, ry, rz, s_mu[t]);
  } else {
    a.Rx[b] = rx;
    a.Ry[b] = ry;
    a.Rz[b] = rz;
    float *w = static_cast<float *>(a.stage) + pair_off(a.qidx[b]);
    const float hx = hi_part(rx), hy = hi_part(ry), hz = hi_part(rz);
    w[kXh] = hx;
    w[kYh] = hy;
    w[kZh] = hz;
    w[kXl] = lo_part(rx, hx);
    w[kYl] = lo_part(ry, hy);
    w[kZl] = lo_part(rz, hz);
  }
}

namespace {
template <typename Kernel>
cudaError_t launch_pdl(Kernel k, int grid, int block, const CloseArgs &a, cudaStream_t s, bool chained) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, a);
}
}  // namespace

cudaError_t launch_close_far(const CloseArgs &a, cudaStream_t s, bool chained) {
  if (a.n_chunks <= 0) return cudaSuccess;
  return launch_pdl(close_far_kernel, a.n_chunks, kFarThreads, a, s, chained);
}

cudaError_t launch_close(const CloseArgs &a, int n_clusters, cudaStream_t s, bool chained) {
  if (n_clusters <= 0) return cudaSuccess;
  return launch_pdl(close_kernel, n_clusters, kCloseThreads, a, s, chained);
}

}  // namespace nb
