// Close-encounter handling: the sub-cycle of each cluster of close pairs
// (impulse multiple time stepping, Tuckerman, Berne and Martyna 1992), FP64.
//
// Per Verlet step the force launch evaluates Eq. 1 at the staged positions,
// the per-body Verlet kernel closes the step for every body, and this kernel
// then corrects the cluster members and starts their next step:
//   complete:  v <- vh + dt/2 (a - a_near)      (a = Eq. 1 just evaluated,
//              vh, a_near saved by the previous sub-cycle at these positions)
//   start:     vh <- v + dt/2 (a - a_near)      (the far half kick)
//              k times, h = dt/k:  vh += h/2 a_near; r += h vh;
//                                  a_near <- A_near(r); vh += h/2 a_near
//              stage r for the next force launch; save vh, a_near.
// A_near(r)_p = sum over p's close pairs (p, j), j ascending, of
// mu_j (r_j - r_p) |r_j - r_p|^-3 (mu_j = G m_j), in the force kernel's own
// FP64 arithmetic, so an isolated pair's far remainder a - a_near is exactly
// zero.  Bodies outside clusters keep the Verlet kernel's result, which is
// the same scheme with no near force.  At the start of an nbody_step call
// (start only) a_near is computed from the state.
#include "nbody_dev.cuh"

namespace nb {

__global__ void __launch_bounds__(kCloseThreads) close_kernel(const CloseArgs a) {
  __shared__ double s_r[3][kCloseThreads], s_mu[kCloseThreads];
  __shared__ double s_d[3][kCloseMaxPairs], s_s[kCloseMaxPairs];
  grid_dependency_wait();    // the state and stage the Verlet kernel wrote
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
  double v[3] = {0.0, 0.0, 0.0}, an[3] = {0.0, 0.0, 0.0}, acc[3] = {0.0, 0.0, 0.0};
  if (own) {
    s_r[0][t] = a.x[b];
    s_r[1][t] = a.y[b];
    s_r[2][t] = a.z[b];
    s_mu[t] = a.G * a.m[b];
    acc[0] = a.ax[b];
    acc[1] = a.ay[b];
    acc[2] = a.az[b];
    if (a.complete) {
      double vn[3];
      for (int d = 0; d < 3; ++d) {
        an[d] = a.an[d * M + mi];
        vn[d] = fma(a.half_dt, acc[d] - an[d], a.vh[d * M + mi]);
      }
      a.vx[b] = vn[0];
      a.vy[b] = vn[1];
      a.vz[b] = vn[2];
      v[0] = vn[0];
      v[1] = vn[1];
      v[2] = vn[2];
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
      const double dx = s_r[0][ib] - s_r[0][ia];
      const double dy = s_r[1][ib] - s_r[1][ia];
      const double dz = s_r[2][ib] - s_r[2][ia];
      s_d[0][q] = dx;
      s_d[1][q] = dy;
      s_d[2][q] = dz;
      s_s[q] = inv_r3(fma(dz, dz, fma(dy, dy, dx * dx)));
    }
    __syncthreads();  // pair terms written
    if (own) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      for (int e = a.mp_off[mi]; e < a.mp_off[mi + 1]; ++e) {
        const int q = a.mp_pair[e] - p0;
        const int ia = a.pr_a[p0 + q] - m0, ib = a.pr_b[p0 + q] - m0;
        const bool first = ia == t;  // the pair's lower body: d = r_b - r_a points to the partner
        const double f = s_mu[first ? ib : ia] * s_s[q];
        const double sg = first ? 1.0 : -1.0;
        s0 = fma(f, sg * s_d[0][q], s0);
        s1 = fma(f, sg * s_d[1][q], s1);
        s2 = fma(f, sg * s_d[2][q], s2);
      }
      an[0] = s0;
      an[1] = s1;
      an[2] = s2;
    }
  };
  if (!a.complete) near();
  double vh[3];
  for (int d = 0; d < 3; ++d) vh[d] = fma(a.half_dt, acc[d] - an[d], v[d]);
  for (int sub = 0; sub < k; ++sub) {
    __syncthreads();  // every thread is done reading the previous positions
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

cudaError_t launch_close(const CloseArgs &a, int n_clusters, cudaStream_t s, bool chained) {
  if (n_clusters <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(n_clusters);
  cfg.blockDim = dim3(kCloseThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, close_kernel, a);
}

}  // namespace nb
