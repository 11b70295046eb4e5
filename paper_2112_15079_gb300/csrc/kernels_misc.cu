// Staging / pre-drift kernel, energy kernels, and the force-launch dispatcher.
#include "nbody_dev.cuh"

namespace nb {

cudaError_t run_step_fp64(int op, int threads, int ipt, int grid, size_t smem, const StepArgs &a, cudaStream_t s,
                          int *occ);
cudaError_t run_step_mixed(int op, int threads, int ipt, int grid, size_t smem, const StepArgs &a, cudaStream_t s,
                           int *occ);

// grid == 0: only raise the dynamic shared-memory limit (see step_launch.cuh).
cudaError_t launch_step(int precision, int threads, int ipt, int grid, size_t smem, const StepArgs &a,
                        cudaStream_t s) {
  const int op = grid == 0 ? 1 : 0;
  return precision == 0 ? run_step_fp64(op, threads, ipt, grid, smem, a, s, nullptr)
                        : run_step_mixed(op, threads, ipt, grid, smem, a, s, nullptr);
}

int step_max_ctas_per_sm(int precision, int threads, int ipt, size_t smem) {
  int occ = 0;
  const StepArgs a{};
  cudaError_t e = precision == 0 ? run_step_fp64(2, threads, ipt, 0, smem, a, nullptr, &occ)
                                 : run_step_mixed(2, threads, ipt, 0, smem, a, nullptr, &occ);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

bool step_config_supported(int precision, int threads, int ipt) {
  (void)precision;
  return (threads == 64 || threads == 128 || threads == 256) && (ipt == 1 || ipt == 2 || ipt == 4);
}

size_t step_smem_bytes(int precision, int tj) {
  (void)precision;  // both layouts take 32 bytes per staged source
  return static_cast<size_t>(kStages) * tj * 32;
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
  if (a.drift) {
    rx = drift(rx, a.vx[p], a.ax[p], a.dt, a.half_dt2);
    ry = drift(ry, a.vy[p], a.ay[p], a.dt, a.half_dt2);
    rz = drift(rz, a.vz[p], a.az[p], a.dt, a.half_dt2);
  }
  const double mu = a.G * m;
  if (PREC == 0) {
    static_cast<double4_32a *>(a.stage)[p] = make_double4_32a(rx, ry, rz, mu);
  } else {
    a.Rx[p] = rx;
    a.Ry[p] = ry;
    a.Rz[p] = rz;
    const int q = a.qidx[p];
    float *w = static_cast<float *>(a.stage) + static_cast<size_t>(q >> 1) * 16 + (q & 1);
    const float hx = hi_part(rx), hy = hi_part(ry), hz = hi_part(rz);
    w[0] = hx;
    w[2] = hy;
    w[4] = hz;
    w[6] = static_cast<float>(mu);
    w[8] = lo_part(rx, hx);
    w[10] = lo_part(ry, hy);
    w[12] = lo_part(rz, hz);
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
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEnergyBlock) energy_kernel(const EnergyArgs a) {
  __shared__ double4_32a tile[kEnergyBlock];
  const Item it = a.items[blockIdx.x];
  const int p = it.i0 + threadIdx.x;
  const bool valid = p < it.i1;
  const int pp = valid ? p : it.i0;
  const double px = a.x[pp], py = a.y[pp], pz = a.z[pp];
  double phi = 0.0;
  for (int j0 = it.j0; j0 < it.j1; j0 += kEnergyBlock) {
    const int j = j0 + threadIdx.x;
    __syncthreads();
    if (j < it.j1) tile[threadIdx.x] = make_double4_32a(a.x[j], a.y[j], a.z[j], a.G * a.m[j]);
    __syncthreads();
    const int cnt = min(kEnergyBlock, it.j1 - j0);
    for (int u = 0; u < cnt; ++u) {
      const double4_32a s = tile[u];
      const double dx = s.x - px, dy = s.y - py, dz = s.z - pz;
      double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
      const bool self = (j0 + u) == pp;
      r2 = self ? 1.0 : r2;
      phi += self ? 0.0 : s.w * inv_r1(r2);
    }
  }
  if (valid) {
    const double m = a.m[p];
    const double v2 = fma(a.vz[p], a.vz[p], fma(a.vy[p], a.vy[p], a.vx[p] * a.vx[p]));
    a.e_kin[p] = 0.5 * m * v2;
    a.e_pot[p] = -0.5 * m * phi;
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
