// Staging / pre-drift kernel, energy kernels, and the force-launch dispatcher.
#include "nbody_dev.cuh"

namespace nb {

cudaError_t launch_step_fp64(int threads, int ipt, int grid, size_t smem, const StepArgs &a, cudaStream_t s);
cudaError_t launch_step_mixed(int threads, int ipt, int grid, size_t smem, const StepArgs &a, cudaStream_t s);

cudaError_t launch_step(int precision, int threads, int ipt, int grid, size_t smem, const StepArgs &a,
                        cudaStream_t s) {
  return precision == 0 ? launch_step_fp64(threads, ipt, grid, smem, a, s)
                        : launch_step_mixed(threads, ipt, grid, smem, a, s);
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
// drift of (r, v, a) (drift == 1), with mu = G m.  FP64: double4_32a (x,y,z,mu).
// Mixed: FP64 positions R plus float4 hi (x,y,z,mu) and lo (x,y,z,0).
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
    static_cast<double4_32a *>(a.stage_a)[p] = make_double4_32a(rx, ry, rz, mu);
  } else {
    a.Rx[p] = rx;
    a.Ry[p] = ry;
    a.Rz[p] = rz;
    const float hx = hi_part(rx), hy = hi_part(ry), hz = hi_part(rz);
    static_cast<float4 *>(a.stage_a)[p] = make_float4(hx, hy, hz, static_cast<float>(mu));
    static_cast<float4 *>(a.stage_b)[p] = make_float4(lo_part(rx, hx), lo_part(ry, hy), lo_part(rz, hz), 0.f);
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
