// Instruction-throughput microbenchmarks that set the roofline denominators
// of the force kernels: FP32 FFMA, FP64 DFMA, MUFU reciprocal square roots
// (f32 and f64 seeds), f32<->f64 conversions, packed f32x2 FFMA; plus the SM
// clock seen during the FFMA run (clock64 against %globaltimer).
// Each thread runs kChains independent dependency chains; every store is
// out[blockIdx.x * blockDim.x + threadIdx.x], inside a buffer of exactly
// grid * block elements.
#include <cstdint>
#include <cuda_runtime.h>

#include "nbody_internal.h"

namespace nb {
namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;

enum Op { kFFMA, kDFMA, kRsqF, kRsqD, kCvt, kFFMA2 };

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float sum2(unsigned long long v) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
  return a + b;
}

template <int OP>
__global__ void __launch_bounds__(kBlock) peak_kernel(int iters, float *out, long long *clk) {
  long long c0 = clock64();
  unsigned long long g0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
  float f[kChains];
  double d[kChains];
  unsigned long long p[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    f[c] = 1.0f + c * 1e-3f + threadIdx.x * 1e-7f;
    d[c] = 1.0 + c * 1e-3 + threadIdx.x * 1e-7;
    p[c] = pack2(f[c], f[c] + 0.5f);
  }
  const unsigned long long pb = pack2(0.9999f, 0.9999f), pc = pack2(1e-4f, 1e-4f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if (OP == kFFMA) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[c]) : "f"(0.9999f), "f"(1e-4f));
      if (OP == kDFMA) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(d[c]) : "d"(0.9999999), "d"(1e-9));
      if (OP == kRsqF) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(f[c]));
      if (OP == kRsqD) asm volatile("rsqrt.approx.ftz.f64 %0, %0;" : "+d"(d[c]));
      if (OP == kCvt) {
        double t;
        asm volatile("cvt.f64.f32 %0, %1;" : "=d"(t) : "f"(f[c]));
        asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(f[c]) : "d"(t));
      }
      if (OP == kFFMA2) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(p[c]) : "l"(pb), "l"(pc));
    }
  }
  float s = 0.f;
  double ds = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    s += f[c] + sum2(p[c]);
    ds += d[c];
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s + static_cast<float>(ds);
  long long c1 = clock64();
  unsigned long long g1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
  if (threadIdx.x == 0) {
    clk[2 * blockIdx.x] = c1 - c0;
    clk[2 * blockIdx.x + 1] = static_cast<long long>(g1 - g0);
  }
}

template <int OP>
cudaError_t time_op(int blocks, int iters, float *out, long long *clk, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
  peak_kernel<OP><<<blocks, kBlock>>>(iters / 8 + 1, out, clk);  // warm-up
  cudaEventRecord(e0);
  peak_kernel<OP><<<blocks, kBlock>>>(iters, out, clk);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e != cudaSuccess) return e;
  return cudaEventElapsedTime(ms, e0, e1);
}

}  // namespace

cudaError_t run_peaks(double *res) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = nsm * 4;
  float *out = nullptr;
  long long *clk = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaMalloc(&out, sizeof(float) * blocks * kBlock)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&clk, sizeof(long long) * 2 * blocks)) != cudaSuccess) {
    cudaFree(out);
    return e;
  }
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const double lanes = static_cast<double>(blocks) * kBlock * kChains;
  struct {
    int op, iters;
    double per;
  } plan[6] = {{kFFMA, 100000, 1}, {kDFMA, 2000, 1}, {kRsqF, 20000, 1},
               {kRsqD, 20000, 1},  {kCvt, 1000, 2},  {kFFMA2, 50000, 2}};
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) {
    float ms = 0.f;
    switch (plan[i].op) {
      case kFFMA: e = time_op<kFFMA>(blocks, plan[i].iters, out, clk, e0, e1, &ms); break;
      case kDFMA: e = time_op<kDFMA>(blocks, plan[i].iters, out, clk, e0, e1, &ms); break;
      case kRsqF: e = time_op<kRsqF>(blocks, plan[i].iters, out, clk, e0, e1, &ms); break;
      case kRsqD: e = time_op<kRsqD>(blocks, plan[i].iters, out, clk, e0, e1, &ms); break;
      case kCvt: e = time_op<kCvt>(blocks, plan[i].iters, out, clk, e0, e1, &ms); break;
      default: e = time_op<kFFMA2>(blocks, plan[i].iters, out, clk, e0, e1, &ms); break;
    }
    res[i] = lanes * plan[i].iters * plan[i].per / (ms * 1e-3) * 1e-9;
    if (i == 0 && e == cudaSuccess) {  // SM clock during the FFMA run
      long long *h = new long long[2 * blocks];
      e = cudaMemcpy(h, clk, sizeof(long long) * 2 * blocks, cudaMemcpyDeviceToHost);
      double mhz = 0.0;
      for (int b = 0; b < blocks; ++b) mhz += static_cast<double>(h[2 * b]) / static_cast<double>(h[2 * b + 1]) * 1e3;
      res[6] = mhz / blocks;
      delete[] h;
    }
  }
  res[7] = nsm;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  cudaFree(clk);
  return e;
}

}  // namespace nb
