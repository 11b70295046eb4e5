// nbody_accel_static: all-pairs gravitational accelerations of one system,
// FP64, without allocating device memory.  Some callers cannot allocate: hosts that reserve all device
// memory up front and forbid allocation afterwards (real-time or embedded
// loops, services with a fixed memory budget), and components that run while
// another allocator owns the device memory, where an extra cudaMalloc may fail
// or stall.  This entry point therefore keeps its scratch (the staged
// sources, the partial sums, the work tables and the fault flags) in one
// file-scope __device__ array of fixed size instead of asking for memory.
//
// The array is shared by every call on a device and keeps the previous
// call's contents; each call rewrites the staged sources and work tables it
// reads and clears the fault flags and the work counter, which must start
// at zero.  Calls whose work overlaps on the GPU
// (concurrent streams, or several host threads) race on the array and give
// wrong results: serialise them.  Every GPU that loads this library holds the
// array (kStaticScratchBytes) until the process exits.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "nbody.h"
#include "nbody_internal.h"

namespace {

constexpr int64_t kMaxBodies = NBODY_STATIC_MAX_BODIES;
constexpr int kThreads = 128;  // targets per block (IPT 1)
constexpr int kTj = 256;       // sources per shared-memory stage
constexpr int kMaxBlocks = static_cast<int>((kMaxBodies + kThreads - 1) / kThreads);

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Layout of the static scratch (byte offsets, each 256-byte aligned).
constexpr size_t kOffStage = 0;                                                  // double4 (x, y, z, G m) [max]
constexpr size_t kOffPartial = kOffStage + 32 * kMaxBodies;                      // double [3][max]
constexpr size_t kOffNsl = kOffPartial + 24 * kMaxBodies;                        // uint16 [max]
constexpr size_t kOffBlks = kOffNsl + align256(2 * kMaxBodies);                  // Blk [kMaxBlocks]
constexpr size_t kOffSegs = kOffBlks + align256(sizeof(nb::Blk) * kMaxBlocks);   // Seg [kMaxBlocks]
constexpr size_t kOffSegOff = kOffSegs + align256(sizeof(nb::Seg) * kMaxBlocks);  // int32 [kMaxBlocks + 1]
constexpr size_t kOffFlags = kOffSegOff + align256(sizeof(int32_t) * (kMaxBlocks + 1));  // unsigned
constexpr size_t kOffDyn = kOffFlags + 16;                                       // int32 [2] chunk counter
constexpr size_t kStaticScratchBytes = kOffFlags + 256;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device addresses of g_static_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Failure messages go where nbody_last_error(NULL) reads them.
nbody_status fail(nbody_status st, const char *msg) {
  nb::set_last_error(msg);
  return st;
}

// One block of kThreads targets per CTA, each against all n sources (no
// split): block b is CTA b's only segment and every body has one partial row.
__global__ void static_tables_kernel(int32_t n, nb::Blk *blks, nb::Seg *segs, int32_t *seg_off, uint16_t *nsl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) nsl[i] = 1;
  const int n_blocks = (n + kThreads - 1) / kThreads;
  if (i > n_blocks) return;
  seg_off[i] = i;
  if (i == n_blocks) return;
  nb::Blk k;
  k.i0 = i * kThreads;
  k.i1 = min(k.i0 + kThreads, n);
  k.q0 = k.i0;
  k.nsplit = 1;
  blks[i] = k;
  nb::Seg sg;
  sg.blk = i;
  sg.s0 = 0;
  sg.s1 = n;
  sg.slot = 0;
  segs[i] = sg;
}

}  // namespace

extern "C" nbody_status nbody_accel_static(int64_t n, double G, const double *x, const double *y, const double *z,
                                           const double *m, double *ax, double *ay, double *az, void *cuda_stream) {
  nb::set_last_error("");
  if (n < 1 || n > kMaxBodies) return fail(NBODY_EINVAL, "n must be in [1, NBODY_STATIC_MAX_BODIES]");
  if (!x || !y || !z || !m || !ax || !ay || !az) return fail(NBODY_EINVAL, "a pointer is NULL");
  if (!(G > 0.0)) return fail(NBODY_EINVAL, "G must be > 0");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(NBODY_ECUDA, "no usable CUDA device");
  // The call ends with a copy to pageable host memory and a synchronize,
  // which a stream capture cannot hold: refuse before touching the stream.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(static_cast<cudaStream_t>(cuda_stream), &cap) != cudaSuccess)
    return fail(NBODY_ECUDA, "cudaStreamIsCapturing failed");
  if (cap != cudaStreamCaptureStatusNone) return fail(NBODY_EINVAL, "the stream is being captured into a graph");
  void *base = nullptr;
  {
    // First call on this device: find the device address of the array (the
    // host-side symbol is only a stand-in and must never reach a kernel).
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess || !p) return fail(NBODY_ECUDA, "cudaGetSymbolAddress failed for the static scratch");
      g_addr[dev] = p;
    }
    base = g_addr[dev];
  }
  unsigned char *s = static_cast<unsigned char *>(base);
  void *stage = s + kOffStage;
  double *partial = reinterpret_cast<double *>(s + kOffPartial);
  uint16_t *nsl = reinterpret_cast<uint16_t *>(s + kOffNsl);
  nb::Blk *blks = reinterpret_cast<nb::Blk *>(s + kOffBlks);
  nb::Seg *segs = reinterpret_cast<nb::Seg *>(s + kOffSegs);
  int32_t *seg_off = reinterpret_cast<int32_t *>(s + kOffSegOff);
  unsigned *flags = reinterpret_cast<unsigned *>(s + kOffFlags);
  int32_t *dyn = reinterpret_cast<int32_t *>(s + kOffDyn);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int N = static_cast<int>(n);
  const int n_blocks = (N + kThreads - 1) / kThreads;

  // The fault flags and the chunk counter start at zero on every call; the
  // tables are rewritten.
  if (cudaMemsetAsync(flags, 0, 256, st) != cudaSuccess) return fail(NBODY_ECUDA, "cudaMemsetAsync failed");
  const int span = N > n_blocks + 1 ? N : n_blocks + 1;
  static_tables_kernel<<<(span + 127) / 128, 128, 0, st>>>(N, blks, segs, seg_off, nsl);
  if (cudaGetLastError() != cudaSuccess) return fail(NBODY_ECUDA, "table launch failed");

  nb::PrepArgs p{};
  // The staging kernel validates positions and masses; it also reads
  // velocities for that check, which this entry point does not take, so the
  // positions stand in for them.
  p.x = x; p.y = y; p.z = z; p.vx = x; p.vy = y; p.vz = z;
  p.m = m;
  p.stage = stage;
  p.flags = flags;
  p.N = N;
  p.drift = 0;
  p.check = 1;
  p.G = G;
  if (nb::launch_prep(0, p, st) != cudaSuccess) return fail(NBODY_ECUDA, "staging launch failed");

  nb::ForceArgs fa{};
  fa.cur = stage;
  fa.partial = partial;
  fa.flags = flags;
  fa.blks = blks;
  fa.segs = segs;
  fa.seg_off = seg_off;
  fa.dyn_ctr = dyn;
  fa.n_dyn = 0;
  fa.N = N;
  fa.tj = kTj;
  fa.stages = nb::kStages;
  if (nb::launch_force(0, kThreads, 1, n_blocks, nb::force_smem_bytes(0, kTj, nb::kStages), fa, st, false) != cudaSuccess)
    return fail(NBODY_ECUDA, "force launch failed");
  nb::VerletArgs va{};
  va.ax = ax; va.ay = ay; va.az = az;
  va.partial = partial;
  va.nsl = nsl;
  va.flags = flags;
  va.N = N;
  va.p_begin = 0;
  va.p_end = N;
  va.mode = nb::kModeForce;
  if (nb::launch_verlet(0, va, st, false) != cudaSuccess) return fail(NBODY_ECUDA, "sum launch failed");

  unsigned f = 0;
  if (cudaMemcpyAsync(&f, flags, sizeof f, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(NBODY_ECUDA, "synchronisation failed");
  if (f & nb::kFlagBadInput) return fail(NBODY_EINVAL, "non-finite position or negative/non-finite mass");
  if (f & nb::kFlagTimeout) return fail(NBODY_ETIMEOUT, "a bounded device wait ran out");
  if (f & nb::kFlagNonFinite) return fail(NBODY_EINVAL, "non-finite acceleration: two bodies coincide");
  return NBODY_OK;
}
