// Internal interface between the host C-ABI (api.cu) and the kernels.
// Not installed; include/nbody.h is the public boundary.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nb {

// Device-side fault flags (bitwise OR into Scratch::flags).
enum : unsigned {
  kFlagNonFinite = 1u,  // an acceleration (or input) was NaN/Inf
  kFlagTimeout = 2u,    // a bounded mbarrier wait ran out
  kFlagBadInput = 4u,   // negative mass or non-finite state at staging time
};

// One unit of force work: targets [i0, i1) of one system against the
// sources [j0, j1) of the same system.  The sources of a target block are
// split into `nsplit` chunks; `slot` is this chunk's index (partial-sum row)
// and `ib` the global index of the target block (arrival counter).
struct Item {
  int32_t i0, i1, j0, j1;
  int32_t slot, nsplit, ib, sys;
};
static_assert(sizeof(Item) == 32, "Item layout");

enum Mode : int32_t {
  kModeForce = 0,  // write a = Eq. 1 only
  kModeStep = 1,   // Eq. 4 kick with the new a, then Eq. 3 drift into the next stage
};

// Arguments of one force launch (passed by value).
struct StepArgs {
  // state (caller-owned or the adjoint's shadow copy)
  double *x, *y, *z, *vx, *vy, *vz;
  double *ax, *ay, *az;  // a at the previous step in, a at this step out
  // staged sources of this step and the stage the epilogue fills for the next
  const void *cur_a, *cur_b;  // FP64: double4 (x,y,z,Gm); mixed: float4 hi, float4 lo
  void *nxt_a, *nxt_b;
  double *Rx, *Ry, *Rz;  // mixed only: FP64 positions of the current step (updated in place)
  double *partial;       // [jsplit][3][N] partial sums
  int32_t *arrive;       // [n_iblocks] arrival counters (self-resetting)
  int32_t *work_ctr;     // persistent-grid work counter (self-resetting)
  int32_t *exit_ctr;
  unsigned *flags;
  const Item *items;
  int32_t n_items;
  int32_t N;
  int32_t tj;
  int32_t mode;
  double dt, half_dt, half_dt2;
};

// Staging / pre-drift over all N bodies: stage r (mode 0) or drift(r, v, a)
// (mode 1) into the stage buffers, with mu = G m.
struct PrepArgs {
  const double *x, *y, *z, *vx, *vy, *vz, *ax, *ay, *az, *m;
  void *stage_a, *stage_b;
  double *Rx, *Ry, *Rz;
  unsigned *flags;
  int32_t N;
  int32_t drift;
  int32_t check;  // validate inputs (finite state, m >= 0)
  double G, dt, half_dt2;
};

struct EnergyArgs {
  const double *x, *y, *z, *vx, *vy, *vz, *m;
  double *e_kin, *e_pot;  // per body
  const Item *items;      // one item per 256-body target block, j = whole system
  int32_t n_items;
  double G;
};

struct ReduceArgs {
  const double *e_kin, *e_pot;
  const int64_t *offsets;  // device copy, n_systems+1
  double *out;             // [2][n_systems]: kinetic, potential
  int32_t n_systems;
};

// Launchers (return the launch's cudaError_t).
cudaError_t launch_prep(int precision, const PrepArgs &a, cudaStream_t s);
cudaError_t launch_step(int precision, int threads, int ipt, int grid, size_t smem,
                        const StepArgs &a, cudaStream_t s);
bool step_config_supported(int precision, int threads, int ipt);
size_t step_smem_bytes(int precision, int tj);
cudaError_t launch_energy(const EnergyArgs &a, cudaStream_t s);
cudaError_t launch_energy_reduce(const ReduceArgs &a, cudaStream_t s);
cudaError_t run_peaks(double *out);
void set_last_error(const char *msg);  // message returned by nbody_last_error(NULL) on this thread

constexpr int kStages = 2;          // shared-memory pipeline depth of the force kernels
constexpr int kFoldEvery = 64;      // mixed path: FP32 sub-sums of 64 sources folded into a float pair
constexpr int kEnergyBlock = 256;

}  // namespace nb
