// Internal interface between the host C-ABI (api.cu) and the kernels.
// Not installed; include/nbody.h is the public boundary.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pair_once_plan.h"
#include "work_plan.h"

namespace nb {

// Device-side fault flags (bitwise OR into the context's flags word).
enum : unsigned {
  kFlagNonFinite = 1u,  // an acceleration (or input) was NaN/Inf
  kFlagTimeout = 2u,    // a bounded mbarrier wait ran out
  kFlagBadInput = 4u,   // negative mass or non-finite state at staging time
};

// Work description shared by the energy kernel: targets [i0, i1) against
// sources [j0, j1) of the same system.
struct Item {
  int32_t i0, i1, j0, j1;
  int32_t slot, nsplit, ib, sys;
};
static_assert(sizeof(Item) == 32, "Item layout");

// Blk (target block) and Seg (segment of a block's sources): work_plan.h.

// Arguments of one force launch (Eq. 1 partial sums).  The work is cut into
// pieces; piece k is the segment list segs[seg_off[k] .. seg_off[k+1]).
// Pieces 0..gridDim.x-1 are the CTAs' equal static shares (CTA c takes piece
// c); pieces gridDim.x .. gridDim.x+n_dyn-1 are small chunks of the rest of
// the work, pulled in order from an atomic counter by whichever CTA is free,
// so CTAs that the warp scheduler favoured absorb the others' lag.  Each
// segment writes a fixed partial row, so results do not depend on which CTA
// ran it.
struct ForceArgs {
  const void *cur;  // staged sources: FP64 double4 (x,y,z,Gm) per body; mixed pair blocks
  double *partial;  // [rows][3][N]: doubles (FP64) or float pairs (mixed), 24 B per row and body
  const int32_t *perm;  // [stage entries] body of each stage entry (mixed, spatial order); NULL: the
                        // block's targets are bodies i0.. in order
  const float4 *boxes;  // mixed: [groups][2] widened box of stage pairs [32 g, 32 g + 32) (box_kernel)
  unsigned *flags;
  const Blk *blks;
  const Seg *segs;
  const int32_t *seg_off;  // [gridDim.x + n_dyn + 1]
  int32_t *dyn_ctr;        // [2]: next dynamic chunk, CTAs done (the last one resets both)
  int32_t n_dyn;
  int32_t N;
  int32_t tj;
  int32_t stages;  // ring depth, kStages..kMaxStages (force_stages)
};

enum Mode : int32_t {
  kModeForce = 0,  // write a = Eq. 1 only
  kModeStep = 1,   // Eq. 4 kick with the new a, then Eq. 3 drift into the next stage
  kModeLeapfrog = 2,  // drift-kick-drift: full kick at the half-step force, two half drifts
};

// Arguments of the per-body Verlet kernel that completes a step: sums the
// force partials of body p (rows 0..nsl[p]-1, in order), then applies Eq. 4
// and Eq. 3 and stages r_{i+1} for the next force launch.
struct VerletArgs {
  double *x, *y, *z, *vx, *vy, *vz;  // state (caller-owned or the adjoint's shadow copy)
  double *ax, *ay, *az;              // a at the previous step in, a at this step out
  const void *cur;                   // staged sources of this step (mixed: mu is copied from here)
  void *nxt;                         // stage of the next step
  double *Rx, *Ry, *Rz;              // mixed only: FP64 positions of the current step (in place)
  const double *partial;
  const uint16_t *nsl;  // [N] partial rows of body p
  const int32_t *qidx;  // [N] stage index of body p (mixed); NULL: p
  unsigned *flags;
  int32_t N;
  int32_t p_begin, p_end;  // the bodies this launch completes: [p_begin, p_end) (all: 0, N)
  int32_t mode;
  int32_t release_early;  // 1: the next force grid may launch at once (it fits one CTA per SM)
  double dt, half_dt, half_dt2;
};

// Vector-Jacobian product of Eq. 1 at staged positions r_k (vjp.cu): for
// every target q, J^T w and the mass term, as one partial row per segment of
// the same kind of work tables as the force kernel ([rows][4][N]).
struct VjpArgs {
  const void *pos;  // positions staged by the forward pass (its layout)
  const int32_t *perm;  // as ForceArgs::perm
  const void *w;    // w per stage entry: FP64 double4; mixed pair blocks (16 B per entry)
  double *partial;  // [rows][4][N]: doubles (FP64) or float pairs (mixed)
  unsigned *flags;
  const Blk *blks;
  const Seg *segs;
  const int32_t *seg_off;  // [gridDim.x + 1]
  int32_t N;
  int32_t tj;
  int32_t stall;  // test hook: CTA 0 never issues its first tile, so its bounded wait runs out
};

// One step of the reverse sweep per body (vjp.cu).
struct AdjArgs {
  double *rho, *nu;  // [3][N] dL/dr, dL/dv
  double *gm;        // [N] dL/dm
  void *w;           // staged w for the next product (same layout as VjpArgs::w)
  const double *partial;
  const uint16_t *nsl;
  const int32_t *qidx;  // mixed: stage index of body p; NULL: p
  unsigned *flags;
  int32_t N;
  int32_t mode;  // 0: step, stage alpha'+dt/2 nu'; 1: step, stage alpha'; 2: last product only
  double G, dt, half_dt, half_dt2;
};

// Single-launch kernels (smalln.cu): all steps of one FP64 system in one
// launch, a thread-block cluster (small systems) or a cooperative grid
// (mid-size systems); state read from and written back to these arrays.
struct SmallArgs {
  double *x, *y, *z, *vx, *vy, *vz, *ax, *ay, *az;
  const double *m;
  unsigned *flags;
  double *xg;      // grid kernel: [2][3][N] position exchange buffers
  unsigned *gbar;  // grid kernel: barrier arrivals, zero at launch
  int32_t N;
  int64_t n_steps;
  double G, dt, half_dt, half_dt2;
  int32_t stall;  // test hook: CTA 0 skips one barrier arrival (the waits run out)
};

// Staging / pre-drift over all N bodies: stage r (drift == 0) or
// drift(r, v, a) (drift == 1), with mu = G m, at stage index qidx[p]
// (mixed; FP64 stages in body order).
struct PrepArgs {
  const double *x, *y, *z, *vx, *vy, *vz, *ax, *ay, *az, *m;
  void *stage;
  const int32_t *qidx;
  double *Rx, *Ry, *Rz;
  unsigned *flags;
  int32_t N;
  int32_t drift;  // 0: stage r; 1: stage the Eq. 3 drift of r; 2: stage r + dt/2 v (leapfrog)
  int32_t check;  // validate inputs (finite state, m >= 0)
  double G, dt, half_dt2;
};

// FP64 force kernel with each pair once (sym.cu): work items are block
// pairs (I, J), I <= J, of one system; block sizes in pair_once_plan.h.
struct SymArgs {
  const double4_32a *cur;  // staged sources (x, y, z, G m) per body
  double *partial;         // [blocks][3][N]: row J of a body of block I holds block J's pull
  const int4 *pairs;       // (first body of the system, its bodies, I, J)
  int32_t n_pairs;
  int32_t *ctr;            // [2]: next item, CTAs done (the last one resets both)
  int32_t N;
  int32_t tiles;           // 32-body tiles per block: 2 (64-body blocks, force_sym_kernel) or wide
};

// Mixed force kernel with each pair once (sym_mixed.cu): block pairs (I, J),
// I <= J, of 32 T stage entries of one system; a CTA of W = T / 4 warps per
// item (pair_once_plan.h).
struct MsymArgs {
  const float *cur;        // mixed stage (pair blocks of two entries)
  const float4 *boxes;     // [groups][2] widened boxes of the stage groups (box_kernel)
  double *partial;         // [blocks][3][N] float pairs: row J of a body of block I holds block J's pull
  const int4 *pairs;       // (first stage entry of the system, its bodies, I, J)
  const int32_t *perm;     // [stage entries] body of each entry
  int32_t n_pairs;
  int32_t *ctr;            // [2]: next item, CTAs done (the last one resets both)
  int32_t N;
  int32_t tiles;           // T: 32-entry tiles per block, kMsymMinTiles .. kMsymMaxTiles (a power of two)
  int32_t warps;           // W = T / 4 warps per CTA
};

// The adjoint's VJP with each pair once (FP64, sym.cu): the same items,
// rows of 4 values per body (J^T w and the mass sum).
struct VjpSymArgs {
  const double4_32a *pos;  // positions staged by the forward pass (x, y, z, G m)
  const double4_32a *w;    // w per body (x, y, z, -)
  double *partial;         // [blocks][4][N]
  const int4 *pairs;
  int32_t n_pairs;
  int32_t *ctr;
  int32_t N;
};

// Close-encounter handling (close.cu): clusters of close pairs sub-cycled in
// FP64 after each step's Verlet kernel.  Members and pairs as CloseSet in
// close_pairs.h (global member / pair indices).
constexpr int kCloseThreads = 256;    // members per cluster at most (one thread each)
constexpr int kCloseMaxPairs = 1024;  // pairs per cluster at most
constexpr int kFarChunk = 4096;       // sources per CTA of the members' far-force kernel
constexpr int kFarPartners = 64;      // close partners of one body at most
struct CloseArgs {
  double *x, *y, *z, *vx, *vy, *vz;  // state (v written in complete mode)
  const double *m;
  double *an, *vh;                   // [3][n_mem]: a_near and the sub-cycle velocity of each member
  double *far_part;                  // [3][n_chunks]: the members' far force, one chunk of sources each
  const int32_t *cl_off, *cl_k, *mem_body, *pr_off, *pr_a, *pr_b, *mp_off, *mp_pair;
  // far-force chunks: chunk g sums member fc_mem[g]'s sources [fc_j0[g], fc_j1[g]);
  // member i's chunks are mch_off[i] .. mch_off[i + 1]
  const int32_t *fc_mem, *fc_j0, *fc_j1, *mch_off;
  int32_t n_chunks;
  void *stage;                       // the next force launch's sources (FP64 double4 / mixed pair blocks)
  const int32_t *qidx;               // mixed: stage entry of each body
  double *Rx, *Ry, *Rz;              // mixed: FP64 staged positions
  unsigned *flags;
  int32_t n_mem;
  int32_t complete;                  // 1: first finish the step the Verlet kernel closed
  int32_t precision;
  double G, dt, half_dt;
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

// Launchers (return the launch's cudaError_t).  `chained`: launch with
// programmatic stream serialization, so the kernel may start while the
// previous one in the stream finishes (each kernel waits for its inputs).
cudaError_t launch_prep(int precision, const PrepArgs &a, cudaStream_t s);
// Mixed stages: fill n_pairs pair blocks with inert padding sources.
cudaError_t launch_pad_fill(void *stage, int64_t n_pairs, cudaStream_t s);
// FP64 stages: fill n entries with inert padding sources.
cudaError_t launch_pad_fill_fp64(void *stage, int64_t n, cudaStream_t s);
cudaError_t launch_force(int precision, int threads, int ipt, int grid, size_t smem, const ForceArgs &a,
                         cudaStream_t s, bool chained);
// Mixed stages: the widened box of every group of kBoxPairs stage pairs
// (boxes[2 g], boxes[2 g + 1]: low and high corner), read by the next force
// launch.  `chained`: programmatic stream serialization, as the force launch.
cudaError_t launch_boxes(const void *stage, int64_t n_pairs, float4 *boxes, cudaStream_t s, bool chained);
cudaError_t launch_verlet(int precision, const VerletArgs &a, cudaStream_t s, bool chained);

// Classical RK4 on y = (r, v), y' = (v, A(r)) (kernels_misc.cu).  rk_stage
// kernel, stage s = 2..5: sums the force partials of body p into a_s (as the
// Verlet kernel does; for s = 5 that is A at the new state), then
//   s = 2, 3: AR += 2 v_s, AV += 2 a_s; r_{s+1} = r + c v_s, v_{s+1} = v + c a_s
//             (c = dt/2 for s = 2, dt for s = 3) -> stage r_{s+1}, V = v_{s+1};
//   s = 4:    r += dt/6 (AR + v_4), v += dt/6 (AV + a_4) -> caller state, stage r;
//   s = 5:    a = a_5; then stage 1 of the next step (as rk_prep).
// rk_prep (stage 1 from the state): AR = v, AV = a, V = v + dt/2 a, stage
// r_2 = r + dt/2 v.
struct RkArgs {
  double *x, *y, *z, *vx, *vy, *vz;  // the state (r, v): read, written at s = 4
  double *ax, *ay, *az;              // A(r) of the state: read by rk_prep, written at s = 5
  const double *m;                   // rk_prep only (mu = G m is staged)
  double *V;                         // [3N] velocity of the current stage
  double *AR, *AV;                   // [3N] weighted sums of the stage derivatives
  const void *cur;                   // staged sources of this stage (mu is copied from here)
  void *nxt;                         // stage written for the next force launch
  const double *partial;
  const uint16_t *nsl;
  const int32_t *qidx;  // [N] stage index of body p (mixed); NULL: p
  unsigned *flags;
  int32_t N;
  int32_t stage;
  int32_t release_early;
  double G, dt;
};
cudaError_t launch_rk_stage(int precision, const RkArgs &a, cudaStream_t s, bool chained);
cudaError_t launch_rk_prep(int precision, const RkArgs &a, cudaStream_t s);
cudaError_t force_set_smem(int precision, int threads, int ipt, size_t smem);  // raise the dynamic smem limit
int force_max_ctas_per_sm(int precision, int threads, int ipt, size_t smem);
bool force_config_supported(int precision, int threads, int ipt);
size_t force_smem_bytes(int precision, int tj, int stages);  // dynamic smem of a ring of `stages` tiles
cudaError_t launch_force_sym(const SymArgs &a, int grid, cudaStream_t s, bool chained);
cudaError_t launch_vjp_sym(const VjpSymArgs &a, int grid, cudaStream_t s);
int force_sym_ctas_per_sm(int tiles);   // resident CTAs per SM (raises the wide kernel's smem limit)
size_t force_sym_smem_bytes(int tiles);
cudaError_t launch_force_msym(const MsymArgs &a, int grid, cudaStream_t s, bool chained);
int force_msym_ctas_per_sm(int tiles, int warps);  // resident CTAs per SM (raises the smem limit)
size_t force_msym_smem_bytes(int tiles, int warps);
cudaError_t launch_close(const CloseArgs &a, int n_clusters, cudaStream_t s, bool chained);
cudaError_t launch_close_far(const CloseArgs &a, cudaStream_t s, bool chained);
cudaError_t launch_energy(const EnergyArgs &a, cudaStream_t s);
cudaError_t launch_energy_reduce(const ReduceArgs &a, cudaStream_t s);
cudaError_t run_peaks(double *out);
int small_max_bodies();
cudaError_t small_prepare();
cudaError_t launch_small(const SmallArgs &a, cudaStream_t s);
int grid_max_bodies();
// Shape of the grid kernel for N bodies on nsm SMs: warps (targets) per CTA
// and CTAs, all resident at once; an error if no shape fits.
cudaError_t grid_shape(int N, int nsm, int *warps, int *ctas);
cudaError_t launch_grid(const SmallArgs &a, int warps, int ctas, cudaStream_t s);
size_t vjp_smem_bytes(int precision, int tj);
int vjp_threads(int precision);
cudaError_t vjp_prepare(int precision, size_t smem, int *occ);  // raise the smem limit, resident CTAs/SM
cudaError_t launch_vjp(int precision, int grid, size_t smem, const VjpArgs &a, cudaStream_t s);
cudaError_t launch_adjoint(int precision, const AdjArgs &a, cudaStream_t s);
cudaError_t launch_adjoint_init(int precision, const AdjArgs &a, const double *dr, const double *dv, cudaStream_t s);
void set_last_error(const char *msg);  // message returned by nbody_last_error(NULL) on this thread

constexpr int kStages = 2;          // shared-memory pipeline depth of the VJP kernels (and the force kernels' least)
constexpr int kMaxStages = 4;       // the force kernels' deepest ring (ForceArgs::stages)
constexpr int kFoldPairs = 64;      // mixed path: packed sub-sums of 64 source pairs folded into a float pair
constexpr float kPadCoord = 1e15f;  // mixed padding source: far away and massless (term exactly 0)
// Mixed force kernel: source groups of kBoxPairs pairs (64 sources) get a
// bounding box before each force launch; a warp whose targets are far from a
// group's box takes the hi-only path for it (see step_kernel.cuh).  kFarEps bounds the
// relative error that dropping the lo parts adds to one term of Eq. 1;
// kFarKappa = 2 / kFarEps + 1 is the separation, in units of the largest lo
// parts, beyond which that bound holds.
constexpr int kBoxPairs = 32;
constexpr float kFarEps = 1e-6f;
constexpr float kFarKappa = 2.0f / kFarEps + 1.0f;
constexpr int kEnergyBlock = 256;

}  // namespace nb
