/*
 * nbody.h -- C ABI of the GB300 (sm_103a) direct-sum N-body library.
 *
 * The method (arXiv:2112.15079, Section 2):
 *   Eq. 1   a_p = sum_{j != p} G m_j (r_j - r_p) / |r_j - r_p|^3
 *   Eq. 3   r_{i+1} = r_i + v_i dt + (1/2) a_i dt^2
 *   Eq. 4   v_{i+1} = v_i + (1/2) (a_i + a_{i+1}) dt
 * integrated at a fixed step dt (0.1 day in the paper), with the total
 * energy as the accuracy criterion (Sections 2 and 4).  No softening: the
 * pair j == p is excluded by index, and two distinct bodies at the same
 * position are rejected.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - State is structure-of-arrays FP64 in DEVICE memory owned by the caller:
 *   x, y, z (positions), vx, vy, vz (velocities), m (masses), each of length
 *   N = offsets[n_systems].  Several independent systems are stored back to
 *   back; system s owns bodies [offsets[s], offsets[s+1]).  Bodies of one
 *   system never interact with bodies of another.
 * - Vectors of 3N doubles ("3N, x|y|z blocks") hold the x components of all
 *   N bodies, then all y components, then all z components.
 * - Units are the caller's; G and dt must be consistent with them.
 * - Every call returns an nbody_status and never aborts or exits.  Work is
 *   asynchronous on the context's stream unless a call says "synchronous".
 *   Faults detected on the device (a non-finite acceleration, a bounded wait
 *   that ran out) are recorded in device flags and reported by the next
 *   synchronous call (nbody_sync, nbody_energy, nbody_grad).  A readable
 *   message is available from nbody_last_error.
 * - The library owns its scratch, graphs and snapshots; nbody_free releases
 *   them.  The caller must keep the bound state buffers alive until then.
 * - A context is not thread-safe; use one context per host thread.
 * - A context belongs to the CUDA device that is current at nbody_init (its
 *   state buffers and stream must live there).  Every later call on it makes
 *   that device current for the call's duration and restores the calling
 *   thread's device afterwards.
 * - Fault-injection hooks for tests (environment variables, unset in normal
 *   use): NBODY_INJECT_ALLOC_FAIL=k fails a context's k-th device allocation
 *   with NBODY_ENOMEM; NBODY_INJECT_WAIT_STALL=k (read by nbody_init) stalls
 *   one bounded device wait in the context's k-th launch that has one (an
 *   adjoint product: one source copy left unissued; a single-launch
 *   nbody_step call: one barrier arrival left out), so that wait runs out
 *   (~2 s), the kernel winds down, and nbody_grad / nbody_sync returns
 *   NBODY_ETIMEOUT.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nbody_ctx nbody_ctx; /* opaque, library-owned */

typedef enum {
  NBODY_OK = 0,
  NBODY_EINVAL = 1,     /* bad argument (null pointer, size, coincident bodies, ...) */
  NBODY_ENOMEM = 2,     /* device or host allocation failed */
  NBODY_ECUDA = 3,      /* a CUDA runtime call failed */
  NBODY_ENONFINITE = 4, /* an acceleration became NaN/Inf (e.g. a collision) */
  NBODY_ETIMEOUT = 5    /* a bounded device-side wait ran out */
} nbody_status;

typedef enum {
  /* FP64 everywhere: differences, 1/|d|^3, products and sums (Eq. 1). */
  NBODY_FP64 = 0,
  /* FP64 state and Verlet update (Eqs. 3-4); r_j - r_p formed from a
   * hi/lo float split of the FP64 positions (about as exact as the FP64
   * difference rounded to FP32); 1/|d|^3 and the m_j-weighted terms in
   * FP32; per-body sums kept as float pairs, folded every 128 terms.
   * Sources are kept in a spatial order; for a group of 64 sources whose
   * distance to a warp's 32 targets exceeds 2e6 times their largest lo
   * parts, the difference is taken from the hi parts alone, which moves each
   * such term by at most 1e-6 relative (see nbody_reorder). */
  NBODY_MIXED = 1
} nbody_precision;

typedef enum {
  /* Velocity Verlet, Eqs. 3-4: one evaluation of Eq. 1 per step. */
  NBODY_VERLET = 0,
  /* Classical fourth-order Runge-Kutta on y = (r, v), y' = (v, A(r)) -- the
   * higher-order method Section 2 names: k1 = f(y), k2 = f(y + dt/2 k1),
   * k3 = f(y + dt/2 k2), k4 = f(y + dt k3), y += dt/6 (k1 + 2 k2 + 2 k3 + k4).
   * Four evaluations of Eq. 1 per step; error O(dt^4). */
  NBODY_RK4 = 1,
  /* Leapfrog (Section 2), drift-kick-drift with synchronised output:
   * r_{n+1/2} = r_n + dt/2 v_n; v_{n+1} = v_n + dt A(r_{n+1/2});
   * r_{n+1} = r_{n+1/2} + dt/2 v_{n+1}.  One evaluation of Eq. 1 per step,
   * taken at the half-step positions; error O(dt^2); time-symmetric. */
  NBODY_LEAPFROG = 2
} nbody_integrator;

typedef struct {
  double G;           /* gravitational constant, > 0 */
  double dt;          /* step size, finite and != 0 (negative runs backwards) */
  int32_t precision;  /* nbody_precision */
  int32_t ckpt_every; /* adjoint checkpoint interval in steps; 0 selects 100 */
  int32_t flags;      /* bitwise OR of NBODY_FLAG_* */
  int32_t integrator; /* nbody_integrator (0, the zero value, is Verlet) */
  /* Path of a JSON file of autotuner results, or NULL (off).  nbody_init
   * takes its work decomposition (nbody_tiles) from the entry for this
   * context's precision, integrator, floor(log2(bodies)),
   * floor(log2(systems)), SM count and kernel build, if there is one;
   * nbody_autotune writes its winner there.  A missing, unreadable or
   * malformed file, or a stale entry (other kernels), is ignored: the
   * context starts from the built-in defaults.  The string is copied. */
  const char *tune_cache;
  /* Close-encounter handling, for bodies whose two-body orbit the step
   * cannot follow (a moon with a period below a few dt is unstable under
   * Eqs. 3-4 at any precision).  An extension beyond Section 2's method:
   * impulse multiple time stepping (Tuckerman, Berne and Martyna, J. Chem.
   * Phys. 97, 1990, 1992) with the force split by pairs.  0 = off.  Else a
   * pair of bodies of one system is close if its two-body angular frequency
   * w = sqrt(G (m_p + m_j) / d^3), at the positions nbody_init (or
   * nbody_reset) sees, has w |dt| > close_omega_dt; bodies joined by close
   * pairs form clusters.  A step then is: v += dt/2 A_far; each cluster
   * takes k = ceil(max w |dt| / substep_omega_dt) velocity-Verlet sub-steps
   * of dt/k on the forces of its close pairs (A_near), FP64, every other
   * body drifts r += dt v; v += dt/2 A_far at the new positions.  A_far is
   * Eq. 1 in the context's precision for a body with no close pair, and for
   * a cluster member the FP64 sum over every body of its system but itself
   * and its close partners.  Without close pairs this is velocity Verlet.
   * Verlet integrator only; nbody_grad, nbody_kernel_times and nbody_shard
   * return EINVAL; at most 256 bodies and 1024 pairs per cluster, 64 close
   * partners per body and 1e6 sub-steps per step, else nbody_init returns
   * EINVAL. */
  double close_omega_dt;
  double substep_omega_dt; /* w h per sub-step, > 0 when close_omega_dt > 0 (e.g. 0.05) */
  /* Block size of the force kernels that evaluate each pair once (see
   * NBODY_FLAG_NO_SYM), 0 = automatic.  A body keeps one partial sum (24 B)
   * per block of its system.
   *   FP64, bodies per block.  Automatic: 64 when every system has at most
   *   65,536 bodies; above, the narrowest of 256 .. 4,096 (powers of two)
   *   whose partial sums take at most 2 GiB, else 4,096 if they take at most
   *   16 GiB (else every ordered pair is evaluated); and only when the
   *   systems hold at least 1.5 block pairs per SM.  Or set: 64, or a power
   *   of two from 256 to 4,096.  Blocks above 64 apply to the force only:
   *   nbody_grad's VJP then evaluates every ordered pair.
   *   Mixed, stage entries per block (the stage holds each system's bodies
   *   in a spatial order).  Automatic: for a largest system of at least
   *   65,536 bodies, the narrowest of 128 .. 2,048 that leaves it at most 128
   *   partial sums per body, if the block pairs keep 8 warps per SM busy and
   *   the sums take at most 16 GiB (else, and below 65,536 bodies, every
   *   ordered pair is evaluated).  Or set: a power of two from 128 to 2,048.
   *   Force only (nbody_grad's VJP evaluates every ordered pair).
   * A set size is used whatever the systems' sizes (for contexts that are
   * not row shards) if the partial sums take at most 16 GiB and 65,535 blocks
   * per system, else nbody_init returns EINVAL. */
  int32_t pair_once_block;
} nbody_opts;

/* Launch nbody_step's kernels directly instead of replaying CUDA graphs. */
#define NBODY_FLAG_NO_GRAPH 1
/* Never use the single-launch kernels (one FP64 Verlet system of at most
 * 4,096 bodies runs every step of an nbody_step call in one launch: of an
 * 8- or 16-CTA cluster up to 96 bodies, of a cooperative grid beyond,
 * unless this flag is set). */
#define NBODY_FLAG_NO_SMALL 2
/* Use the force kernel that evaluates every ordered pair (p, j) on its
 * own, instead of the default one that evaluates each pair once and applies
 * it to both bodies (a_p += mu_j |d|^-3 d, a_j -= mu_p |d|^-3 d: Eq. 1 to
 * rounding, 20 FP64 operations per two interactions instead of 32; mixed:
 * 16 FP32 operations per two interactions of a far pair instead of 24).
 * FP64 uses it for contexts that are not row shards, when the systems hold
 * at least 1.5 block pairs per SM (64-body blocks: about 1,200 bodies in one
 * system; below that the other kernel is faster) and the partial sums fit;
 * mixed for systems of at least 65,536 bodies (nbody_opts.pair_once_block). */
#define NBODY_FLAG_NO_SYM 4

/* Work decomposition of the force kernels (see nbody_set_tiles).  The work
 * of a step -- every target block (at most threads * ipt bodies of one
 * system) times the sources of its system -- is laid out as one line.  Three
 * quarters of it are cut into SMs * ctas_per_sm equal static shares, one per
 * CTA; the last quarter into ctas_per_sm * SMs * jsplit small chunks that
 * CTAs pull as they finish (jsplit = 0: all static).  Each piece writes fixed
 * partial-sum rows, added in a fixed order, so results do not depend on the
 * schedule. */
typedef struct {
  int32_t threads;     /* threads per CTA; (threads, ipt) pairs built: FP64 (64|128|256|512, 1),
                        * (128|256, 2); mixed (128|256|512|1024, 1), (256|384|512|768, 2),
                        * (128|256, 4) */
  int32_t ipt;         /* target bodies per thread */
  int32_t tj;          /* source bodies per shared-memory stage: multiple of 64, 64..2048 */
  int32_t jsplit;      /* dynamic chunks per CTA, 0..64 */
  int32_t ctas_per_sm; /* CTAs per SM, >= 1 (capped at what fits) */
} nbody_tiles;

/* Create a context bound to caller-owned state.
 *   out        receives the context (set to NULL on failure).
 *   n_systems  number of independent systems, >= 1.
 *   offsets    HOST array of n_systems+1 int64: 0 = offsets[0] < offsets[1]
 *              < ... ; every system holds at least 1 body; N = offsets[n_systems]
 *              must be < 2^31.
 *   x..vz      DEVICE arrays of N doubles, updated in place by nbody_step.
 *   m          DEVICE array of N doubles (masses, >= 0), read at init and by
 *              nbody_reset; later changes need nbody_reset.
 *   o          options (copied).
 *   cuda_stream a cudaStream_t, or NULL for the legacy default stream (the
 *              context then orders its own private stream after it).
 * Computes a_0 = Eq. 1 at the initial positions and snapshots (r_0, v_0) for
 * nbody_grad.  Synchronous.  EINVAL if any pointer is NULL, sizes or options
 * are out of range, or two bodies of one system share a position. */
nbody_status nbody_init(nbody_ctx **out, int64_t n_systems, const int64_t *offsets,
                        double *x, double *y, double *z, double *vx, double *vy,
                        double *vz, const double *m, const nbody_opts *o,
                        void *cuda_stream);

/* Advance every system by n_steps steps of the context's integrator, in
 * place.  n_steps == 0 is a no-op; n_steps < 0 is EINVAL.  Asynchronous.
 * Velocity Verlet (Eqs. 3, 1, 4): each step is a force launch (Eq. 1) and a
 * per-body Verlet launch (Eqs. 4, 3), chained; leapfrog likewise, with the
 * force at the half-step positions.  RK4: each step is four
 * (force launch, per-body stage launch) pairs; the last evaluation is Eq. 1
 * at the new positions, so the context's acceleration always belongs to the
 * current state.  Consecutive steps are replayed from cached CUDA graphs
 * unless NBODY_FLAG_NO_GRAPH is set or the stream is already being
 * captured.  One FP64 Verlet system of at most 4,096 bodies instead runs
 * all n_steps in a single launch (see NBODY_FLAG_NO_SMALL). */
nbody_status nbody_step(nbody_ctx *ctx, int64_t n_steps);

/* Copy the acceleration at the current positions (Eq. 1, as used by the
 * last step) into DEVICE arrays ax, ay, az of N doubles.  (Leapfrog: Eq. 1
 * at the last half-step positions, the only force it evaluates.)
 * Asynchronous. */
nbody_status nbody_accel(nbody_ctx *ctx, double *ax, double *ay, double *az);

/* Re-read the bound state after the caller changed x..vz or m: recompute
 * a = Eq. 1 at the current positions and re-take the nbody_grad snapshot;
 * mixed precision also re-sorts the sources spatially (nbody_reorder), so
 * the context then computes bitwise what a new one on this state would.
 * Asynchronous (but reads the positions and validates them synchronously,
 * like nbody_init). */
nbody_status nbody_reset(nbody_ctx *ctx);

/* The block size (FP64 bodies, 64 .. 4,096; mixed stage entries, 128 ..
 * 2,048; see nbody_opts.pair_once_block) in *on if the context's force
 * launches evaluate each pair once (see NBODY_FLAG_NO_SYM), else 0.  HOST
 * pointer. */
nbody_status nbody_pair_once(const nbody_ctx *ctx, int32_t *on);

/* Close-encounter handling (nbody_opts.close_omega_dt): the close pairs,
 * clusters, cluster members and the largest sub-step count of the current
 * set (all 0 when off).  Any output pointer may be NULL; HOST memory. */
nbody_status nbody_close_info(const nbody_ctx *ctx, int64_t *n_pairs, int32_t *n_clusters, int32_t *n_members,
                              int32_t *k_max);

/* Mixed precision: re-sort each system's sources into a spatial (Morton)
 * order of the current positions.  nbody_init and nbody_reset sort; the
 * order only decides how many source groups the force kernel finds far from
 * a warp's targets (those take its hi-only path, see NBODY_MIXED) and the
 * order of the sums, never what is summed.  As bodies move, groups spread
 * and fewer are far: call this between steps of a long run.  No-op for FP64
 * contexts.  Synchronous. */
nbody_status nbody_reorder(nbody_ctx *ctx);

/* Total energy of each system at the current state (Sections 2 and 4):
 *   E_s = sum_p (1/2) m_p |v_p|^2 - sum_{p<j} G m_p m_j / |r_j - r_p|,
 * FP64 with compensated, fixed-order (deterministic) reductions.
 * e_host: HOST array of n_systems doubles.  Synchronous. */
nbody_status nbody_energy(nbody_ctx *ctx, double *e_host);

/* Gradient of a loss L(r_T, v_T) through T = n_steps Verlet steps started
 * from the snapshot (r_0, v_0) taken by nbody_init / nbody_reset, by the
 * discrete adjoint of Eqs. 1, 3, 4 (reverse sweep with checkpoints every
 * ckpt_every steps and recomputation in between).  The bound state is not
 * modified.
 *   dL_dr_T  DEVICE, 3N (x|y|z blocks): dL/dr_T.
 *   dL_dv_T  DEVICE, 3N, or NULL for zero.
 *   dL_dr0, dL_dv0  DEVICE, 3N outputs; dL_dm DEVICE, N output.
 * Runs in the context's precision.  Verlet contexts only: EINVAL for RK4
 * and leapfrog.
 * Synchronous. */
nbody_status nbody_grad(nbody_ctx *ctx, int64_t n_steps, const double *dL_dr_T,
                        const double *dL_dv_T, double *dL_dr0, double *dL_dv0,
                        double *dL_dm);

/* Wait for the context's stream and report device-side faults. Synchronous. */
nbody_status nbody_sync(nbody_ctx *ctx);

/* Current work decomposition, and an override (validated; EINVAL if out of
 * range).  Changing tiles drops cached graphs and re-sizes scratch. */
nbody_status nbody_get_tiles(const nbody_ctx *ctx, nbody_tiles *t);
nbody_status nbody_set_tiles(nbody_ctx *ctx, const nbody_tiles *t);

/* Time each candidate decomposition on the bound state for `probe_steps`
 * steps of the general (two-kernel) path, the one tiles shape, then the six
 * fastest again three times each over 4 x probe_steps steps, and keep the
 * one with the best time; a context whose nbody_step runs a single-launch
 * kernel keeps doing so.  (An FP64 context on the pair-once kernel, see
 * NBODY_FLAG_NO_SYM, has no decomposition to choose: its current tiles are
 * timed and kept.)  The bound state is restored afterwards.  best (HOST, may be
 * NULL) receives the winner, best_ms its time per step.  With a tune_cache
 * (nbody_opts) the winner is also written there (replacing the entry with
 * the same key); if that file cannot be written the call returns
 * NBODY_EINVAL after keeping the winner.  Synchronous. */
nbody_status nbody_autotune(nbody_ctx *ctx, int32_t probe_steps, nbody_tiles *best,
                            double *best_ms);

/* Kernel durations of the general path, for roofline accounting (not part of
 * the method).  Advances the bound state by n_steps Verlet steps (Eqs. 3-4)
 * exactly as nbody_step does, but launches each step's two kernels, the
 * Eq. 1 force kernel and the per-body Verlet kernel, unchained and without a
 * graph, each bracketed by CUDA events on the context's stream.  The small
 * single-cluster path is not used.  HOST out[4] receives: [0] mean force
 * kernel duration (ms), [1] mean Verlet kernel duration (ms), [2] mean time
 * per step from the first event to the last (ms), [3] n_steps.
 * n_steps >= 1, else NBODY_EINVAL.  Verlet contexts only: EINVAL for RK4
 * and leapfrog.
 * Synchronous. */
nbody_status nbody_kernel_times(nbody_ctx *ctx, int32_t n_steps, double *out);

/* Largest system nbody_accel_static accepts. */
#define NBODY_STATIC_MAX_BODIES 65536

/* All-pairs gravitational accelerations of ONE system, FP64, without
 * allocating device memory: a deployment variant of the force kernel.
 * Some callers cannot allocate: a host that reserves all device
 * memory at start-up and forbids allocation afterwards (a real-time loop, a
 * service with a fixed memory budget), or a component running while another
 * allocator owns the device memory, where one more cudaMalloc may fail or
 * stall.  This call uses no context and calls no cudaMalloc/cudaFree: its
 * scratch (staged sources, partial sums, work tables, fault flags) lives in one
 * fixed-size __device__ array inside the library, about 3.7 MB, which every
 * GPU that loads the library holds until the process exits.
 *   n        bodies, 1 <= n <= NBODY_STATIC_MAX_BODIES, else NBODY_EINVAL.
 *   G        gravitational constant, > 0.
 *   x, y, z, m   DEVICE arrays of n doubles (positions, masses >= 0).
 *   ax, ay, az   DEVICE arrays of n doubles, written with a_p.
 *   cuda_stream  stream to run on (NULL: legacy default stream).
 * Synchronous: returns after the results are written, so it cannot be
 * captured into a CUDA graph: on a stream that is capturing it returns
 * NBODY_EINVAL before any work.  EINVAL for coincident bodies or non-finite
 * input.  Messages: nbody_last_error(NULL).  The first call on a device looks
 * up the device address of the array (cudaGetSymbolAddress).
 * All calls on a device share the array and it keeps the last call's
 * contents; each call re-stages its inputs and clears its counters, but calls
 * that overlap on the GPU (other streams or host threads) race on the array
 * and must be serialised by the caller.  Results match nbody_init +
 * nbody_accel in FP64 to rounding (the source order of the sum differs). */
nbody_status nbody_accel_static(int64_t n, double G, const double *x, const double *y, const double *z,
                                const double *m, double *ax, double *ay, double *az, void *cuda_stream);

/* Row shards (Section 3's distributed method: each of `world` processes
 * owns a block of bodies, sums Eq. 1 for them over every body, and all
 * exchange the new positions after every step).  Turns a context of ONE
 * system integrated with velocity Verlet into rank `rank` of `world`:
 * every rank binds the same whole state; rank k owns bodies [k C, (k+1) C)
 * (C = ceil(N / world) rounded up to even; the last chunks may be short or
 * empty).  The source buffer becomes `world` chunks of C entries of 32 bytes
 * (rank k's bodies in chunk k, the rest inert padding), and the current
 * positions of all bodies are staged for the first step (the Eq. 3 drift),
 * so every rank starts with the same complete buffer.  Synchronous.  EINVAL
 * for several systems, RK4 or leapfrog, a context that is already a shard,
 * or rank/world out of range.  A shard then steps only with
 * nbody_shard_step; nbody_step, nbody_accel, nbody_reset, nbody_reorder,
 * nbody_energy, nbody_grad, nbody_set_tiles, nbody_autotune and
 * nbody_kernel_times return EINVAL (the bound state of other ranks' bodies
 * is not kept up to date). */
nbody_status nbody_shard(nbody_ctx *ctx, int32_t rank, int32_t world);

/* One Verlet step of this rank's bodies: Eq. 1 for its bodies against every
 * source of the current buffer, Eq. 4 and Eq. 3, and their next positions
 * staged into this rank's chunk of the next buffer.  Before the next
 * nbody_shard_step, every rank's chunk must be copied into every other
 * rank's buffer (an all-gather; see nbody_shard_buffer).  Asynchronous on the
 * context's stream. */
nbody_status nbody_shard_step(nbody_ctx *ctx);

/* The DEVICE buffer the next nbody_shard_step reads: `world` chunks of
 * *chunk_bytes bytes (32 bytes per entry), chunk k starting at byte
 * k * *chunk_bytes.  After nbody_shard_step this rank's chunk is current;
 * an in-place all-gather of the chunks (e.g. ncclAllGather with send buffer
 * = this rank's chunk, receive buffer = the whole buffer), ordered on the
 * context's stream, completes it.  The buffer alternates between two
 * allocations, so ask again after every step. */
nbody_status nbody_shard_buffer(const nbody_ctx *ctx, void **stage, int64_t *chunk_bytes);

/* Release the context and everything it owns.  NULL is a no-op. */
void nbody_free(nbody_ctx *ctx);

/* Message of the last failure on ctx; with ctx == NULL, the last failure of
 * a call that has no context (nbody_init, nbody_accel_static, nbody_peaks)
 * on this thread. */
const char *nbody_last_error(const nbody_ctx *ctx);

/* Peak-rate microbenchmarks on the current device (instruction throughput,
 * not part of the method).  HOST out[8] receives, in units of 1e9
 * lane-operations per second: [0] FP32 FFMA, [1] FP64 DFMA,
 * [2] MUFU rsqrt.approx.f32, [3] rsqrt.approx.f64, [4] cvt f32<->f64,
 * [5] packed f32x2 FFMA (lane count), and [6] the mean SM clock in MHz
 * during the FFMA run, [7] the number of SMs.  Synchronous. */
nbody_status nbody_peaks(double *out);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_H */
