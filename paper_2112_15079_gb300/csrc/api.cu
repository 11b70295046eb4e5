// Host side of the C ABI declared in include/nbody.h: context lifetime,
// validation, scratch ownership, stream-K work tables (planned by
// work_plan.h), the choice between the single-launch kernels (one FP64
// Verlet system of up to 4,096 bodies) and the general two-kernel path,
// CUDA-graph replay of Verlet, leapfrog and RK4 steps, the adjoint sweep,
// energy, tiles/autotuning and device-fault reporting.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "nbody.h"
#include "nbody_internal.h"
#include "close_pairs.h"
#include "tune_cache.h"

// Hash of the kernel sources of this build (set by the build script): the
// tune cache keys its entries with it.
#ifndef NBODY_KERNEL_HASH
#define NBODY_KERNEL_HASH "unknown"
#endif

using nb::Item;

namespace {

thread_local std::string g_init_error;

constexpr int kGraphChunk = 64;  // steps per cached graph (even: stage parity repeats)
constexpr int kSmallClusterMax = 96;  // bodies: the cluster kernel up to here, then the grid kernel

// Stream-K work tables of one kernel family (force or VJP): target blocks,
// segments per piece, the partial-row array and its row count per body.
struct Work {
  nb::Blk *blks = nullptr;
  nb::Seg *segs = nullptr;
  int32_t *seg_off = nullptr;
  uint16_t *nsl = nullptr;  // [N] partial rows of each body
  std::vector<uint16_t> nsl_rank;  // the plan's rows per block position (body order before any reordering)
  std::vector<int64_t> plan_off, plan_soff;  // the target ranges it was planned for (positions, stage entries)
  double *partial = nullptr;
  int32_t *dyn_ctr = nullptr;  // [2] dynamic-chunk counter (self-resetting)
  int n_blks = 0, rows = 0, grid = 0, n_dyn = 0;
  int occ = 0;  // CTAs of the kernel that fit on one SM
  size_t smem = 0;
  int stages = nb::kStages;  // force kernel: ring depth
  // FP64 force kernel with each pair once (sym.cu): block-pair items
  int4 *sym_pairs = nullptr;
  int n_sym = 0;
  int sym_tiles = 0;  // 32-body tiles per block (2: 64-body blocks)
};

// Adjoint workspace, allocated by the first nbody_grad and kept.
struct Adjoint {
  Work vj;                         // VJP work tables
  double *rho = nullptr, *nu = nullptr, *gm = nullptr;  // [3N], [3N], [N]
  void *w = nullptr;               // staged w (stage layout)
  double *shadow = nullptr;        // [9][N]: x, y, z, vx, vy, vz, ax, ay, az of the recomputation
  double *ckpt = nullptr;          // [n_ckpt][6][N]
  int64_t n_ckpt = 0;
  void *store = nullptr;           // [K + 1] staged positions of one segment
  int64_t store_len = 0;
};

}  // namespace

namespace nb {
void set_last_error(const char *msg) { g_init_error = msg; }
}  // namespace nb

// A widened box (the force kernel's far test widens the hi-part box by
// kFarKappa times the largest lo part); empty: no real body inside.
struct PlanBox {
  float lo[3], hi[3];
  bool empty;
};

struct nbody_ctx {
  int dev = 0, nsm = 0;
  int64_t n_sys = 0;
  std::vector<int64_t> offsets;
  int32_t N = 0;
  double *x = nullptr, *y = nullptr, *z = nullptr, *vx = nullptr, *vy = nullptr, *vz = nullptr;
  const double *m = nullptr;
  nbody_opts o{};
  std::string tune_cache;  // copy of o.tune_cache ("" = off)
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;  // where work runs (user stream, or private when user passed NULL)
  bool own_stream = false;
  cudaStream_t cap_stream = nullptr;  // graph capture only
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;

  // scratch
  std::vector<void *> allocs;
  int alloc_seq = 0;  // device allocations made so far (fault injection counts these)
  int64_t wait_seq = 0;      // launches with a stallable bounded wait (adjoint products, single-launch steps)
  int64_t stall_at = 0;      // test hook (NBODY_INJECT_WAIT_STALL=k): the k-th of them stalls
  double *a = nullptr;               // [3][N] acceleration at the current positions
  void *stage[2] = {nullptr, nullptr};  // ping-pong staged sources (layout per precision)
  int64_t n_stage = 0;               // stage entries (mixed: systems padded to even length)
  std::vector<int64_t> soff;         // stage offset of each system
  int32_t *qidx = nullptr;           // [N] stage index of each body (mixed)
  int32_t *perm = nullptr;           // [n_stage] body of each stage entry (mixed; padding: any body)
  float4 *boxes = nullptr;           // mixed: [n_stage / 64 rounded up][2] source-group boxes of the next force launch
  std::vector<int32_t> qidx_h;       // host copy of qidx (mixed)
  // mixed, for planning (see chunk_costs): per stage entry its hi parts and
  // the magnitudes of its lo parts ([n_stage][6]); per source group of
  // 2 kBoxPairs entries its widened box
  std::vector<float> ent;
  std::vector<PlanBox> gbox;
  // Targets and sources of the force launches: system s's targets are the
  // block positions [tgt_off[s], tgt_off[s+1]) at stage entries from
  // tgt_soff[s]; its sources are the stage entries [src_b[s], src_b[s] +
  // src_n[s]).  Unsharded: the systems themselves.
  std::vector<int64_t> tgt_off, tgt_soff, src_b, src_n;
  // Row shard (nbody_shard): this rank completes bodies [sh_begin, sh_end);
  // the stage holds sh_world chunks of sh_chunk entries (rank k's bodies at
  // entries [k sh_chunk, ...), then inert padding).
  int32_t sh_world = 0, sh_rank = 0;
  // Close-encounter handling (nbody_opts.close_omega_dt > 0): the clusters
  // of close pairs (host copy and device tables), and per member a_near and
  // the sub-cycle velocity ([3][members]).
  bool close_on = false;
  nb::CloseSet close;
  std::vector<int32_t> fc_mem, fc_j0, fc_j1, mch_off;  // the members' far-force chunks (CloseArgs)
  int32_t *close_tab = nullptr;
  double *close_an = nullptr, *close_vh = nullptr, *close_far = nullptr;
  int64_t sh_chunk = 0, sh_begin = 0, sh_end = 0;
  int sh_cur = 0;  // the stage the next shard step reads
  double *R = nullptr;               // [3][N] mixed: FP64 positions of the staged step
  double *rk = nullptr;              // RK4: [3][3N] stage velocity V, sums AR and AV
  double *snap = nullptr;            // [6][N] r0, v0 for nbody_grad
  unsigned *flags = nullptr;
  int64_t *offsets_dev = nullptr;
  double *e_body = nullptr;          // [2][N]
  double *e_out = nullptr;           // [2][n_sys]
  Item *eitems = nullptr;
  int n_eitems = 0;

  // tile-dependent scratch (stream-K work tables of the force kernel)
  nbody_tiles tiles{};
  Work fw;
  Adjoint adj;

  bool small = false;  // the single-launch cluster kernel serves nbody_step
  bool grid = false;   // the single-launch cooperative grid kernel serves nbody_step
  int grid_warps = 0, grid_ctas = 0;
  double *xg = nullptr;      // grid kernel: [2][3][N] position exchange
  unsigned *gbar = nullptr;  // grid kernel: barrier arrivals
  std::map<int, cudaGraphExec_t> graphs;
  std::string err;
};

namespace {

nbody_status fail(nbody_ctx *c, nbody_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c)
    c->err = buf;
  else
    g_init_error = buf;
  return st;
}

#define NB_CUDA(c, call)                                                                               \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) return fail((c), NBODY_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Optional host-side fault injection for tests: NBODY_INJECT_ALLOC_FAIL=k
// makes the k-th device allocation of a context fail with NBODY_ENOMEM.
nbody_status dalloc(nbody_ctx *c, void **p, size_t bytes) {
  *p = nullptr;
  const int seq = ++c->alloc_seq;
  if (const char *inj = std::getenv("NBODY_INJECT_ALLOC_FAIL")) {
    if (std::atoi(inj) == seq) return fail(c, NBODY_ENOMEM, "injected allocation failure (allocation %d)", seq);
  }
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(c, NBODY_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  c->allocs.push_back(*p);
  return NBODY_OK;
}

void dfree(nbody_ctx *c, void *p) {
  if (!p) return;
  cudaFree(p);
  c->allocs.erase(std::remove(c->allocs.begin(), c->allocs.end(), p), c->allocs.end());
}

void drop_graphs(nbody_ctx *c) {
  for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
}

// Ordering with the caller's stream when the work runs on a private stream.
nbody_status begin_work(nbody_ctx *c) {
  if (c->own_stream) {
    NB_CUDA(c, cudaEventRecord(c->ev_in, c->user_stream));
    NB_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_in, 0));
  }
  return NBODY_OK;
}
nbody_status end_work(nbody_ctx *c) {
  if (c->own_stream) {
    NB_CUDA(c, cudaEventRecord(c->ev_out, c->stream));
    NB_CUDA(c, cudaStreamWaitEvent(c->user_stream, c->ev_out, 0));
  }
  return NBODY_OK;
}

bool tiles_valid(const nbody_tiles &t, int precision) {
  return nb::force_config_supported(precision, t.threads, t.ipt) && t.tj >= 64 && t.tj <= 2048 &&
         t.tj % 64 == 0 && t.jsplit >= 0 && t.jsplit <= 64 && t.ctas_per_sm >= 1 && t.ctas_per_sm <= 32;
}

nb::TuneKey tune_key(const nbody_ctx *c) {
  nb::TuneKey k;
  k.precision = c->o.precision;
  k.integrator = c->o.integrator;
  k.n_log2 = nb::floor_log2(c->N);
  k.systems_log2 = nb::floor_log2(c->n_sys);
  k.sms = c->nsm;
  k.kernels = NBODY_KERNEL_HASH;
  return k;
}

nbody_tiles default_tiles(const nbody_ctx *c) {
  // The autotuner's picks on GB300: FP64 is bound by the FP64 pipe (~90% busy)
  // with three 128-thread CTAs per SM at every size; the mixed path takes two
  // 512-thread CTAs per SM with one target per thread up to ~32k bodies (short
  // shares, more warps), and beyond one 512-thread CTA per SM with two
  // targets per thread and dynamic chunks: the shares are planned by the
  // host's far/near cost estimate, but run-time differences between SMs
  // remain (65,536 bodies: 1.81 ms with 8 chunks per CTA against 1.92 ms
  // with static shares only; 262,144: 27.3 ms with 16 against 27.7 with 8).
  nbody_tiles t{};
  t.jsplit = 0;  // static shares only (dynamic chunks add partial rows)
  t.tj = 1024;
  if (c->o.precision == NBODY_FP64) {
    t.threads = 128;
    t.ipt = 1;
    t.ctas_per_sm = 3;
  } else if (c->N <= 32768) {
    t.threads = 512;
    t.ipt = 1;
    t.ctas_per_sm = 2;
  } else {
    t.threads = 512;
    t.ipt = 2;
    t.ctas_per_sm = 1;
    t.jsplit = c->N <= 131072 ? 8 : 16;
  }
  return t;
}

void free_work(nbody_ctx *c, Work &w);

// Rows per BODY from the plan's rows per block position: position r of
// system s is stage entry soff[s] + (r - offsets[s]), which holds body
// perm[...] -- so body p takes the rows of position offsets[s] + (qidx[p] -
// soff[s]).  Without a reordered stage (FP64) the two coincide.
nbody_status upload_nsl(nbody_ctx *c, Work &wk) {
  if (!wk.nsl) return NBODY_OK;
  std::vector<uint16_t> body(static_cast<size_t>(c->N), 0);  // bodies outside the plan's targets: 0 rows
  const size_t n_sys = wk.plan_soff.size();
  for (size_t s = 0; s < n_sys; ++s) {
    const int64_t q0 = wk.plan_soff[s], n = wk.plan_off[s + 1] - wk.plan_off[s];
    for (int64_t r = 0; r < n; ++r) {
      const int64_t q = q0 + r;  // stage entry of block position plan_off[s] + r
      const int64_t p = c->qidx_h.empty() ? q : -1;
      if (p >= 0) body[p] = wk.nsl_rank[wk.plan_off[s] + r];
    }
  }
  if (!c->qidx_h.empty()) {  // reordered stage: body p sits at entry qidx[p]
    std::vector<int64_t> pos_of_entry(static_cast<size_t>(c->n_stage), -1);
    for (size_t s = 0; s < n_sys; ++s)
      for (int64_t r = 0; r < wk.plan_off[s + 1] - wk.plan_off[s]; ++r)
        pos_of_entry[wk.plan_soff[s] + r] = wk.plan_off[s] + r;
    for (int32_t p = 0; p < c->N; ++p) {
      const int64_t r = pos_of_entry[c->qidx_h[p]];
      if (r >= 0) body[p] = wk.nsl_rank[r];
    }
  }
  NB_CUDA(c, cudaMemcpy(wk.nsl, body.data(), sizeof(uint16_t) * body.size(), cudaMemcpyHostToDevice));
  return NBODY_OK;
}

nb::ChunkCost chunk_costs(const nbody_ctx *c, const nbody_tiles &t);

// Build stream-K work tables (the plan is work_plan.h's) and upload them.
// row_doubles: 8-byte words per body and partial row (3 force, 4 VJP).
nbody_status build_work(nbody_ctx *c, Work &wk, const nbody_tiles &t, int occ, int row_doubles) {
  free_work(c, wk);
  if (occ < 1) return fail(c, NBODY_EINVAL, "tiles do not fit on an SM (threads %d, ipt %d, tj %d)", t.threads, t.ipt, t.tj);
  const int64_t cps = std::min<int64_t>(t.ctas_per_sm, occ);
  nb::WorkPlan plan;
  const bool own_src = c->src_b.empty();
  // the mixed force kernel's pairs cost 12 or 18 operations (far or near
  // groups): its shares are cut by cost
  const bool by_cost = row_doubles == 3 && !c->gbox.empty();
  const nb::ChunkCost cost = by_cost ? chunk_costs(c, t) : nb::ChunkCost{};
  const std::string why = nb::plan_work(c->tgt_off, c->tgt_soff, c->o.precision == NBODY_MIXED, t.threads, t.ipt,
                                        t.jsplit, static_cast<int64_t>(c->nsm) * cps, plan,
                                        own_src ? nullptr : &c->src_b, own_src ? nullptr : &c->src_n,
                                        by_cost ? &cost : nullptr);
  if (!why.empty()) return fail(c, NBODY_EINVAL, "%s", why.c_str());
  wk.plan_off = c->tgt_off;
  wk.plan_soff = c->tgt_soff;
  const std::vector<nb::Blk> &blks = plan.blks;
  const std::vector<nb::Seg> &segs = plan.segs;
  const std::vector<int32_t> &seg_off = plan.seg_off;
  const std::vector<uint16_t> &nsl = plan.nsl;
  const int rows = plan.rows;
  const int64_t G = plan.grid, D = plan.n_dyn;
  wk.nsl_rank = nsl;
  wk.n_dyn = static_cast<int>(D);
  wk.n_blks = static_cast<int>(blks.size());
  wk.rows = rows;
  wk.grid = static_cast<int>(G);
  wk.occ = occ;
  auto upload = [&]() -> nbody_status {
    nbody_status st;
    if ((st = dalloc(c, reinterpret_cast<void **>(&wk.blks), sizeof(nb::Blk) * blks.size())) != NBODY_OK) return st;
    if ((st = dalloc(c, reinterpret_cast<void **>(&wk.segs), sizeof(nb::Seg) * segs.size())) != NBODY_OK) return st;
    if ((st = dalloc(c, reinterpret_cast<void **>(&wk.seg_off), sizeof(int32_t) * seg_off.size())) != NBODY_OK)
      return st;
    if ((st = dalloc(c, reinterpret_cast<void **>(&wk.nsl), sizeof(uint16_t) * static_cast<size_t>(c->N))) != NBODY_OK)
      return st;
    if ((st = dalloc(c, reinterpret_cast<void **>(&wk.dyn_ctr), sizeof(int32_t) * 2)) != NBODY_OK) return st;
    if ((st = dalloc(c, reinterpret_cast<void **>(&wk.partial),
                     sizeof(double) * row_doubles * static_cast<size_t>(rows) * c->N)) != NBODY_OK)
      return st;
    NB_CUDA(c, cudaMemset(wk.dyn_ctr, 0, sizeof(int32_t) * 2));
    // (nsl: one entry per body, those outside the planned targets 0)
    NB_CUDA(c, cudaMemcpy(wk.blks, blks.data(), sizeof(nb::Blk) * blks.size(), cudaMemcpyHostToDevice));
    NB_CUDA(c, cudaMemcpy(wk.segs, segs.data(), sizeof(nb::Seg) * segs.size(), cudaMemcpyHostToDevice));
    NB_CUDA(c, cudaMemcpy(wk.seg_off, seg_off.data(), sizeof(int32_t) * seg_off.size(), cudaMemcpyHostToDevice));
    return upload_nsl(c, wk);
  };
  const nbody_status st = upload();
  if (st != NBODY_OK) free_work(c, wk);  // all or nothing: no half-built tables
  return st;
}

// Block size of the pair-once force kernels for this context
// (pair_once_plan.h), or 0 where the every-ordered-pair kernel runs: row
// shards, NBODY_FLAG_NO_SYM, and the cases pair_once_block turns down.
int sym_block(const nbody_ctx *c) {
  if (c->sh_world > 0 || (c->o.flags & NBODY_FLAG_NO_SYM)) return 0;
  std::vector<int64_t> sizes(static_cast<size_t>(c->n_sys));
  for (int64_t s = 0; s < c->n_sys; ++s) sizes[s] = c->offsets[s + 1] - c->offsets[s];
  return nb::pair_once_block(sizes, c->o.precision == NBODY_MIXED, c->nsm, c->o.pair_once_block);
}

// Work tables of the pair-once kernels: the block pairs (I, J), I <= J, of
// every system, off-diagonal items first, blocks of B bodies (FP64: 64, or
// wide: force only) or stage entries (mixed, force only); each body has one
// partial row per block of its system (row_doubles values each: 3 force,
// 4 VJP).  An item is (first stage entry of the system, its bodies, I, J).
nbody_status build_sym_work(nbody_ctx *c, Work &wk, int row_doubles, int B) {
  free_work(c, wk);
  if (B != nb::kSymBlock && row_doubles != 3) return fail(c, NBODY_EINVAL, "wide pair-once blocks are force-only");
  const bool mixed = c->o.precision == NBODY_MIXED;
  std::vector<int4> off_diag, diag;
  int64_t rows = 1;
  std::vector<uint16_t> nsl(static_cast<size_t>(c->N), 0);
  for (int64_t s = 0; s < c->n_sys; ++s) {
    const int64_t b = c->offsets[s], ns = c->offsets[s + 1] - b;
    const int nb = static_cast<int>((ns + B - 1) / B);
    rows = std::max<int64_t>(rows, nb);
    for (int64_t p = b; p < b + ns; ++p) nsl[p] = static_cast<uint16_t>(nb);
    for (int I = 0; I < nb; ++I)
      for (int J = I; J < nb; ++J)
        (I == J ? diag : off_diag).push_back(make_int4(static_cast<int>(c->soff[s]), static_cast<int>(ns), I, J));
  }
  std::vector<int4> pairs = std::move(off_diag);
  pairs.insert(pairs.end(), diag.begin(), diag.end());
  if (rows > 65535 || pairs.size() > static_cast<size_t>(INT32_MAX))
    return fail(c, NBODY_EINVAL, "too many pair-once blocks (%lld in a system)", static_cast<long long>(rows));
  const int occ = mixed ? nb::force_msym_ctas_per_sm(B / 32, B / 128) : nb::force_sym_ctas_per_sm(B / 32);
  if (occ < 1) return fail(c, NBODY_ECUDA, "the pair-once FP64 kernel does not fit on an SM");
  wk.nsl_rank = nsl;
  wk.plan_off = c->tgt_off;
  wk.plan_soff = c->tgt_soff;
  wk.n_sym = static_cast<int>(pairs.size());
  wk.sym_tiles = B / 32;
  wk.rows = static_cast<int>(rows);
  wk.grid = static_cast<int>(std::min<int64_t>(pairs.size(), static_cast<int64_t>(c->nsm) * occ));
  wk.occ = occ;
  wk.n_dyn = 0;
  auto upload = [&]() -> nbody_status {
    nbody_status st;
    if ((st = dalloc(c, reinterpret_cast<void **>(&wk.sym_pairs), sizeof(int4) * pairs.size())) != NBODY_OK) return st;
    if ((st = dalloc(c, reinterpret_cast<void **>(&wk.nsl), sizeof(uint16_t) * static_cast<size_t>(c->N))) != NBODY_OK)
      return st;
    if ((st = dalloc(c, reinterpret_cast<void **>(&wk.dyn_ctr), sizeof(int32_t) * 2)) != NBODY_OK) return st;
    if ((st = dalloc(c, reinterpret_cast<void **>(&wk.partial),
                     sizeof(double) * row_doubles * static_cast<size_t>(rows) * c->N)) != NBODY_OK)
      return st;
    NB_CUDA(c, cudaMemset(wk.dyn_ctr, 0, sizeof(int32_t) * 2));
    NB_CUDA(c, cudaMemcpy(wk.sym_pairs, pairs.data(), sizeof(int4) * pairs.size(), cudaMemcpyHostToDevice));
    return upload_nsl(c, wk);
  };
  const nbody_status st = upload();
  if (st != NBODY_OK) free_work(c, wk);
  return st;
}

void free_work(nbody_ctx *c, Work &w) {
  dfree(c, w.sym_pairs);
  w.sym_pairs = nullptr;
  w.n_sym = 0;
  dfree(c, w.blks);
  dfree(c, w.segs);
  dfree(c, w.seg_off);
  dfree(c, w.nsl);
  dfree(c, w.partial);
  dfree(c, w.dyn_ctr);
  w = Work{};
}

// Build the force kernel's tables for tiles t and make t current.  The new
// tables are built aside: on failure the context keeps its previous tiles
// and tables, which stay a matching pair.
nbody_status build_items(nbody_ctx *c, const nbody_tiles &t) {
  drop_graphs(c);
  if (const int B = sym_block(c)) {  // the tiles stay the context's, for nbody_get_tiles; this kernel has none
    Work nw;
    const nbody_status st = build_sym_work(c, nw, 3, B);
    if (st != NBODY_OK) return st;
    free_work(c, c->fw);
    c->fw = nw;
    c->tiles = t;
    return NBODY_OK;
  }
  // The deepest ring (kMaxStages down to kStages tiles) at which the CTAs
  // per SM the tiles ask for still fit: a deeper ring lets the warps of a
  // CTA drift further apart and the next segment's tiles load earlier.
  // A ring above the per-CTA shared-memory limit is refused by the runtime
  // (invalid argument): the next shallower one is tried.
  int stages = nb::kStages, occ = 0;
  size_t smem = 0;
  for (int k = nb::kMaxStages; k >= nb::kStages; --k) {
    smem = nb::force_smem_bytes(c->o.precision, t.tj, k);
    if (k > nb::kStages && nb::force_set_smem(c->o.precision, t.threads, t.ipt, smem) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (k == nb::kStages) NB_CUDA(c, nb::force_set_smem(c->o.precision, t.threads, t.ipt, smem));
    occ = nb::force_max_ctas_per_sm(c->o.precision, t.threads, t.ipt, smem);
    stages = k;
    if (occ >= t.ctas_per_sm) break;
  }
  Work nw;
  const nbody_status st = build_work(c, nw, t, occ, 3);
  if (st != NBODY_OK) return st;  // (the shared-memory limit was only raised)
  nw.smem = smem;
  nw.stages = stages;
  free_work(c, c->fw);
  c->fw = nw;
  c->tiles = t;
  return NBODY_OK;
}

// Pointers of one state (the bound caller state, or the adjoint's shadow).
struct State {
  double *x, *y, *z, *vx, *vy, *vz, *ax, *ay, *az;
};

State bound_state(nbody_ctx *c) {
  const size_t N = c->N;
  return {c->x, c->y, c->z, c->vx, c->vy, c->vz, c->a, c->a + N, c->a + 2 * N};
}

nb::PrepArgs prep_args(nbody_ctx *c, const State &s, int drift, int check, void *stage = nullptr) {
  const size_t N = c->N;
  nb::PrepArgs p{};
  p.x = s.x; p.y = s.y; p.z = s.z; p.vx = s.vx; p.vy = s.vy; p.vz = s.vz;
  p.ax = s.ax; p.ay = s.ay; p.az = s.az;
  p.m = c->m;
  p.stage = stage ? stage : c->stage[0];
  p.qidx = c->qidx;
  p.Rx = c->R;
  p.Ry = c->R ? c->R + N : nullptr;
  p.Rz = c->R ? c->R + 2 * N : nullptr;
  p.flags = c->flags;
  p.N = c->N;
  p.drift = drift;
  p.check = check;
  p.G = c->o.G;
  p.dt = c->o.dt;
  p.half_dt2 = 0.5 * c->o.dt * c->o.dt;
  return p;
}

int n_clusters(const nbody_ctx *c) { return static_cast<int>(c->close.cl_k.size()); }

// Arguments of the cluster kernel writing the stage `nxt`; complete: first
// finish the step the Verlet kernel just closed.
nb::CloseArgs close_args(nbody_ctx *c, const State &s, void *nxt, int complete) {
  const size_t N = c->N;
  const nb::CloseSet &cs = c->close;
  nb::CloseArgs a{};
  a.x = s.x; a.y = s.y; a.z = s.z; a.vx = s.vx; a.vy = s.vy; a.vz = s.vz;
  a.m = c->m;
  a.an = c->close_an;
  a.vh = c->close_vh;
  a.far_part = c->close_far;
  // close_tab: cl_off, cl_k, mem_body, pr_off, pr_a, pr_b, mp_off, mp_pair, fc_mem, fc_j0, fc_j1, mch_off
  int32_t *t = c->close_tab;
  a.cl_off = t;
  a.cl_k = (t += cs.cl_off.size());
  a.mem_body = (t += cs.cl_k.size());
  a.pr_off = (t += cs.mem_body.size());
  a.pr_a = (t += cs.pr_off.size());
  a.pr_b = (t += cs.pr_a.size());
  a.mp_off = (t += cs.pr_b.size());
  a.mp_pair = (t += cs.mp_off.size());
  a.fc_mem = (t += cs.mp_pair.size());
  a.fc_j0 = (t += c->fc_mem.size());
  a.fc_j1 = (t += c->fc_j0.size());
  a.mch_off = (t += c->fc_j1.size());
  a.n_chunks = static_cast<int32_t>(c->fc_mem.size());
  a.stage = nxt;
  a.qidx = c->qidx;
  a.Rx = c->R;
  a.Ry = c->R ? c->R + N : nullptr;
  a.Rz = c->R ? c->R + 2 * N : nullptr;
  a.flags = c->flags;
  a.n_mem = static_cast<int32_t>(cs.mem_body.size());
  a.complete = complete;
  a.precision = c->o.precision;
  a.G = c->o.G;
  a.dt = c->o.dt;
  a.half_dt = 0.5 * c->o.dt;
  return a;
}

// The close pairs and clusters of the bound positions (close_pairs.h), on
// the host, and their device tables.  Synchronous.
nbody_status build_close(nbody_ctx *c) {
  const size_t N = c->N, b = sizeof(double) * N;
  std::vector<double> h(4 * N);
  NB_CUDA(c, cudaMemcpyAsync(h.data(), c->x, b, cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(c, cudaMemcpyAsync(h.data() + N, c->y, b, cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(c, cudaMemcpyAsync(h.data() + 2 * N, c->z, b, cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(c, cudaMemcpyAsync(h.data() + 3 * N, c->m, b, cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  nb::CloseSet cs;
  const std::string why = nb::find_close_set(c->n_sys, c->offsets.data(), h.data(), h.data() + N, h.data() + 2 * N,
                                             h.data() + 3 * N, c->o.G, c->o.dt, c->o.close_omega_dt,
                                             c->o.substep_omega_dt, cs);
  if (!why.empty()) return fail(c, NBODY_EINVAL, "%s", why.c_str());
  for (size_t k = 0; k + 1 < cs.cl_off.size(); ++k) {
    if (cs.cl_off[k + 1] - cs.cl_off[k] > nb::kCloseThreads || cs.pr_off[k + 1] - cs.pr_off[k] > nb::kCloseMaxPairs)
      return fail(c, NBODY_EINVAL, "a cluster of close pairs has more than %d bodies or %d pairs", nb::kCloseThreads,
                  nb::kCloseMaxPairs);
  }
  const size_t nm = cs.mem_body.size();
  for (size_t i = 0; i < nm; ++i)
    if (cs.mp_off[i + 1] - cs.mp_off[i] > nb::kFarPartners)
      return fail(c, NBODY_EINVAL, "a body has more than %d close partners", nb::kFarPartners);
  // far-force chunks: each member's system in kFarChunk sources
  std::vector<int32_t> fc_mem, fc_j0, fc_j1, mch_off{0};
  for (size_t i = 0; i < nm; ++i) {
    const int64_t p = cs.mem_body[i];
    const int64_t sys = std::upper_bound(c->offsets.begin(), c->offsets.end(), p) - c->offsets.begin() - 1;
    for (int64_t j = c->offsets[sys]; j < c->offsets[sys + 1]; j += nb::kFarChunk) {
      fc_mem.push_back(static_cast<int32_t>(i));
      fc_j0.push_back(static_cast<int32_t>(j));
      fc_j1.push_back(static_cast<int32_t>(std::min<int64_t>(j + nb::kFarChunk, c->offsets[sys + 1])));
    }
    mch_off.push_back(static_cast<int32_t>(fc_mem.size()));
  }
  dfree(c, c->close_tab);
  dfree(c, c->close_an);
  dfree(c, c->close_vh);
  dfree(c, c->close_far);
  c->close_tab = nullptr;
  c->close_an = c->close_vh = c->close_far = nullptr;
  std::vector<int32_t> tab;
  for (const std::vector<int32_t> *v : {&cs.cl_off, &cs.cl_k, &cs.mem_body, &cs.pr_off, &cs.pr_a, &cs.pr_b,
                                        &cs.mp_off, &cs.mp_pair, &fc_mem, &fc_j0, &fc_j1, &mch_off})
    tab.insert(tab.end(), v->begin(), v->end());
  nbody_status st;
  if ((st = dalloc(c, reinterpret_cast<void **>(&c->close_tab), sizeof(int32_t) * tab.size())) != NBODY_OK ||
      (st = dalloc(c, reinterpret_cast<void **>(&c->close_an), sizeof(double) * 3 * nm)) != NBODY_OK ||
      (st = dalloc(c, reinterpret_cast<void **>(&c->close_vh), sizeof(double) * 3 * nm)) != NBODY_OK ||
      (st = dalloc(c, reinterpret_cast<void **>(&c->close_far), sizeof(double) * 3 * fc_mem.size())) != NBODY_OK)
    return st;
  c->fc_mem = std::move(fc_mem);
  c->fc_j0 = std::move(fc_j0);
  c->fc_j1 = std::move(fc_j1);
  c->mch_off = std::move(mch_off);
  NB_CUDA(c, cudaMemcpy(c->close_tab, tab.data(), sizeof(int32_t) * tab.size(), cudaMemcpyHostToDevice));
  c->close = std::move(cs);
  drop_graphs(c);  // graphs hold the previous tables' launches
  return NBODY_OK;
}

nb::ForceArgs force_args(nbody_ctx *c, const void *cur) {
  nb::ForceArgs a{};
  a.cur = cur;
  a.partial = c->fw.partial;
  a.perm = c->perm;
  a.boxes = c->boxes;
  a.flags = c->flags;
  a.blks = c->fw.blks;
  a.segs = c->fw.segs;
  a.seg_off = c->fw.seg_off;
  a.dyn_ctr = c->fw.dyn_ctr;
  a.n_dyn = c->fw.n_dyn;
  a.N = c->N;
  a.tj = c->tiles.tj;
  a.stages = c->fw.stages;
  return a;
}

nb::VerletArgs verlet_args(nbody_ctx *c, const State &s, const void *cur, void *nxt, int mode) {
  const size_t N = c->N;
  nb::VerletArgs a{};
  a.x = s.x; a.y = s.y; a.z = s.z; a.vx = s.vx; a.vy = s.vy; a.vz = s.vz;
  a.ax = s.ax; a.ay = s.ay; a.az = s.az;
  a.cur = cur;
  a.nxt = nxt;
  a.Rx = c->R;
  a.Ry = c->R ? c->R + N : nullptr;
  a.Rz = c->R ? c->R + 2 * N : nullptr;
  a.partial = c->fw.partial;
  a.nsl = c->fw.nsl;
  a.qidx = c->qidx;
  a.flags = c->flags;
  a.N = c->N;
  a.p_begin = c->sh_world > 0 ? static_cast<int32_t>(c->sh_begin) : 0;  // a row shard completes its own bodies
  a.p_end = c->sh_world > 0 ? static_cast<int32_t>(c->sh_end) : c->N;
  a.mode = mode;
  a.release_early = c->fw.occ == 1 ? 1 : 0;
  a.dt = c->o.dt;
  a.half_dt = 0.5 * c->o.dt;
  a.half_dt2 = 0.5 * c->o.dt * c->o.dt;
  return a;
}

nb::RkArgs rk_args(nbody_ctx *c, const State &s, const void *cur, void *nxt, int stage) {
  const size_t N = c->N;
  nb::RkArgs a{};
  a.x = s.x; a.y = s.y; a.z = s.z; a.vx = s.vx; a.vy = s.vy; a.vz = s.vz;
  a.ax = s.ax; a.ay = s.ay; a.az = s.az;
  a.m = c->m;
  a.V = c->rk;
  a.AR = c->rk + 3 * N;
  a.AV = c->rk + 6 * N;
  a.cur = cur;
  a.nxt = nxt;
  a.partial = c->fw.partial;
  a.nsl = c->fw.nsl;
  a.qidx = c->qidx;
  a.flags = c->flags;
  a.N = c->N;
  a.stage = stage;
  a.release_early = c->fw.occ == 1 ? 1 : 0;
  a.G = c->o.G;
  a.dt = c->o.dt;
  return a;
}

// The force launch of one step from the staged sources `cur`.
nbody_status launch_force_kernel(nbody_ctx *c, const void *cur, cudaStream_t st, bool chained) {
  if (c->fw.sym_pairs) {
    nb::SymArgs a{};
    a.cur = static_cast<const double4_32a *>(cur);
    a.partial = c->fw.partial;
    a.pairs = c->fw.sym_pairs;
    a.n_pairs = c->fw.n_sym;
    a.ctr = c->fw.dyn_ctr;
    a.N = c->N;
    a.tiles = c->fw.sym_tiles;
    if (c->o.precision == NBODY_MIXED) {
      nb::MsymArgs m{};
      m.cur = static_cast<const float *>(cur);
      m.boxes = c->boxes;
      m.partial = c->fw.partial;
      m.pairs = c->fw.sym_pairs;
      m.perm = c->perm;
      m.n_pairs = c->fw.n_sym;
      m.ctr = c->fw.dyn_ctr;
      m.N = static_cast<int32_t>(c->N);
      m.tiles = c->fw.sym_tiles;
      m.warps = c->fw.sym_tiles / 4;
      NB_CUDA(c, nb::launch_force_msym(m, c->fw.grid, st, chained));
      return NBODY_OK;
    }
    NB_CUDA(c, nb::launch_force_sym(a, c->fw.grid, st, chained));
    return NBODY_OK;
  }
  NB_CUDA(c, nb::launch_force(c->o.precision, c->tiles.threads, c->tiles.ipt, c->fw.grid, c->fw.smem,
                              force_args(c, cur), st, chained));
  return NBODY_OK;
}

// One Verlet step (or, kModeForce, only a = Eq. 1) from the staged sources
// `cur`, staging the next positions into `nxt`: the force kernel, then the
// per-body Verlet kernel, chained.
// With `ev` (three events) the kernels run unchained, bracketed by ev[0],
// ev[1] and ev[2], so that each one's duration can be read alone.
nbody_status launch_one_step(nbody_ctx *c, const State &s, const void *cur, void *nxt, int mode, cudaStream_t st,
                             const cudaEvent_t *ev = nullptr) {
  const bool chained = ev == nullptr;
  if (c->o.precision == NBODY_MIXED) NB_CUDA(c, nb::launch_boxes(cur, c->n_stage / 2, c->boxes, st, chained));
  if (ev) NB_CUDA(c, cudaEventRecord(ev[0], st));
  nbody_status fs;
  if ((fs = launch_force_kernel(c, cur, st, chained)) != NBODY_OK) return fs;
  if (ev) NB_CUDA(c, cudaEventRecord(ev[1], st));
  NB_CUDA(c, nb::launch_verlet(c->o.precision, verlet_args(c, s, cur, nxt, mode), st, chained));
  if (ev) NB_CUDA(c, cudaEventRecord(ev[2], st));
  return NBODY_OK;
}

// One RK4 step from stage 1 (staged r_2, V = v_2, AR, AV set): four (force,
// stage-completion) pairs, s = 2..5, ping-ponging between the two stages
// (an even count, so every step starts from stage[0]).
nbody_status launch_rk4_step(nbody_ctx *c, const State &s, cudaStream_t st) {
  for (int k = 0; k < 4; ++k) {
    const void *cur = c->stage[k & 1];
    void *nxt = c->stage[1 - (k & 1)];
    if (c->o.precision == NBODY_MIXED) NB_CUDA(c, nb::launch_boxes(cur, c->n_stage / 2, c->boxes, st, true));
    nbody_status fs;
    if ((fs = launch_force_kernel(c, cur, st, true)) != NBODY_OK) return fs;
    NB_CUDA(c, nb::launch_rk_stage(c->o.precision, rk_args(c, s, cur, nxt, 2 + k), st, true));
  }
  return NBODY_OK;
}

nbody_status launch_steps(nbody_ctx *c, const State &s, int n, cudaStream_t st) {
  for (int i = 0; i < n; ++i) {
    nbody_status r =
        c->o.integrator == NBODY_RK4
            ? launch_rk4_step(c, s, st)
            : launch_one_step(c, s, c->stage[i & 1], c->stage[1 - (i & 1)],
                              c->o.integrator == NBODY_LEAPFROG ? nb::kModeLeapfrog : nb::kModeStep, st);
    if (r != NBODY_OK) return r;
    // close pairs: finish this step for the cluster members and sub-cycle
    // them into the next stage
    if (c->close_on) {
      const nb::CloseArgs ca = close_args(c, s, c->stage[1 - (i & 1)], 1);
      NB_CUDA(c, nb::launch_close_far(ca, st, true));
      NB_CUDA(c, nb::launch_close(ca, n_clusters(c), st, true));
    }
  }
  return NBODY_OK;
}

nbody_status graph_for(nbody_ctx *c, int n, cudaGraphExec_t *out) {
  auto f = c->graphs.find(n);
  if (f != c->graphs.end()) {
    *out = f->second;
    return NBODY_OK;
  }
  NB_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  nbody_status st = launch_steps(c, bound_state(c), n, c->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (st != NBODY_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(c, NBODY_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(c, NBODY_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  c->graphs[n] = ex;
  *out = ex;
  return NBODY_OK;
}

// Force-only launch: a = Eq. 1 at the positions staged in stage[0].
nbody_status launch_force(nbody_ctx *c, const State &s) {
  return launch_one_step(c, s, c->stage[0], c->stage[1], nb::kModeForce, c->stream);
}

// Synchronise and turn device flags into a status (flags are cleared).
nbody_status check_flags(nbody_ctx *c, bool init_phase) {
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  unsigned f = 0;
  NB_CUDA(c, cudaMemcpy(&f, c->flags, sizeof f, cudaMemcpyDeviceToHost));
  if (f) NB_CUDA(c, cudaMemset(c->flags, 0, sizeof(unsigned)));
  if (f & nb::kFlagBadInput)
    return fail(c, NBODY_EINVAL, "invalid state: non-finite position/velocity or negative/non-finite mass");
  if (f & nb::kFlagTimeout) return fail(c, NBODY_ETIMEOUT, "a bounded device wait ran out (kernel wound down)");
  if (f & nb::kFlagNonFinite) {
    if (init_phase)
      return fail(c, NBODY_EINVAL,
                  "non-finite acceleration at the given positions: two bodies of one system coincide");
    return fail(c, NBODY_ENONFINITE, "an acceleration became non-finite (close encounter or collision)");
  }
  return NBODY_OK;
}

// Bit i of q moved to bit 3i (21 bits in, 63 out).
uint64_t spread3(uint32_t q) {
  uint64_t k = 0;
  for (int i = 0; i < 21; ++i) k |= static_cast<uint64_t>((q >> i) & 1u) << (3 * i);
  return k;
}

// Planning data of the mixed stage, from the positions in body order h
// ([3][N]) and the stage order perm: each entry's hi parts and lo-part
// magnitudes, and each source group's widened box (as the box kernel makes
// it: padding entries excluded).
void plan_boxes(nbody_ctx *c, const std::vector<double> &h, const std::vector<int32_t> &perm) {
  const size_t N = c->N;
  const int64_t ns = c->n_stage, GS = 2 * nb::kBoxPairs;
  c->ent.assign(static_cast<size_t>(6 * ns), 0.f);
  std::vector<char> real(static_cast<size_t>(ns), 0);
  for (int64_t q = 0; q < ns; ++q) {
    const int32_t p = perm[q];
    real[q] = c->qidx_h[p] == q;
    for (int k = 0; k < 3; ++k) {
      const double x = h[k * N + p];
      const float hi = static_cast<float>(x);
      c->ent[6 * q + k] = hi;
      c->ent[6 * q + 3 + k] = std::fabs(static_cast<float>(x - static_cast<double>(hi)));
    }
  }
  c->gbox.assign(static_cast<size_t>((ns + GS - 1) / GS), PlanBox{});
  for (size_t g = 0; g < c->gbox.size(); ++g) {
    PlanBox b{{INFINITY, INFINITY, INFINITY}, {-INFINITY, -INFINITY, -INFINITY}, true};
    float l[3] = {0.f, 0.f, 0.f};
    for (int64_t q = static_cast<int64_t>(g) * GS; q < std::min(ns, static_cast<int64_t>(g + 1) * GS); ++q) {
      if (!real[q]) continue;
      for (int k = 0; k < 3; ++k) {
        b.lo[k] = std::min(b.lo[k], c->ent[6 * q + k]);
        b.hi[k] = std::max(b.hi[k], c->ent[6 * q + k]);
        l[k] = std::max(l[k], c->ent[6 * q + 3 + k]);
      }
      b.empty = false;
    }
    const float w = nb::kFarKappa * std::sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
    for (int k = 0; k < 3; ++k) {
      b.lo[k] -= w;
      b.hi[k] += w;
    }
    c->gbox[g] = b;
  }
}

// Planning cost of the mixed force launch per target block and chunk of the
// block's sources.  Each busy warp of the block (lane l of warp w holds the
// block's entries 32 (ipt w + k) + l, the last entry standing in past the
// block's end, as in the kernel) gets the widened box of its targets;
// against a source group whose box is disjoint from it (the kernel's far
// test) a pair costs 12 FP32 lane operations per target, else 18.  A chunk's
// weight per unit is that cost summed over the busy warps.  Chunks are one
// source group (kBoxPairs units) unless that means more than about 2e7 box
// tests; then several, and one group per chunk is tested.
// Relative cost of a (warp, source pair) step on the far and the near path.
constexpr int64_t kCostFar = 12, kCostNear = 18;

nb::ChunkCost chunk_costs(const nbody_ctx *c, const nbody_tiles &t) {
  const int64_t B = static_cast<int64_t>(t.threads) * t.ipt;
  const std::vector<nb::Blk> blks = nb::make_blocks(c->tgt_off, c->tgt_soff, B);
  const int64_t n_sys = static_cast<int64_t>(c->tgt_off.size()) - 1;
  struct Src {
    int64_t sb, len;
  };
  std::vector<Src> src(blks.size());
  int64_t tests = 0;
  {
    size_t k = 0;
    for (int64_t s = 0; s < n_sys; ++s) {
      const int64_t e = c->tgt_off[s + 1], ns = e - c->tgt_off[s];
      const int64_t sb = c->src_b.empty() ? c->tgt_soff[s] : c->src_b[s];
      const int64_t sn = c->src_n.empty() ? ns : c->src_n[s];
      for (; k < blks.size() && blks[k].i0 < e; ++k) {
        src[k] = {sb, (sn + 1) / 2};
        const int64_t busy = (blks[k].i1 - blks[k].i0 + 32 * t.ipt - 1) / (32 * t.ipt);
        tests += busy * ((src[k].len + nb::kBoxPairs - 1) / nb::kBoxPairs);
      }
    }
  }
  nb::ChunkCost cost;
  const int64_t m = std::max<int64_t>(1, (tests + 19999999) / 20000000);
  cost.chunk_units = nb::kBoxPairs * m;
  cost.w.resize(blks.size());
  std::vector<PlanBox> wb;
  for (size_t k = 0; k < blks.size(); ++k) {
    const nb::Blk &bk = blks[k];
    const int64_t cnt = bk.i1 - bk.i0, nw = (cnt + 32 * t.ipt - 1) / (32 * t.ipt);
    wb.assign(static_cast<size_t>(nw), PlanBox{});
    for (int64_t w = 0; w < nw; ++w) {
      PlanBox b{{INFINITY, INFINITY, INFINITY}, {-INFINITY, -INFINITY, -INFINITY}, false};
      float l[3] = {0.f, 0.f, 0.f};
      for (int64_t r = 32 * t.ipt * w; r < 32 * t.ipt * (w + 1); ++r) {
        const int64_t q = bk.q0 + std::min(r, cnt - 1);
        for (int d = 0; d < 3; ++d) {
          b.lo[d] = std::min(b.lo[d], c->ent[6 * q + d]);
          b.hi[d] = std::max(b.hi[d], c->ent[6 * q + d]);
          l[d] = std::max(l[d], c->ent[6 * q + 3 + d]);
        }
      }
      const float wd = nb::kFarKappa * std::sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
      for (int d = 0; d < 3; ++d) {
        b.lo[d] -= wd;
        b.hi[d] += wd;
      }
      wb[w] = b;
    }
    const int64_t len = src[k].len, nch = (len + cost.chunk_units - 1) / cost.chunk_units;
    std::vector<int64_t> &wk = cost.w[k];
    wk.assign(static_cast<size_t>(nch), 0);
    for (int64_t ch = 0; ch < nch; ++ch) {
      const int64_t u0 = ch * cost.chunk_units, u1 = std::min(len, u0 + cost.chunk_units);
      const int64_t g = (src[k].sb / 2 + (u0 + u1 - 1) / 2) / nb::kBoxPairs;  // the group at the chunk's middle
      const PlanBox &gb = c->gbox[std::min<size_t>(static_cast<size_t>(g), c->gbox.size() - 1)];
      int64_t sum = 0;
      for (const PlanBox &b : wb) {
        const bool far = gb.empty || gb.lo[0] > b.hi[0] || gb.lo[1] > b.hi[1] || gb.lo[2] > b.hi[2] ||
                         b.lo[0] > gb.hi[0] || b.lo[1] > gb.hi[1] || b.lo[2] > gb.hi[2];
        sum += far ? kCostFar : kCostNear;
      }
      wk[ch] = sum;
    }
  }
  return cost;
}

// Spatial order of each system's stage (mixed path): the bodies of a system
// sorted by the Morton code of their position in the system's bounding box
// (21 bits per axis; ties by body index), so that consecutive stage entries
// -- a warp's targets, a tile's source groups -- sit near each other and far
// groups take the force kernel's hi-only path.  Any order gives Eq. 1 to
// rounding; the order only decides which pairs are far (and the order of
// the sums).  Synchronous: reads the bound positions.  A system with a
// non-finite coordinate keeps body order (staging then reports it).
nbody_status spatial_order(nbody_ctx *c) {
  if (c->o.precision != NBODY_MIXED) return NBODY_OK;
  const size_t N = c->N, b = sizeof(double) * N;
  std::vector<double> h(3 * N);
  NB_CUDA(c, cudaMemcpyAsync(h.data(), c->x, b, cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(c, cudaMemcpyAsync(h.data() + N, c->y, b, cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(c, cudaMemcpyAsync(h.data() + 2 * N, c->z, b, cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  c->qidx_h.assign(N, 0);
  std::vector<int32_t> perm(static_cast<size_t>(c->n_stage), 0);
  std::vector<std::pair<uint64_t, int32_t>> key;
  // Ranges sorted independently: (first body, end body, first stage entry,
  // end stage entry) -- each system, or each rank's chunk of a row shard.
  struct Range {
    int64_t b, e, q, qe;
  };
  std::vector<Range> ranges;
  if (c->sh_world > 0) {
    for (int64_t k = 0; k < c->sh_world; ++k)
      ranges.push_back({std::min<int64_t>(k * c->sh_chunk, N), std::min<int64_t>((k + 1) * c->sh_chunk, N),
                        k * c->sh_chunk, (k + 1) * c->sh_chunk});
  } else {
    for (int64_t s = 0; s < c->n_sys; ++s) ranges.push_back({c->offsets[s], c->offsets[s + 1], c->soff[s], c->soff[s + 1]});
  }
  for (const Range &rg : ranges) {
    const int64_t b0 = rg.b, e0 = rg.e;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool finite = true;
    for (int64_t p = b0; p < e0; ++p)
      for (int k = 0; k < 3; ++k) {
        const double v = h[k * N + p];
        finite = finite && std::isfinite(v);
        lo[k] = std::min(lo[k], v);
        hi[k] = std::max(hi[k], v);
      }
    const double span = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]});
    key.clear();
    for (int64_t p = b0; p < e0; ++p) {
      uint64_t code = 0;
      if (finite && span > 0.0) {
        const double scale = ((1u << 21) - 1) / span;
        for (int k = 0; k < 3; ++k) {
          const double t = std::floor((h[k * N + p] - lo[k]) * scale);
          const uint32_t q = static_cast<uint32_t>(std::min(std::max(t, 0.0), double((1u << 21) - 1)));
          code |= spread3(q) << k;
        }
      }
      key.emplace_back(code, static_cast<int32_t>(p));
    }
    std::sort(key.begin(), key.end());
    for (int64_t r = 0; r < e0 - b0; ++r) {
      const int64_t slot = rg.q + r;
      c->qidx_h[key[r].second] = static_cast<int32_t>(slot);
      perm[slot] = key[r].second;
    }
    for (int64_t slot = rg.q + (e0 - b0); slot < rg.qe; ++slot) perm[slot] = static_cast<int32_t>(std::min<int64_t>(b0, N - 1));
  }
  plan_boxes(c, h, perm);
  NB_CUDA(c, cudaMemcpyAsync(c->qidx, c->qidx_h.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, c->stream));
  NB_CUDA(c, cudaMemcpyAsync(c->perm, perm.data(), sizeof(int32_t) * perm.size(), cudaMemcpyHostToDevice, c->stream));
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  return NBODY_OK;
}

nbody_status snapshot(nbody_ctx *c) {
  const size_t N = c->N, b = sizeof(double) * N;
  double *src[6] = {c->x, c->y, c->z, c->vx, c->vy, c->vz};
  for (int k = 0; k < 6; ++k) NB_CUDA(c, cudaMemcpyAsync(c->snap + k * N, src[k], b, cudaMemcpyDeviceToDevice, c->stream));
  return NBODY_OK;
}

// Stage the current positions, compute a = Eq. 1, snapshot; synchronous.
nbody_status refresh(nbody_ctx *c) {
  nbody_status st;
  if ((st = begin_work(c)) != NBODY_OK) return st;
  const State s = bound_state(c);
  NB_CUDA(c, nb::launch_prep(c->o.precision, prep_args(c, s, 0, 1), c->stream));
  if ((st = launch_force(c, s)) != NBODY_OK) return st;
  if ((st = snapshot(c)) != NBODY_OK) return st;
  if ((st = end_work(c)) != NBODY_OK) return st;
  return check_flags(c, true);
}

nbody_status alloc_scratch(nbody_ctx *c) {
  const size_t N = c->N;
  nbody_status st;
  // Stage layout: FP64 in body order; mixed in pair blocks with every system
  // padded to an even number of entries.
  c->soff.assign(c->n_sys + 1, 0);
  for (int64_t s = 0; s < c->n_sys; ++s) {
    const int64_t ns = c->offsets[s + 1] - c->offsets[s];
    c->soff[s + 1] = c->soff[s] + (c->o.precision == NBODY_MIXED ? (ns + 1) / 2 * 2 : ns);
  }
  c->n_stage = c->soff[c->n_sys];
  c->tgt_off = c->offsets;
  c->tgt_soff.assign(c->soff.begin(), c->soff.end() - 1);
#define NB_ALLOC(ptr, bytes) \
  if ((st = dalloc(c, reinterpret_cast<void **>(&(ptr)), (bytes))) != NBODY_OK) return st;
  NB_ALLOC(c->a, sizeof(double) * 3 * N);
  NB_ALLOC(c->stage[0], 32 * static_cast<size_t>(c->n_stage));
  NB_ALLOC(c->stage[1], 32 * static_cast<size_t>(c->n_stage));
  if (c->o.precision == NBODY_MIXED) {
    NB_ALLOC(c->R, sizeof(double) * 3 * N);
    NB_ALLOC(c->qidx, sizeof(int32_t) * N);
    NB_ALLOC(c->perm, sizeof(int32_t) * static_cast<size_t>(c->n_stage));
    NB_ALLOC(c->boxes, 2 * sizeof(float4) * static_cast<size_t>((c->n_stage / 2 + nb::kBoxPairs - 1) / nb::kBoxPairs));
    for (int b = 0; b < 2; ++b) NB_CUDA(c, nb::launch_pad_fill(c->stage[b], c->n_stage / 2, c->stream));
  }
  if (c->o.integrator == NBODY_RK4) NB_ALLOC(c->rk, sizeof(double) * 9 * N);
  NB_ALLOC(c->snap, sizeof(double) * 6 * N);
  NB_ALLOC(c->flags, sizeof(unsigned));
  NB_ALLOC(c->offsets_dev, sizeof(int64_t) * (c->n_sys + 1));
  NB_ALLOC(c->e_body, sizeof(double) * 2 * N);
  NB_ALLOC(c->e_out, sizeof(double) * 2 * c->n_sys);
#undef NB_ALLOC
  NB_CUDA(c, cudaMemset(c->flags, 0, sizeof(unsigned)));
  NB_CUDA(c, cudaMemcpy(c->offsets_dev, c->offsets.data(), sizeof(int64_t) * (c->n_sys + 1), cudaMemcpyHostToDevice));
  // energy items: blocks of kEnergyBlock targets against the whole system
  std::vector<Item> e;
  for (int64_t s = 0; s < c->n_sys; ++s) {
    for (int64_t i0 = c->offsets[s]; i0 < c->offsets[s + 1]; i0 += nb::kEnergyBlock) {
      Item it{};
      it.i0 = static_cast<int32_t>(i0);
      it.i1 = static_cast<int32_t>(std::min<int64_t>(i0 + nb::kEnergyBlock, c->offsets[s + 1]));
      it.j0 = static_cast<int32_t>(c->offsets[s]);
      it.j1 = static_cast<int32_t>(c->offsets[s + 1]);
      it.nsplit = 1;
      it.sys = static_cast<int32_t>(s);
      e.push_back(it);
    }
  }
  c->n_eitems = static_cast<int>(e.size());
  if ((st = dalloc(c, reinterpret_cast<void **>(&c->eitems), sizeof(Item) * e.size())) != NBODY_OK) return st;
  NB_CUDA(c, cudaMemcpy(c->eitems, e.data(), sizeof(Item) * e.size(), cudaMemcpyHostToDevice));
  return NBODY_OK;
}

void destroy(nbody_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  for (void *p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  delete c;
}

constexpr int kVjpTile = 512;  // sources per shared-memory stage of the VJP kernel

// Adjoint workspace: VJP tables (fixed tiles), adjoint state, the
// recomputation's shadow state, checkpoints for n_steps and the segment store.
nbody_status ensure_adjoint(nbody_ctx *c, int64_t n_steps) {
  Adjoint &A = c->adj;
  const int prec = c->o.precision;
  const size_t N = c->N;
  const int64_t K = c->o.ckpt_every;
  nbody_status st;
  if (!A.shadow) {  // first use, or an earlier attempt failed part way: start clean
    free_work(c, A.vj);
    for (void *q : {static_cast<void *>(A.rho), static_cast<void *>(A.nu), static_cast<void *>(A.gm), A.w})
      dfree(c, q);
    A.rho = A.nu = A.gm = nullptr;
    A.w = nullptr;
    nbody_tiles t{};
    t.threads = nb::vjp_threads(prec);
    t.ipt = 1;
    t.tj = kVjpTile;
    t.jsplit = 0;
    t.ctas_per_sm = 32;
    if (sym_block(c) == nb::kSymBlock) {  // FP64: the VJP evaluates each pair once too (64-body blocks)
      if ((st = build_sym_work(c, A.vj, 4, nb::kSymBlock)) != NBODY_OK) return st;
    } else {
      const size_t smem = nb::vjp_smem_bytes(prec, t.tj);
      int occ = 0;
      NB_CUDA(c, nb::vjp_prepare(prec, smem, &occ));
      if ((st = build_work(c, A.vj, t, occ, 4)) != NBODY_OK) return st;
      A.vj.smem = smem;
    }
    const size_t wbytes = (prec == NBODY_FP64 ? 32 : 16) * static_cast<size_t>(c->n_stage);
    if ((st = dalloc(c, reinterpret_cast<void **>(&A.rho), sizeof(double) * 3 * N)) != NBODY_OK) return st;
    if ((st = dalloc(c, reinterpret_cast<void **>(&A.nu), sizeof(double) * 3 * N)) != NBODY_OK) return st;
    if ((st = dalloc(c, reinterpret_cast<void **>(&A.gm), sizeof(double) * N)) != NBODY_OK) return st;
    if ((st = dalloc(c, &A.w, wbytes)) != NBODY_OK) return st;
    if ((st = dalloc(c, reinterpret_cast<void **>(&A.shadow), sizeof(double) * 9 * N)) != NBODY_OK) return st;
    NB_CUDA(c, cudaMemset(A.w, 0, wbytes));  // padding entries stay 0
  }
  const int64_t need_ckpt = (n_steps + K - 1) / K + 1;
  if (A.n_ckpt < need_ckpt) {
    dfree(c, A.ckpt);
    A.ckpt = nullptr;
    A.n_ckpt = 0;
    if ((st = dalloc(c, reinterpret_cast<void **>(&A.ckpt), sizeof(double) * 6 * N * need_ckpt)) != NBODY_OK) return st;
    A.n_ckpt = need_ckpt;
  }
  const int64_t need_store = std::min<int64_t>(K, std::max<int64_t>(n_steps, 1)) + 1;
  if (A.store_len < need_store) {
    dfree(c, A.store);
    A.store = nullptr;
    A.store_len = 0;
    const size_t stage_bytes = 32 * static_cast<size_t>(c->n_stage);
    if ((st = dalloc(c, &A.store, stage_bytes * need_store)) != NBODY_OK) return st;
    if (prec == NBODY_MIXED)
      for (int64_t j = 0; j < need_store; ++j)
        NB_CUDA(c, nb::launch_pad_fill(static_cast<unsigned char *>(A.store) + stage_bytes * j, c->n_stage / 2,
                                       c->stream));
    A.store_len = need_store;
  }
  return NBODY_OK;
}

// Makes the context's device (current at nbody_init) current for one call
// and gives the calling thread its own device back afterwards, so a context
// may be driven from a thread that works on another GPU.
class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess) prev_ = cur;
  }
  ~DeviceGuard() {
    if (prev_ >= 0) cudaSetDevice(prev_);
  }
  DeviceGuard(const DeviceGuard &) = delete;
  DeviceGuard &operator=(const DeviceGuard &) = delete;

 private:
  int prev_ = -1;
};

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

nbody_status nbody_init(nbody_ctx **out, int64_t n_systems, const int64_t *offsets, double *x, double *y, double *z,
                        double *vx, double *vy, double *vz, const double *m, const nbody_opts *o, void *cuda_stream) {
  g_init_error.clear();
  if (!out) return fail(nullptr, NBODY_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_systems < 1) return fail(nullptr, NBODY_EINVAL, "n_systems must be >= 1 (got %lld)", (long long)n_systems);
  if (!offsets) return fail(nullptr, NBODY_EINVAL, "offsets is NULL");
  if (!x || !y || !z || !vx || !vy || !vz || !m) return fail(nullptr, NBODY_EINVAL, "a state pointer is NULL");
  if (!o) return fail(nullptr, NBODY_EINVAL, "opts is NULL");
  if (offsets[0] != 0) return fail(nullptr, NBODY_EINVAL, "offsets[0] must be 0");
  for (int64_t s = 0; s < n_systems; ++s)
    if (offsets[s + 1] <= offsets[s])
      return fail(nullptr, NBODY_EINVAL, "system %lld is empty or offsets are not increasing", (long long)s);
  if (offsets[n_systems] >= (int64_t(1) << 31))
    return fail(nullptr, NBODY_EINVAL, "too many bodies (%lld >= 2^31)", (long long)offsets[n_systems]);
  if (!(o->G > 0.0) || !std::isfinite(o->G)) return fail(nullptr, NBODY_EINVAL, "G must be finite and > 0");
  if (!(o->dt != 0.0) || !std::isfinite(o->dt)) return fail(nullptr, NBODY_EINVAL, "dt must be finite and non-zero");
  if (o->precision != NBODY_FP64 && o->precision != NBODY_MIXED)
    return fail(nullptr, NBODY_EINVAL, "unknown precision %d", o->precision);
  if (o->ckpt_every < 0) return fail(nullptr, NBODY_EINVAL, "ckpt_every must be >= 0");
  if (o->flags & ~(NBODY_FLAG_NO_GRAPH | NBODY_FLAG_NO_SMALL | NBODY_FLAG_NO_SYM))
    return fail(nullptr, NBODY_EINVAL, "unknown flags");
  if (o->integrator != NBODY_VERLET && o->integrator != NBODY_RK4 && o->integrator != NBODY_LEAPFROG)
    return fail(nullptr, NBODY_EINVAL, "unknown integrator %d", o->integrator);
  if (!(o->close_omega_dt >= 0.0) || !std::isfinite(o->close_omega_dt))
    return fail(nullptr, NBODY_EINVAL, "close_omega_dt must be finite and >= 0");
  if (o->close_omega_dt > 0.0) {
    if (!(o->substep_omega_dt > 0.0) || !std::isfinite(o->substep_omega_dt))
      return fail(nullptr, NBODY_EINVAL, "substep_omega_dt must be finite and > 0 with close_omega_dt > 0");
    if (o->integrator != NBODY_VERLET)
      return fail(nullptr, NBODY_EINVAL, "close-encounter handling runs with the Verlet integrator only");
  }
  if (const int B = o->pair_once_block) {
    const bool pow2 = B > 0 && (B & (B - 1)) == 0;
    if (o->precision == NBODY_MIXED) {
      if (!(pow2 && B >= 32 * nb::kMsymMinTiles && B <= 32 * nb::kMsymMaxTiles))
        return fail(nullptr, NBODY_EINVAL, "pair_once_block (mixed) must be 0 or a power of two from %d to %d",
                    32 * nb::kMsymMinTiles, 32 * nb::kMsymMaxTiles);
    } else if (B != nb::kSymBlock && !(pow2 && B >= 32 * nb::kSymWideMinTiles && B <= 32 * nb::kSymWideMaxTiles)) {
      return fail(nullptr, NBODY_EINVAL, "pair_once_block must be 0, 64 or a power of two from %d to %d",
                  32 * nb::kSymWideMinTiles, 32 * nb::kSymWideMaxTiles);
    }
    int64_t rows = 1;
    for (int64_t s = 0; s < n_systems; ++s) rows = std::max(rows, (offsets[s + 1] - offsets[s] + B - 1) / B);
    if (rows > 65535 || rows * 3 * static_cast<int64_t>(sizeof(double)) * offsets[n_systems] > nb::kSymRowLimit)
      return fail(nullptr, NBODY_EINVAL, "pair_once_block %d: the partial rows would exceed %lld bytes", B,
                  static_cast<long long>(nb::kSymRowLimit));
  }

  nbody_ctx *c = new (std::nothrow) nbody_ctx;
  if (!c) return fail(nullptr, NBODY_ENOMEM, "host allocation failed");
  c->n_sys = n_systems;
  c->offsets.assign(offsets, offsets + n_systems + 1);
  c->N = static_cast<int32_t>(offsets[n_systems]);
  c->x = x; c->y = y; c->z = z; c->vx = vx; c->vy = vy; c->vz = vz; c->m = m;
  c->o = *o;
  if (o->tune_cache) c->tune_cache = o->tune_cache;
  c->o.tune_cache = nullptr;  // the context keeps its own copy
  if (c->o.ckpt_every == 0) c->o.ckpt_every = 100;
  c->user_stream = static_cast<cudaStream_t>(cuda_stream);
  // Optional host-side test hook: NBODY_INJECT_WAIT_STALL=k stalls one
  // bounded wait in the context's k-th launch that has one: the first source
  // tile of CTA 0 stays unissued in an adjoint product (VJP launch), or CTA 0
  // leaves out one barrier arrival in a single-launch step call.  The wait
  // runs out and nbody_grad / nbody_sync report ETIMEOUT.  (The force kernels
  // carry no test code.)
  if (const char *inj = std::getenv("NBODY_INJECT_WAIT_STALL")) c->stall_at = std::atoll(inj);

  auto bail = [&](nbody_status st) {
    g_init_error = c->err;
    destroy(c);
    return st;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&c->dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev)) != cudaSuccess) {
    fail(c, NBODY_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    return bail(NBODY_ECUDA);
  }
  // The pointers must be device (or managed) memory of this device.
  const void *ptrs[7] = {x, y, z, vx, vy, vz, m};
  for (const void *p : ptrs) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess || (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      fail(c, NBODY_EINVAL, "state pointers must be device memory");
      return bail(NBODY_EINVAL);
    }
  }
  if (c->user_stream == nullptr) {
    if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess) {
      fail(c, NBODY_ECUDA, "stream creation failed: %s", cudaGetErrorString(e));
      return bail(NBODY_ECUDA);
    }
    c->own_stream = true;
  } else {
    c->stream = c->user_stream;
  }
  if ((e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming)) != cudaSuccess) {
    fail(c, NBODY_ECUDA, "stream/event creation failed: %s", cudaGetErrorString(e));
    return bail(NBODY_ECUDA);
  }
  nbody_status st = alloc_scratch(c);
  if (st != NBODY_OK) return bail(st);
  if ((st = begin_work(c)) != NBODY_OK || (st = spatial_order(c)) != NBODY_OK) return bail(st);
  // Tiles: the tune cache's entry for this context, if it has a usable one,
  // else the defaults.
  bool tiled = false;
  nb::TuneEntry te;
  if (!c->tune_cache.empty() && nb::tune_cache_lookup(c->tune_cache, tune_key(c), te)) {
    nbody_tiles t{};
    t.threads = te.threads;
    t.ipt = te.ipt;
    t.tj = te.tj;
    t.jsplit = te.jsplit;
    t.ctas_per_sm = te.ctas_per_sm;
    tiled = tiles_valid(t, c->o.precision) && build_items(c, t) == NBODY_OK;
    cudaGetLastError();
  }
  if (!tiled && (st = build_items(c, default_tiles(c))) != NBODY_OK) return bail(st);
  // One FP64 Verlet system: every step of a call in one launch, a cluster up
  // to kSmallClusterMax bodies, a cooperative grid up to the grid kernel's
  // limit (each faster than the general path there).
  c->close_on = c->o.close_omega_dt > 0.0;
  if (c->close_on && (st = build_close(c)) != NBODY_OK) return bail(st);
  const bool single = c->n_sys == 1 && c->o.precision == NBODY_FP64 && c->o.integrator == NBODY_VERLET &&
                      !(c->o.flags & NBODY_FLAG_NO_SMALL) && !c->close_on;
  c->small = single && c->N <= std::min(kSmallClusterMax, nb::small_max_bodies());
  if (c->small && nb::small_prepare() != cudaSuccess) {  // no 16-CTA clusters here: the next path
    cudaGetLastError();
    c->small = false;
  }
  c->grid = single && !c->small && c->N <= nb::grid_max_bodies() &&
            nb::grid_shape(c->N, c->nsm, &c->grid_warps, &c->grid_ctas) == cudaSuccess;
  cudaGetLastError();
  if (c->grid) {
    if ((st = dalloc(c, reinterpret_cast<void **>(&c->xg), sizeof(double) * 6 * c->N)) != NBODY_OK) return bail(st);
    if ((st = dalloc(c, reinterpret_cast<void **>(&c->gbar), sizeof(unsigned))) != NBODY_OK) return bail(st);
  }
  if ((st = refresh(c)) != NBODY_OK) return bail(st);
  *out = c;
  return NBODY_OK;
}

nbody_status nbody_step(nbody_ctx *c, int64_t n_steps) {
  if (!c) return NBODY_EINVAL;
  const DeviceGuard dg(c->dev);
  if (c->sh_world > 0) return fail(c, NBODY_EINVAL, "a row shard steps with nbody_shard_step");
  if (n_steps < 0) return fail(c, NBODY_EINVAL, "n_steps must be >= 0");
  if (n_steps == 0) return NBODY_OK;
  nbody_status st;
  if ((st = begin_work(c)) != NBODY_OK) return st;
  const State s = bound_state(c);
  if (c->small) {
    nb::SmallArgs sa{};
    sa.x = s.x; sa.y = s.y; sa.z = s.z; sa.vx = s.vx; sa.vy = s.vy; sa.vz = s.vz;
    sa.ax = s.ax; sa.ay = s.ay; sa.az = s.az;
    sa.m = c->m;
    sa.flags = c->flags;
    sa.N = c->N;
    sa.n_steps = n_steps;
    sa.G = c->o.G;
    sa.dt = c->o.dt;
    sa.half_dt = 0.5 * c->o.dt;
    sa.half_dt2 = 0.5 * c->o.dt * c->o.dt;
    sa.stall = ++c->wait_seq == c->stall_at ? 1 : 0;
    cudaError_t e = nb::launch_small(sa, c->stream);
    if (e == cudaSuccess) return end_work(c);
    cudaGetLastError();  // cluster launch refused: fall back to the general path for good
    c->small = false;
  }
  if (c->grid) {
    nb::SmallArgs sa{};
    sa.x = s.x; sa.y = s.y; sa.z = s.z; sa.vx = s.vx; sa.vy = s.vy; sa.vz = s.vz;
    sa.ax = s.ax; sa.ay = s.ay; sa.az = s.az;
    sa.m = c->m;
    sa.flags = c->flags;
    sa.xg = c->xg;
    sa.gbar = c->gbar;
    sa.N = c->N;
    sa.G = c->o.G;
    sa.dt = c->o.dt;
    sa.half_dt = 0.5 * c->o.dt;
    sa.half_dt2 = 0.5 * c->o.dt * c->o.dt;
    // The barrier counts arrivals in 32 bits: steps x CTAs per launch < 2^31.
    const int64_t chunk = std::max<int64_t>(1, (int64_t(1) << 31) / c->grid_ctas);
    bool refused = false;
    for (int64_t done = 0; done < n_steps;) {
      sa.n_steps = std::min<int64_t>(chunk, n_steps - done);
      sa.stall = ++c->wait_seq == c->stall_at ? 1 : 0;
      NB_CUDA(c, cudaMemsetAsync(c->gbar, 0, sizeof(unsigned), c->stream));
      if (nb::launch_grid(sa, c->grid_warps, c->grid_ctas, c->stream) != cudaSuccess) {
        cudaGetLastError();  // cooperative launch refused: the general path, for good
        c->grid = false;
        refused = true;
        n_steps -= done;
        break;
      }
      done += sa.n_steps;
    }
    if (!refused) return end_work(c);
  }
  if (c->o.integrator == NBODY_RK4)  // stage 1 of the first step, from (r, v, a)
    NB_CUDA(c, nb::launch_rk_prep(c->o.precision, rk_args(c, s, nullptr, c->stage[0], 1), c->stream));
  else if (c->o.integrator == NBODY_LEAPFROG)  // the first half-step drift
    NB_CUDA(c, nb::launch_prep(c->o.precision, prep_args(c, s, 2, 0), c->stream));
  else  // Eq. 3 drift of the first step
    NB_CUDA(c, nb::launch_prep(c->o.precision, prep_args(c, s, 1, 0), c->stream));
  if (c->close_on) {  // the cluster members' first step starts from the state
    const nb::CloseArgs ca = close_args(c, s, c->stage[0], 0);
    NB_CUDA(c, nb::launch_close_far(ca, c->stream, true));
    NB_CUDA(c, nb::launch_close(ca, n_clusters(c), c->stream, true));
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  NB_CUDA(c, cudaStreamIsCapturing(c->stream, &cs));
  if ((c->o.flags & NBODY_FLAG_NO_GRAPH) || cs != cudaStreamCaptureStatusNone) {
    int64_t left = n_steps;
    while (left > 0) {  // parity restarts at 0 after each even chunk
      const int n = static_cast<int>(std::min<int64_t>(left, kGraphChunk));
      if ((st = launch_steps(c, s, n, c->stream)) != NBODY_OK) return st;
      left -= n;
    }
  } else {
    const int64_t full = n_steps / kGraphChunk;
    const int rem = static_cast<int>(n_steps % kGraphChunk);
    cudaGraphExec_t g;
    if (full > 0) {
      if ((st = graph_for(c, kGraphChunk, &g)) != NBODY_OK) return st;
      for (int64_t k = 0; k < full; ++k) NB_CUDA(c, cudaGraphLaunch(g, c->stream));
    }
    if (rem > 0) {
      if ((st = graph_for(c, rem, &g)) != NBODY_OK) return st;
      NB_CUDA(c, cudaGraphLaunch(g, c->stream));
    }
  }
  return end_work(c);
}

nbody_status nbody_accel(nbody_ctx *c, double *ax, double *ay, double *az) {
  if (!c) return NBODY_EINVAL;
  const DeviceGuard dg(c->dev);
  if (c->sh_world > 0) return fail(c, NBODY_EINVAL, "a row shard steps with nbody_shard_step");
  if (!ax || !ay || !az) return fail(c, NBODY_EINVAL, "output pointer is NULL");
  nbody_status st;
  if ((st = begin_work(c)) != NBODY_OK) return st;
  const size_t N = c->N, b = sizeof(double) * N;
  NB_CUDA(c, cudaMemcpyAsync(ax, c->a, b, cudaMemcpyDeviceToDevice, c->stream));
  NB_CUDA(c, cudaMemcpyAsync(ay, c->a + N, b, cudaMemcpyDeviceToDevice, c->stream));
  NB_CUDA(c, cudaMemcpyAsync(az, c->a + 2 * N, b, cudaMemcpyDeviceToDevice, c->stream));
  return end_work(c);
}

nbody_status nbody_reset(nbody_ctx *c) {
  if (!c) return NBODY_EINVAL;
  const DeviceGuard dg(c->dev);
  if (c->sh_world > 0) return fail(c, NBODY_EINVAL, "a row shard steps with nbody_shard_step");
  // As nbody_init: the spatial order of the new positions (mixed), so a reset
  // context computes bitwise what a new one would.
  nbody_status st;
  if ((st = begin_work(c)) != NBODY_OK) return st;
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  if ((st = spatial_order(c)) != NBODY_OK || (st = upload_nsl(c, c->adj.vj)) != NBODY_OK ||
      (c->o.precision == NBODY_MIXED && (st = build_items(c, c->tiles)) != NBODY_OK))
    return st;
  if (c->close_on && (st = build_close(c)) != NBODY_OK) return st;  // the pairs of the new positions
  return refresh(c);
}

nbody_status nbody_pair_once(const nbody_ctx *c, int32_t *on) {
  if (!c || !on) return NBODY_EINVAL;
  *on = c->fw.sym_pairs != nullptr ? 32 * c->fw.sym_tiles : 0;
  return NBODY_OK;
}

nbody_status nbody_close_info(const nbody_ctx *c, int64_t *n_pairs, int32_t *n_clusters, int32_t *n_members,
                              int32_t *k_max) {
  if (!c) return NBODY_EINVAL;
  if (n_pairs) *n_pairs = c->close.n_pairs;
  if (n_clusters) *n_clusters = static_cast<int32_t>(c->close.cl_k.size());
  if (n_members) *n_members = static_cast<int32_t>(c->close.mem_body.size());
  if (k_max) *k_max = c->close.k_max;
  return NBODY_OK;
}

nbody_status nbody_reorder(nbody_ctx *c) {
  if (!c) return NBODY_EINVAL;
  const DeviceGuard dg(c->dev);
  if (c->sh_world > 0) return fail(c, NBODY_EINVAL, "a row shard steps with nbody_shard_step");
  nbody_status st;
  if ((st = begin_work(c)) != NBODY_OK) return st;
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  if ((st = spatial_order(c)) != NBODY_OK) return st;
  // the order moved bodies between stage entries, and the planning costs changed
  if (c->o.precision == NBODY_MIXED && (st = build_items(c, c->tiles)) != NBODY_OK) return st;
  if ((st = upload_nsl(c, c->adj.vj)) != NBODY_OK) return st;
  return end_work(c);
}

nbody_status nbody_energy(nbody_ctx *c, double *e_host) {
  if (!c) return NBODY_EINVAL;
  const DeviceGuard dg(c->dev);
  if (c->sh_world > 0) return fail(c, NBODY_EINVAL, "a row shard steps with nbody_shard_step");
  if (!e_host) return fail(c, NBODY_EINVAL, "e_host is NULL");
  nbody_status st;
  if ((st = begin_work(c)) != NBODY_OK) return st;
  const size_t N = c->N;
  nb::EnergyArgs ea{};
  ea.x = c->x; ea.y = c->y; ea.z = c->z; ea.vx = c->vx; ea.vy = c->vy; ea.vz = c->vz; ea.m = c->m;
  ea.e_kin = c->e_body;
  ea.e_pot = c->e_body + N;
  ea.items = c->eitems;
  ea.n_items = c->n_eitems;
  ea.G = c->o.G;
  NB_CUDA(c, nb::launch_energy(ea, c->stream));
  nb::ReduceArgs ra{};
  ra.e_kin = c->e_body;
  ra.e_pot = c->e_body + N;
  ra.offsets = c->offsets_dev;
  ra.out = c->e_out;
  ra.n_systems = static_cast<int32_t>(c->n_sys);
  NB_CUDA(c, nb::launch_energy_reduce(ra, c->stream));
  std::vector<double> h(2 * c->n_sys);
  NB_CUDA(c, cudaMemcpyAsync(h.data(), c->e_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->stream));
  if ((st = end_work(c)) != NBODY_OK) return st;
  if ((st = check_flags(c, false)) != NBODY_OK) return st;
  for (int64_t s = 0; s < c->n_sys; ++s) e_host[s] = h[s] + h[c->n_sys + s];
  return NBODY_OK;
}

nbody_status nbody_sync(nbody_ctx *c) {
  if (!c) return NBODY_EINVAL;
  const DeviceGuard dg(c->dev);
  return check_flags(c, false);
}

nbody_status nbody_get_tiles(const nbody_ctx *c, nbody_tiles *t) {
  if (!c || !t) return NBODY_EINVAL;
  *t = c->tiles;
  return NBODY_OK;
}

nbody_status nbody_set_tiles(nbody_ctx *c, const nbody_tiles *t) {
  if (!c) return NBODY_EINVAL;
  const DeviceGuard dg(c->dev);
  if (c->sh_world > 0) return fail(c, NBODY_EINVAL, "a row shard steps with nbody_shard_step");
  if (!t || !tiles_valid(*t, c->o.precision))
    return fail(c, NBODY_EINVAL, "invalid tiles (see nbody.h: supported threads/ipt pairs, tj 64..2048 step 64, jsplit 0..64, ctas_per_sm 1..32)");
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  return build_items(c, *t);
}

nbody_status nbody_autotune(nbody_ctx *c, int32_t probe_steps, nbody_tiles *best, double *best_ms) {
  if (!c) return NBODY_EINVAL;
  const DeviceGuard dg(c->dev);
  if (c->sh_world > 0) return fail(c, NBODY_EINVAL, "a row shard steps with nbody_shard_step");
  if (probe_steps < 1) return fail(c, NBODY_EINVAL, "probe_steps must be >= 1");
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  // Tiles shape only the general path (and nbody_accel / nbody_grad): time
  // that path even where a single-launch kernel serves nbody_step.
  struct PathGuard {
    nbody_ctx *c;
    bool small, grid;
    ~PathGuard() {
      c->small = small;
      c->grid = grid;
    }
  } const keep{c, c->small, c->grid};
  c->small = c->grid = false;
  const size_t N = c->N, b = sizeof(double) * N;
  // Save the bound state and a; every candidate starts from it.
  double *save = nullptr;
  nbody_status st = dalloc(c, reinterpret_cast<void **>(&save), 9 * b);
  if (st != NBODY_OK) return st;
  // The copies go on the context's stream, so the probes are ordered after
  // them (a device-to-device cudaMemcpy may return before it completes, and
  // the context's stream does not wait for the legacy default stream).
  double *src[9] = {c->x, c->y, c->z, c->vx, c->vy, c->vz, c->a, c->a + N, c->a + 2 * N};
  for (int k = 0; k < 9; ++k)
    NB_CUDA(c, cudaMemcpyAsync(save + k * N, src[k], b, cudaMemcpyDeviceToDevice, c->stream));
  auto restore = [&]() -> nbody_status {
    for (int k = 0; k < 9; ++k)
      NB_CUDA(c, cudaMemcpyAsync(src[k], save + k * N, b, cudaMemcpyDeviceToDevice, c->stream));
    return NBODY_OK;
  };
  std::vector<nbody_tiles> cand;
  const bool mixed = c->o.precision == NBODY_MIXED;
  for (int th : {64, 128, 256, 384, 512, 768, 1024})
    for (int ip : {1, 2, 4})
      for (int tj : {128, 256, 512, 1024, 2048})
        for (int cps : {1, 2, 3, 4, 6, 8})
          for (int js : {0, 1, 2, 4, 8, 16}) {
          if (!nb::force_config_supported(c->o.precision, th, ip)) continue;
          // FP64 is bound by the FP64 pipe: only the barrier spacing (tj) and the warp count matter
          if (!mixed && tj < 512) continue;
          if (mixed && tj > 1024) continue;
          // at most 1024 threads per SM; the mixed path wants >= 512 threads or >= 1024 targets per SM
          if (th * cps > 1024 || (mixed && th * cps < 512 && th * cps * ip < 1024)) continue;
          // Dynamic chunks (jsplit) add partial rows; they pay only where the
          // cost per interaction varies between shares: the mixed path, whose
          // far source groups cost 12 lane operations against 18 for near ones.
          if (js > 0 && !mixed) continue;
          nbody_tiles t;
          t.threads = th;
          t.ipt = ip;
          t.tj = tj;
          t.ctas_per_sm = cps;
          t.jsplit = js;
          cand.push_back(t);
        }
  // the pair-once FP64 kernel has no tiles to choose: time the current ones only
  if (sym_block(c)) cand.assign(1, c->tiles);
  cudaEvent_t e0, e1;
  NB_CUDA(c, cudaEventCreate(&e0));
  NB_CUDA(c, cudaEventCreate(&e1));
  // One timing: build t, a warm-up call with the timed step count (so the
  // timed call replays a cached graph instead of capturing one while the GPU
  // waits), the timed call, and the state restored.  ms per step, or < 0.
  auto time_tiles = [&](const nbody_tiles &t, int32_t steps) -> double {
    if ((st = build_items(c, t)) != NBODY_OK) return -1.0;
    if ((st = nbody_step(c, steps)) != NBODY_OK) return -1.0;
    cudaEventRecord(e0, c->stream);
    if ((st = nbody_step(c, steps)) != NBODY_OK) return -1.0;
    cudaEventRecord(e1, c->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = fail(c, NBODY_ECUDA, "autotune timing failed");
      return -1.0;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if ((st = restore()) != NBODY_OK) return -1.0;
    return static_cast<double>(ms) / steps;
  };
  // First pass: every candidate once.  Second pass: the fastest few again, three
  // times each over 4x the steps, keeping each one's best: single short
  // probes of candidates a few percent apart pick the wrong one too often.
  std::vector<std::pair<double, size_t>> r1;
  for (size_t i = 0; i < cand.size() && st == NBODY_OK; ++i) {
    const double ms = time_tiles(cand[i], probe_steps);
    if (ms >= 0.0) r1.emplace_back(ms, i);
  }
  std::sort(r1.begin(), r1.end());
  nbody_tiles win = c->tiles;
  double win_ms = 1e300;
  const int32_t steps2 = probe_steps > (1 << 28) ? probe_steps : 4 * probe_steps;
  for (size_t r = 0; r < r1.size() && r < 6 && st == NBODY_OK; ++r) {
    double best_t = 1e300;
    for (int rep = 0; rep < 3 && st == NBODY_OK; ++rep) {
      const double ms = time_tiles(cand[r1[r].second], steps2);
      if (ms >= 0.0) best_t = std::min(best_t, ms);
    }
    if (best_t < win_ms) {
      win_ms = best_t;
      win = cand[r1[r].second];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  nbody_status st2 = restore();
  if (cudaStreamSynchronize(c->stream) != cudaSuccess && st2 == NBODY_OK)
    st2 = fail(c, NBODY_ECUDA, "autotune restore failed");
  dfree(c, save);
  if (st != NBODY_OK) return st;
  if (st2 != NBODY_OK) return st2;
  if ((st = build_items(c, win)) != NBODY_OK) return st;
  if ((st = check_flags(c, false)) != NBODY_OK) return st;
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms;
  if (!c->tune_cache.empty()) {
    nb::TuneEntry te;
    te.threads = win.threads;
    te.ipt = win.ipt;
    te.tj = win.tj;
    te.jsplit = win.jsplit;
    te.ctas_per_sm = win.ctas_per_sm;
    te.ms_per_step = win_ms;
    const std::string why = nb::tune_cache_store(c->tune_cache, tune_key(c), te);
    if (!why.empty()) return fail(c, NBODY_EINVAL, "tune cache not written: %s", why.c_str());
  }
  return NBODY_OK;
}

nbody_status nbody_kernel_times(nbody_ctx *c, int32_t n_steps, double *out) {
  if (!c || !out) return NBODY_EINVAL;
  const DeviceGuard dg(c->dev);
  if (c->sh_world > 0) return fail(c, NBODY_EINVAL, "a row shard steps with nbody_shard_step");
  if (c->o.integrator != NBODY_VERLET) return fail(c, NBODY_EINVAL, "nbody_kernel_times times Verlet steps only");
  if (c->close_on) return fail(c, NBODY_EINVAL, "nbody_kernel_times times plain Verlet steps (no close pairs)");
  if (n_steps < 1) return fail(c, NBODY_EINVAL, "n_steps must be >= 1");
  nbody_status st;
  if ((st = begin_work(c)) != NBODY_OK) return st;
  const State s = bound_state(c);
  std::vector<cudaEvent_t> ev(3 * static_cast<size_t>(n_steps), nullptr);
  for (cudaEvent_t &e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      for (cudaEvent_t &f : ev)
        if (f) cudaEventDestroy(f);
      return fail(c, NBODY_ECUDA, "cudaEventCreate failed");
    }
  auto run = [&]() -> nbody_status {
    NB_CUDA(c, nb::launch_prep(c->o.precision, prep_args(c, s, 1, 0), c->stream));
    for (int32_t i = 0; i < n_steps; ++i) {
      const int k = (i % kGraphChunk) & 1;  // same staging parity as nbody_step
      nbody_status r = launch_one_step(c, s, c->stage[k], c->stage[1 - k], nb::kModeStep, c->stream, &ev[3 * i]);
      if (r != NBODY_OK) return r;
    }
    NB_CUDA(c, cudaEventSynchronize(ev.back()));
    double f = 0, v = 0;
    for (int32_t i = 0; i < n_steps; ++i) {
      float a = 0.f, b = 0.f;
      NB_CUDA(c, cudaEventElapsedTime(&a, ev[3 * i], ev[3 * i + 1]));
      NB_CUDA(c, cudaEventElapsedTime(&b, ev[3 * i + 1], ev[3 * i + 2]));
      f += a;
      v += b;
    }
    float all = 0.f;
    NB_CUDA(c, cudaEventElapsedTime(&all, ev.front(), ev.back()));
    out[0] = f / n_steps;
    out[1] = v / n_steps;
    out[2] = static_cast<double>(all) / n_steps;
    out[3] = n_steps;
    return NBODY_OK;
  };
  st = run();
  for (cudaEvent_t &e : ev) cudaEventDestroy(e);
  if (st != NBODY_OK) return st;
  return end_work(c);
}

nbody_status nbody_grad(nbody_ctx *c, int64_t n_steps, const double *dL_dr_T, const double *dL_dv_T, double *dL_dr0,
                        double *dL_dv0, double *dL_dm) {
  if (!c) return NBODY_EINVAL;
  const DeviceGuard dg(c->dev);
  if (c->sh_world > 0) return fail(c, NBODY_EINVAL, "a row shard steps with nbody_shard_step");
  if (n_steps < 0) return fail(c, NBODY_EINVAL, "n_steps must be >= 0");
  if (!dL_dr_T || !dL_dr0 || !dL_dv0 || !dL_dm) return fail(c, NBODY_EINVAL, "a gradient pointer is NULL");
  if (n_steps > (int64_t(1) << 31)) return fail(c, NBODY_EINVAL, "n_steps too large");
  if (c->o.integrator != NBODY_VERLET) return fail(c, NBODY_EINVAL, "the adjoint covers Verlet (Eqs. 3-4) only");
  if (c->close_on) return fail(c, NBODY_EINVAL, "the adjoint covers plain Verlet (no close pairs)");
  nbody_status st;
  if ((st = ensure_adjoint(c, n_steps)) != NBODY_OK) return st;
  if ((st = begin_work(c)) != NBODY_OK) return st;
  Adjoint &A = c->adj;
  const int prec = c->o.precision;
  const size_t N = c->N, b = sizeof(double) * N;
  const int64_t T = n_steps, K = c->o.ckpt_every;
  const State sh = {A.shadow, A.shadow + N, A.shadow + 2 * N, A.shadow + 3 * N, A.shadow + 4 * N,
                    A.shadow + 5 * N, A.shadow + 6 * N, A.shadow + 7 * N, A.shadow + 8 * N};
  const size_t stage_bytes = 32 * static_cast<size_t>(c->n_stage);
  auto store = [&](int64_t j) { return static_cast<unsigned char *>(A.store) + stage_bytes * j; };
  auto ckpt = [&](int64_t k) { return A.ckpt + static_cast<size_t>(k) * 6 * N; };

  // Forward from the snapshot (r0, v0), keeping (r, v) every K steps.
  NB_CUDA(c, cudaMemcpyAsync(A.shadow, c->snap, 6 * b, cudaMemcpyDeviceToDevice, c->stream));
  NB_CUDA(c, nb::launch_prep(prec, prep_args(c, sh, 0, 0), c->stream));
  if ((st = launch_one_step(c, sh, c->stage[0], c->stage[1], nb::kModeForce, c->stream)) != NBODY_OK) return st;
  NB_CUDA(c, cudaMemcpyAsync(ckpt(0), A.shadow, 6 * b, cudaMemcpyDeviceToDevice, c->stream));
  const int64_t nseg = (T + K - 1) / K;
  for (int64_t sgi = 0; sgi < nseg - 1; ++sgi) {  // the last segment needs no checkpoint at its end
    NB_CUDA(c, nb::launch_prep(prec, prep_args(c, sh, 1, 0), c->stream));
    int64_t left = K;
    while (left > 0) {
      const int n = static_cast<int>(std::min<int64_t>(left, kGraphChunk));
      if ((st = launch_steps(c, sh, n, c->stream)) != NBODY_OK) return st;
      left -= n;
    }
    NB_CUDA(c, cudaMemcpyAsync(ckpt(sgi + 1), A.shadow, 6 * b, cudaMemcpyDeviceToDevice, c->stream));
  }

  // Reverse sweep.
  nb::AdjArgs ad{};
  ad.rho = A.rho;
  ad.nu = A.nu;
  ad.gm = A.gm;
  ad.w = A.w;
  ad.partial = A.vj.partial;
  ad.nsl = A.vj.nsl;
  ad.qidx = c->qidx;
  ad.flags = c->flags;
  ad.N = c->N;
  ad.G = c->o.G;
  ad.dt = c->o.dt;
  ad.half_dt = 0.5 * c->o.dt;
  ad.half_dt2 = 0.5 * c->o.dt * c->o.dt;
  ad.mode = T > 0 ? 0 : 1;
  NB_CUDA(c, nb::launch_adjoint_init(prec, ad, dL_dr_T, dL_dv_T, c->stream));
  nb::VjpArgs vj{};
  vj.w = A.w;
  vj.perm = c->perm;
  vj.partial = A.vj.partial;
  vj.flags = c->flags;
  vj.blks = A.vj.blks;
  vj.segs = A.vj.segs;
  vj.seg_off = A.vj.seg_off;
  vj.N = c->N;
  vj.tj = kVjpTile;
  auto product = [&](const void *pos, int mode) -> nbody_status {
    if (A.vj.sym_pairs) {  // pair-once (FP64): no bounded wait to stall
      nb::VjpSymArgs vs{};
      vs.pos = static_cast<const double4_32a *>(pos);
      vs.w = static_cast<const double4_32a *>(A.w);
      vs.partial = A.vj.partial;
      vs.pairs = A.vj.sym_pairs;
      vs.n_pairs = A.vj.n_sym;
      vs.ctr = A.vj.dyn_ctr;
      vs.N = c->N;
      NB_CUDA(c, nb::launch_vjp_sym(vs, A.vj.grid, c->stream));
    } else {
      vj.pos = pos;
      vj.stall = ++c->wait_seq == c->stall_at ? 1 : 0;
      NB_CUDA(c, nb::launch_vjp(prec, A.vj.grid, A.vj.smem, vj, c->stream));
    }
    ad.mode = mode;
    NB_CUDA(c, nb::launch_adjoint(prec, ad, c->stream));
    return NBODY_OK;
  };
  for (int64_t sgi = nseg - 1; sgi >= 0; --sgi) {
    // Recompute the staged positions r_{s0} .. r_{s0+len} of this segment.
    const int64_t s0 = sgi * K, len = std::min(K, T - s0);
    NB_CUDA(c, cudaMemcpyAsync(A.shadow, ckpt(sgi), 6 * b, cudaMemcpyDeviceToDevice, c->stream));
    NB_CUDA(c, nb::launch_prep(prec, prep_args(c, sh, 0, 0, store(0)), c->stream));
    if ((st = launch_one_step(c, sh, store(0), store(1), nb::kModeForce, c->stream)) != NBODY_OK) return st;
    NB_CUDA(c, nb::launch_prep(prec, prep_args(c, sh, 1, 0, store(1)), c->stream));
    for (int64_t j = 1; j < len; ++j)
      if ((st = launch_one_step(c, sh, store(j), store(j + 1), nb::kModeStep, c->stream)) != NBODY_OK) return st;
    // Iterations i = s0+len-1 .. s0 use r_{i+1} = store[i+1-s0].
    for (int64_t i = s0 + len - 1; i >= s0; --i)
      if ((st = product(store(i + 1 - s0), i == 0 ? 1 : 0)) != NBODY_OK) return st;
  }
  if (T == 0)  // no segment staged r_0: the shadow still holds the snapshot
    NB_CUDA(c, nb::launch_prep(prec, prep_args(c, sh, 0, 0, store(0)), c->stream));
  if ((st = product(store(0), 2)) != NBODY_OK) return st;  // the last product, at r_0

  NB_CUDA(c, cudaMemcpyAsync(dL_dr0, A.rho, 3 * b, cudaMemcpyDeviceToDevice, c->stream));
  NB_CUDA(c, cudaMemcpyAsync(dL_dv0, A.nu, 3 * b, cudaMemcpyDeviceToDevice, c->stream));
  NB_CUDA(c, cudaMemcpyAsync(dL_dm, A.gm, b, cudaMemcpyDeviceToDevice, c->stream));
  if ((st = end_work(c)) != NBODY_OK) return st;
  return check_flags(c, false);
}

nbody_status nbody_shard(nbody_ctx *c, int32_t rank, int32_t world) {
  if (!c) return NBODY_EINVAL;
  const DeviceGuard dg(c->dev);
  if (c->sh_world > 0) return fail(c, NBODY_EINVAL, "the context is already a row shard");
  if (world < 1 || rank < 0 || rank >= world) return fail(c, NBODY_EINVAL, "need 0 <= rank < world");
  if (c->n_sys != 1) return fail(c, NBODY_EINVAL, "row shards take one system");
  if (c->o.integrator != NBODY_VERLET) return fail(c, NBODY_EINVAL, "row shards run velocity Verlet");
  if (c->close_on) return fail(c, NBODY_EINVAL, "row shards run plain Verlet (no close pairs)");
  nbody_status st;
  if ((st = begin_work(c)) != NBODY_OK) return st;
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  const int64_t N = c->N;
  const int64_t C = ((N + world - 1) / world + 1) / 2 * 2;  // equal chunks, whole source pairs
  const int64_t n_stage = C * world;
  // Stages of world equal chunks: bodies of rank k at entries [k C, ...),
  // the rest inert padding (every entry starts as padding; staging
  // overwrites the real ones).
  drop_graphs(c);
  for (int b = 0; b < 2; ++b) {
    dfree(c, c->stage[b]);
    c->stage[b] = nullptr;
  }
  dfree(c, c->perm);
  c->perm = nullptr;
  for (int b = 0; b < 2; ++b) {
    if ((st = dalloc(c, &c->stage[b], 32 * static_cast<size_t>(n_stage))) != NBODY_OK) return st;
    NB_CUDA(c, c->o.precision == NBODY_MIXED ? nb::launch_pad_fill(c->stage[b], n_stage / 2, c->stream)
                                             : nb::launch_pad_fill_fp64(c->stage[b], n_stage, c->stream));
  }
  if (c->o.precision == NBODY_MIXED) {
    dfree(c, c->boxes);
    c->boxes = nullptr;
    if ((st = dalloc(c, reinterpret_cast<void **>(&c->perm), sizeof(int32_t) * static_cast<size_t>(n_stage))) !=
            NBODY_OK ||
        (st = dalloc(c, reinterpret_cast<void **>(&c->boxes),
                     2 * sizeof(float4) * static_cast<size_t>((n_stage / 2 + nb::kBoxPairs - 1) / nb::kBoxPairs))) !=
            NBODY_OK)
      return st;
  }
  c->n_stage = n_stage;
  c->soff = {0, n_stage};
  c->sh_world = world;
  c->sh_rank = rank;
  c->sh_chunk = C;
  c->sh_begin = std::min<int64_t>(rank * C, N);
  c->sh_end = std::min<int64_t>(c->sh_begin + C, N);
  c->sh_cur = 0;
  c->small = c->grid = false;
  // the adjoint's workspace is laid out for the old stage; shards take no gradient
  free_work(c, c->adj.vj);
  for (void *q : {static_cast<void *>(c->adj.rho), static_cast<void *>(c->adj.nu), static_cast<void *>(c->adj.gm),
                  c->adj.w, static_cast<void *>(c->adj.shadow), static_cast<void *>(c->adj.ckpt), c->adj.store})
    dfree(c, q);
  c->adj = Adjoint{};
  if ((st = spatial_order(c)) != NBODY_OK) return st;
  // This rank's targets against every source of the system.
  c->tgt_off = {c->sh_begin, c->sh_end};
  c->tgt_soff = {c->sh_begin};
  c->src_b = {0};
  c->src_n = {n_stage};
  if (c->sh_end > c->sh_begin && (st = build_items(c, c->tiles)) != NBODY_OK) return st;
  // Every rank holds the whole state: stage the first step's Eq. 3 drift of
  // every body, so the first shard step needs no exchange.
  NB_CUDA(c, nb::launch_prep(c->o.precision, prep_args(c, bound_state(c), 1, 0), c->stream));
  if ((st = end_work(c)) != NBODY_OK) return st;
  return check_flags(c, false);
}

nbody_status nbody_shard_step(nbody_ctx *c) {
  if (!c) return NBODY_EINVAL;
  const DeviceGuard dg(c->dev);
  if (c->sh_world == 0) return fail(c, NBODY_EINVAL, "not a row shard (see nbody_shard)");
  nbody_status st;
  if ((st = begin_work(c)) != NBODY_OK) return st;
  const int k = c->sh_cur;
  if (c->sh_end > c->sh_begin &&
      (st = launch_one_step(c, bound_state(c), c->stage[k], c->stage[1 - k], nb::kModeStep, c->stream)) != NBODY_OK)
    return st;
  c->sh_cur = 1 - k;
  return end_work(c);
}

nbody_status nbody_shard_buffer(const nbody_ctx *c, void **stage, int64_t *chunk_bytes) {
  if (!c || !stage || !chunk_bytes || c->sh_world == 0) return NBODY_EINVAL;
  *stage = c->stage[c->sh_cur];
  *chunk_bytes = 32 * c->sh_chunk;
  return NBODY_OK;
}

void nbody_free(nbody_ctx *c) {
  if (!c) return;
  const DeviceGuard dg(c->dev);
  destroy(c);
}

const char *nbody_last_error(const nbody_ctx *c) { return c ? c->err.c_str() : g_init_error.c_str(); }

nbody_status nbody_peaks(double *out) {
  if (!out) return NBODY_EINVAL;
  cudaError_t e = nb::run_peaks(out);
  if (e != cudaSuccess) return fail(nullptr, NBODY_ECUDA, "peaks: %s", cudaGetErrorString(e));
  return NBODY_OK;
}

}  // extern "C"
