// Test-only C entry point over the library's host work planner
// (paper_2112_15079_gb300/csrc/work_plan.h).  tests/test_work_plan.py builds
// it with g++ and checks the plan's invariants on the CPU; no CUDA involved.
#include <cstdint>
#include <cstring>
#include <vector>

#include "work_plan.h"

// meta[0..4] = blocks, segments, grid, dynamic chunks, rows.  Returns 0, or
// 1 when the planner refuses, 2 when a capacity is too small.  src_b / src_n
// (NULL or n_sys entries each) are the planner's optional source ranges;
// cw (NULL, or the weights of every block's chunks, block k's at
// cw[cw_off[k] .. cw_off[k+1])) with chunk_units its optional cost model.
extern "C" int wp_plan(int64_t n_sys, const int64_t *offsets, const int64_t *soff, int mixed, int threads, int ipt,
                       int jsplit, int64_t slots, int64_t cap_blks, int64_t cap_segs, int64_t cap_pieces,
                       int32_t *blks, int32_t *segs, int32_t *seg_off, uint16_t *nsl, int64_t *meta,
                       const int64_t *src_b, const int64_t *src_n, const int64_t *cw, const int64_t *cw_off,
                       int64_t n_cw_blks, int64_t chunk_units) {
  const std::vector<int64_t> off(offsets, offsets + n_sys + 1), so(soff, soff + n_sys + 1);
  nb::ChunkCost cost;
  cost.chunk_units = chunk_units;
  for (int64_t k = 0; cw && k < n_cw_blks; ++k) cost.w.emplace_back(cw + cw_off[k], cw + cw_off[k + 1]);
  const std::vector<int64_t> sb(src_b ? src_b : nullptr, src_b ? src_b + n_sys : nullptr);
  const std::vector<int64_t> sn(src_n ? src_n : nullptr, src_n ? src_n + n_sys : nullptr);
  nb::WorkPlan p;
  if (!nb::plan_work(off, so, mixed != 0, threads, ipt, jsplit, slots, p, src_b ? &sb : nullptr,
                     src_n ? &sn : nullptr, cw ? &cost : nullptr)
           .empty())
    return 1;
  meta[0] = static_cast<int64_t>(p.blks.size());
  meta[1] = static_cast<int64_t>(p.segs.size());
  meta[2] = p.grid;
  meta[3] = p.n_dyn;
  meta[4] = p.rows;
  if (meta[0] > cap_blks || meta[1] > cap_segs || static_cast<int64_t>(p.seg_off.size()) > cap_pieces + 1) return 2;
  std::memcpy(blks, p.blks.data(), sizeof(nb::Blk) * p.blks.size());
  std::memcpy(segs, p.segs.data(), sizeof(nb::Seg) * p.segs.size());
  std::memcpy(seg_off, p.seg_off.data(), sizeof(int32_t) * p.seg_off.size());
  std::memcpy(nsl, p.nsl.data(), sizeof(uint16_t) * p.nsl.size());
  return 0;
}
