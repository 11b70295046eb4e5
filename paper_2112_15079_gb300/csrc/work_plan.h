// Host-side plan of one stream-K force (or VJP) launch: target blocks, their
// source segments, the pieces (CTA shares) that hold the segments, and the
// partial rows per body.  Plain C++ without CUDA, so the library and a CPU
// test build the same code.
//
// The plan: each system's targets are cut into blocks of balanced size (at
// most threads * ipt bodies).  The work line lists, block by block, the
// sources of the block's system in units of `unit` sources (2 on the mixed
// path, whose stage pairs sources; 1 on the FP64 path), each unit weighted by
// the warps the block keeps busy (or by a cost model, below).  The first
// three quarters of every block's line (all of it when jsplit == 0), block
// after block, are cut into `grid` equal static shares; the last quarters,
// block after block, into grid * jsplit chunks handed out at run time.  A
// segment is the part of one block inside one piece; its slot is its rank
// within the block, which fixes the partial row it writes and its place in
// the summation order.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

namespace nb {

// Force kernels: a target block of one system (at most threads * ipt
// consecutive bodies [i0, i1); q0 = stage index of body i0) whose source
// range is cut into `nsplit` contiguous segments processed by different CTAs.
struct Blk {
  int32_t i0, i1, q0, nsplit;
};
static_assert(sizeof(Blk) == 16, "Blk layout");

// One segment: sources [s0, s1) (stage indices) of block `blk`; `slot` is the
// segment's rank within the block: the partial-sum row it writes, and its
// place in the fixed summation order.
struct Seg {
  int32_t blk, s0, s1, slot;
};
static_assert(sizeof(Seg) == 16, "Seg layout");

struct WorkPlan {
  std::vector<Blk> blks;
  std::vector<Seg> segs;
  std::vector<int32_t> seg_off;  // [grid + n_dyn + 1]: piece k holds segs[seg_off[k] .. seg_off[k+1])
  std::vector<uint16_t> nsl;     // [N]: partial rows of each body (its block's nsplit)
  int rows = 1;                  // the largest nsplit
  int64_t grid = 0;              // static shares (one per CTA)
  int64_t n_dyn = 0;             // dynamic chunks
};

// offsets: [n_sys + 1] body offsets of the systems' targets; soff: [n_sys + 1]
// their stage offsets (the mixed stage pads every system to an even length).
// By default each system's sources are its targets' stage entries; with
// src_begin / src_count ([n_sys] each) system s takes the src_count[s]
// stage entries from src_begin[s] instead (a row shard: a block of targets
// against every source of the system).  slots: SMs x resident CTAs per SM
// the launch may use.  Returns an empty string on success, else the reason
// the plan cannot be made.
//
// cost (optional): the relative cost of each block's sources, piecewise
// constant over chunks of cost->chunk_units units: cost->w[k][c] is the
// weight of one unit of chunk c of block k (blocks as make_blocks returns
// them).  Without it every unit of a block weighs the warps the block keeps
// busy.  With it the line is cut into shares of equal cost, so on the mixed
// path, where a (warp, source group) pair costs 12 or 18 lane operations per
// interaction as the group is far or near, the shares still finish together.
struct ChunkCost {
  int64_t chunk_units = 1;
  std::vector<std::vector<int64_t>> w;
};

// The target blocks of each system: at most B = threads * ipt consecutive
// bodies, sizes balanced within the system; q0 = stage index of body i0.
inline std::vector<Blk> make_blocks(const std::vector<int64_t> &offsets, const std::vector<int64_t> &soff,
                                    int64_t B) {
  std::vector<Blk> out;
  const int64_t n_sys = static_cast<int64_t>(offsets.size()) - 1;
  for (int64_t s = 0; s < n_sys; ++s) {
    const int64_t b = offsets[s], e = offsets[s + 1], ns = e - b;
    const int64_t nb_s = (ns + B - 1) / B;
    for (int64_t k = 0; k < nb_s; ++k) {
      const int64_t i0 = b + ns * k / nb_s, i1 = b + ns * (k + 1) / nb_s;
      Blk blk;
      blk.i0 = static_cast<int32_t>(i0);
      blk.i1 = static_cast<int32_t>(i1);
      blk.q0 = static_cast<int32_t>(soff[s] + (i0 - b));
      blk.nsplit = 0;
      out.push_back(blk);
    }
  }
  return out;
}

inline std::string plan_work(const std::vector<int64_t> &offsets, const std::vector<int64_t> &soff, bool mixed,
                             int threads, int ipt, int jsplit, int64_t slots, WorkPlan &out,
                             const std::vector<int64_t> *src_begin = nullptr,
                             const std::vector<int64_t> *src_count = nullptr, const ChunkCost *cost = nullptr) {
  out = WorkPlan{};
  const int64_t n_sys = static_cast<int64_t>(offsets.size()) - 1;
  const int64_t B = static_cast<int64_t>(threads) * ipt;
  const int64_t unit = mixed ? 2 : 1;
  if (n_sys < 1 || B < 1 || slots < 1) return "empty work";
  out.blks = make_blocks(offsets, soff, B);
  if (cost && cost->w.size() != out.blks.size()) return "cost model does not match the blocks";
  // per block: first source, units, line length; with a cost
  // model also the line offset at the start of each chunk
  std::vector<int64_t> bj0, bunits, blen;
  std::vector<std::vector<int64_t>> pre;
  int64_t W = 0;
  {
    size_t k = 0;
    for (int64_t s = 0; s < n_sys; ++s) {
      const int64_t b = offsets[s], e = offsets[s + 1], ns = e - b;
      const int64_t sb = src_begin ? (*src_begin)[s] : soff[s];  // first source (stage entry)
      const int64_t sn = src_count ? (*src_count)[s] : ns;       // sources
      const int64_t len = (sn + unit - 1) / unit;  // units of this system's (padded) source range
      for (; k < out.blks.size() && out.blks[k].i0 < e; ++k) {
        const Blk &blk = out.blks[k];
        int64_t L;
        if (cost) {
          const std::vector<int64_t> &w = cost->w[k];
          const int64_t cu = cost->chunk_units, nch = (len + cu - 1) / cu;
          if (static_cast<int64_t>(w.size()) != nch) return "cost model does not match the sources";
          std::vector<int64_t> p(nch + 1, 0);
          for (int64_t c = 0; c < nch; ++c)
            p[c + 1] = p[c] + std::max<int64_t>(w[c], 1) * (std::min(len, (c + 1) * cu) - c * cu);
          L = p[nch];
          pre.push_back(std::move(p));
        } else {
          // warps with at least one target: warp w holds the block's targets
          // [32 ipt w, 32 ipt (w + 1))
          L = len * ((blk.i1 - blk.i0 + 32 * ipt - 1) / (32 * ipt));
        }
        bj0.push_back(sb);
        bunits.push_back(len);
        blen.push_back(L);
        W += L;
      }
    }
  }
  int64_t units_total = 0;
  for (int64_t u : bunits) units_total += u;
  // Pieces must not get too short: every piece of a block adds a partial row
  // that the per-body kernel adds for each of the block's bodies, and below a
  // few thousand bodies those sums (FP64 TwoSum at GB300's 1/64 FP64 rate, on
  // the FP64 path) cost more than the extra pieces gain in parallelism.  A
  // piece gets at least c * sqrt(U) units, U the longest block's units: c = 1/2
  // for mixed; for FP64 c = 1 below 800 units, 2 below 2000, 3 beyond (the
  // best of c = 1, 1.5, 2, 3 measured from 65 to 5,003 bodies; from about
  // 5,000 bodies on the shares are longer than that anyway).
  int64_t umax = 1;
  for (int64_t u : bunits) umax = std::max(umax, u);
  const double cmin = mixed ? 0.5 : umax < 800 ? 1.0 : umax < 2000 ? 2.0 : 3.0;
  const int64_t umin = std::max<int64_t>(1, static_cast<int64_t>(std::ceil(cmin * std::sqrt(static_cast<double>(umax)))));
  const int64_t G = std::max<int64_t>(1, std::min<int64_t>(units_total / umin, slots));
  const int64_t D = std::min<int64_t>(static_cast<int64_t>(jsplit) * G, std::max<int64_t>(units_total - G, 0));
  // Unit boundary of position x of block k's line (the same rounding for
  // both neighbours of a cut, so segments tile each block exactly).
  auto cut = [&](size_t k, int64_t x) -> int64_t {
    const int64_t off = std::min(std::max<int64_t>(x, 0), blen[k]);
    if (!cost) {
      const int64_t bw = blen[k] / bunits[k];
      return (off + bw / 2) / bw;
    }
    const std::vector<int64_t> &p = pre[k];
    const int64_t c = std::max<int64_t>(0, (std::upper_bound(p.begin(), p.end(), off) - p.begin()) - 1);
    if (c >= static_cast<int64_t>(p.size()) - 1) return bunits[k];
    const int64_t w = std::max<int64_t>(cost->w[k][c], 1);
    return std::min(bunits[k], c * cost->chunk_units + (off - p[c] + w / 2) / w);
  };
  // The static line: the first three quarters of every block's line (all of
  // it without dynamic chunks), block after block; then the dynamic line:
  // the remaining quarter of every block's line.  So every block gets a
  // share of the dynamic chunks, and its bodies about as many partial rows
  // as any other block's.
  struct Span {
    size_t k;
    int64_t a, b;  // positions [a, b) of block k's line
  };
  std::vector<Span> spans;
  for (size_t k = 0; k < out.blks.size(); ++k) spans.push_back({k, 0, D > 0 ? blen[k] - blen[k] / 4 : blen[k]});
  int64_t Ws = 0;
  for (const Span &sp : spans) Ws += sp.b - sp.a;
  if (D > 0)
    for (size_t k = 0; k < out.blks.size(); ++k) spans.push_back({k, blen[k] - blen[k] / 4, blen[k]});
  std::vector<int64_t> cuts;  // piece boundaries on the concatenated line
  for (int64_t g = 0; g <= G; ++g) cuts.push_back(Ws * g / G);
  for (int64_t d = 1; d <= D; ++d) cuts.push_back(Ws + (W - Ws) * d / D);
  const int64_t P = static_cast<int64_t>(cuts.size()) - 1;
  out.seg_off.assign(P + 1, 0);
  size_t i = 0;
  int64_t at = 0;  // line position of span i
  for (int64_t g = 0; g < P; ++g) {
    const int64_t lo = cuts[g], hi = cuts[g + 1];
    out.seg_off[g] = static_cast<int32_t>(out.segs.size());
    while (i < spans.size() && at + (spans[i].b - spans[i].a) <= lo) {
      at += spans[i].b - spans[i].a;
      ++i;
    }
    int64_t at_j = at;
    for (size_t j = i; j < spans.size() && at_j < hi; at_j += spans[j].b - spans[j].a, ++j) {
      const Span &sp = spans[j];
      const int64_t x0 = sp.a + std::max<int64_t>(lo - at_j, 0), x1 = sp.a + std::min(hi - at_j, sp.b - sp.a);
      const int64_t u0 = cut(sp.k, x0), u1 = cut(sp.k, x1);
      if (u1 <= u0) continue;
      Seg sg;
      sg.blk = static_cast<int32_t>(sp.k);
      sg.s0 = static_cast<int32_t>(bj0[sp.k] + u0 * unit);
      sg.s1 = static_cast<int32_t>(bj0[sp.k] + std::min(u1 * unit, bunits[sp.k] * unit));
      sg.slot = out.blks[sp.k].nsplit++;
      out.segs.push_back(sg);
    }
  }
  out.seg_off[P] = static_cast<int32_t>(out.segs.size());
  // Per body: how many partial rows its block has.
  out.nsl.assign(static_cast<size_t>(offsets[n_sys]), 0);
  out.rows = 1;
  for (const Blk &k : out.blks) {
    out.rows = std::max(out.rows, static_cast<int>(k.nsplit));
    for (int32_t p = k.i0; p < k.i1; ++p) out.nsl[p] = static_cast<uint16_t>(k.nsplit);
  }
  if (out.rows > 65535) return "too many source splits (" + std::to_string(out.rows) + ")";
  out.grid = G;
  out.n_dyn = D;
  return "";
}

}  // namespace nb
