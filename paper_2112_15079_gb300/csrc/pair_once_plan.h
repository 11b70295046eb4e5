// Block size of the pair-once force kernels (sym.cu, sym_mixed.cu) for a
// context, host side.  Plain C++ without CUDA, so the library and a CPU test
// build the same code.
//
// A body keeps one partial row (24 B) per block of its system, and the
// per-body kernel reads them every step; the block pairs (I, J), I <= J, are
// the work items.  The choice:
//   FP64 (bodies per block): 64 when every system has at most kSymMaxBodies
//   (rows <= 1.6 GB at 65,536); else the narrowest wide block (256 .. 4,096
//   bodies) whose rows fit in kSymRowBudget, else 4,096 if they fit in
//   kSymRowLimit (else none); used when the systems hold at least 1.5 block
//   pairs per SM (with fewer, one CTA carries a system's whole sum and the
//   stream-K kernel is faster: measured on GB300, 1,031 bodies / 153 pairs
//   60.8 against 55.3 us per step, 1,283 bodies / 231 pairs 62.5 against
//   96.2).
//   Mixed (stage entries per block): for a largest system of at least
//   kMsymMinBodies (measured on GB300: 65,536 bodies 1.63 against 1.82 ms
//   per step, 1,048,576 bodies 395 against 430 ms; 10,425 bodies 75 against
//   68 us, where the per-body kernel reads 82 rows per body and does not
//   overlap), the narrowest block (128 .. 2,048 entries) that leaves the
//   largest system at most kMsymMaxRows rows per body, if the rows fit in
//   kSymRowLimit and the block pairs give at least 8 warps per SM (each warp
//   holds 128 targets).
// A requested block size is used as asked (nbody_init checks its rows
// against kSymRowLimit and 65,535 blocks per system).
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace nb {

// FP64, 64-body blocks (force_sym_kernel): pairs (I, J), I <= J.
constexpr int kSymBlock = 64;
constexpr int kSymThreads = 64;       // two warps: one 32-body tile of block I each
constexpr int kSymMaxBodies = 65536;  // per system, by default (the partial rows are [blocks][3][N])
// FP64 wide blocks of 32 T bodies (force_sym_wide_kernel) above that: T tiles.
constexpr int kSymWideWarps = 4;
constexpr int kSymWideThreads = 32 * kSymWideWarps;
constexpr int kSymWideMinTiles = 8;    // 256 bodies
constexpr int kSymWideMaxTiles = 128;  // 4,096 bodies (96 KB of shared sums)
// Mixed blocks of 32 T stage entries (force_msym_kernel), W = T / 4 warps.
constexpr int kMsymMinTiles = 4;   // 128 entries: one warp's four target tiles
constexpr int kMsymMaxTiles = 64;  // 2,048 entries
constexpr int kMsymMaxWarps = kMsymMaxTiles / 4;

constexpr int64_t kSymRowBudget = int64_t(2) << 30;
constexpr int64_t kSymRowLimit = int64_t(16) << 30;
constexpr int64_t kMsymMaxRows = 128;
constexpr int64_t kMsymMinBodies = 65536;

// Rows per body of the largest system with blocks of B, and their bytes
// ([rows][3][N], 8 B per entry) for N bodies in all.
inline int64_t pair_once_rows(const std::vector<int64_t> &sizes, int64_t B) {
  int64_t rows = 1;
  for (int64_t n : sizes) rows = std::max(rows, (n + B - 1) / B);
  return rows;
}

inline int64_t pair_once_row_bytes(const std::vector<int64_t> &sizes, int64_t B) {
  int64_t N = 0;
  for (int64_t n : sizes) N += n;
  return pair_once_rows(sizes, B) * 3 * 8 * N;
}

// The block pairs (I, J), I <= J, of all systems.
inline int64_t pair_once_items(const std::vector<int64_t> &sizes, int64_t B) {
  int64_t pairs = 0;
  for (int64_t n : sizes) {
    const int64_t nb = (n + B - 1) / B;
    pairs += nb * (nb + 1) / 2;
  }
  return pairs;
}

// sizes: bodies per system; nsm: the GPU's SMs; requested: the caller's
// block size (0 = automatic).  Returns the block size, or 0 for the
// every-ordered-pair kernel.
inline int pair_once_block(const std::vector<int64_t> &sizes, bool mixed, int64_t nsm, int requested) {
  if (requested > 0) return requested;
  int64_t nmax = 0;
  for (int64_t n : sizes) nmax = std::max(nmax, n);
  if (mixed) {
    if (nmax < kMsymMinBodies) return 0;
    int64_t B = 32 * kMsymMinTiles;
    while (B < 32 * kMsymMaxTiles && pair_once_rows(sizes, B) > kMsymMaxRows) B *= 2;
    if (pair_once_row_bytes(sizes, B) > kSymRowLimit) return 0;
    return pair_once_items(sizes, B) * (B / 128) >= 8 * nsm ? static_cast<int>(B) : 0;
  }
  int64_t B = kSymBlock;
  if (nmax > kSymMaxBodies) {
    B = 32 * kSymWideMinTiles;
    while (B < 32 * kSymWideMaxTiles && pair_once_row_bytes(sizes, B) > kSymRowBudget) B *= 2;
    if (pair_once_row_bytes(sizes, B) > kSymRowLimit) return 0;
  }
  return 2 * pair_once_items(sizes, B) >= 3 * nsm ? static_cast<int>(B) : 0;
}

}  // namespace nb
