// Test-only C entry points over the library's pair-once block choice
// (paper_2112_15079_gb300/csrc/pair_once_plan.h).  tests/test_pair_once_plan.py
// builds it with g++ and checks the choice on the CPU; no CUDA involved.
#include <cstdint>
#include <vector>

#include "pair_once_plan.h"

extern "C" int po_block(const int64_t *sizes, int64_t n_sys, int mixed, int64_t nsm, int requested) {
  const std::vector<int64_t> v(sizes, sizes + n_sys);
  return nb::pair_once_block(v, mixed != 0, nsm, requested);
}

extern "C" int64_t po_row_bytes(const int64_t *sizes, int64_t n_sys, int64_t block) {
  const std::vector<int64_t> v(sizes, sizes + n_sys);
  return nb::pair_once_row_bytes(v, block);
}
