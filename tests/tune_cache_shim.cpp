// Test-only C entry points over the library's autotuner cache
// (paper_2112_15079_gb300/csrc/tune_cache.h).  tests/test_tune_cache.py
// builds this with g++ and checks the file round trip and the handling of
// damaged files on the CPU; no CUDA involved.
#include <string>

#include "tune_cache.h"

namespace {
nb::TuneKey key_of(int precision, int integrator, int n_log2, int systems_log2, int sms, const char *kernels) {
  nb::TuneKey k;
  k.precision = precision;
  k.integrator = integrator;
  k.n_log2 = n_log2;
  k.systems_log2 = systems_log2;
  k.sms = sms;
  k.kernels = kernels;
  return k;
}
}  // namespace

// tiles[5] = threads, ipt, tj, jsplit, ctas_per_sm.  Returns 0 on success.
extern "C" int tc_store(const char *path, int precision, int integrator, int n_log2, int systems_log2, int sms,
                        const char *kernels, const int *tiles, double ms) {
  nb::TuneEntry e;
  e.threads = tiles[0];
  e.ipt = tiles[1];
  e.tj = tiles[2];
  e.jsplit = tiles[3];
  e.ctas_per_sm = tiles[4];
  e.ms_per_step = ms;
  return nb::tune_cache_store(path, key_of(precision, integrator, n_log2, systems_log2, sms, kernels), e).empty() ? 0
                                                                                                                   : 1;
}

// Returns 1 and fills tiles[5], *ms if the file holds the entry, else 0.
extern "C" int tc_lookup(const char *path, int precision, int integrator, int n_log2, int systems_log2, int sms,
                         const char *kernels, int *tiles, double *ms) {
  nb::TuneEntry e;
  if (!nb::tune_cache_lookup(path, key_of(precision, integrator, n_log2, systems_log2, sms, kernels), e)) return 0;
  tiles[0] = e.threads;
  tiles[1] = e.ipt;
  tiles[2] = e.tj;
  tiles[3] = e.jsplit;
  tiles[4] = e.ctas_per_sm;
  *ms = e.ms_per_step;
  return 1;
}

extern "C" int tc_floor_log2(long long v) { return nb::floor_log2(v); }
