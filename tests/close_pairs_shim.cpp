// Test-only C entry point over the library's host close-pair finder
// (paper_2112_15079_gb300/csrc/close_pairs.h).  tests/test_close_pairs.py
// builds it with g++ and checks it against a brute-force search on the CPU.
#include <cstdint>
#include <cstring>
#include <string>

#include "close_pairs.h"

// Fills the close pairs as (body, body) into pairs[2 * cap] and, per body,
// its cluster id (-1: none) and its cluster's sub-step count; meta = [pairs,
// clusters, members, k_max].  Returns 0, 1 if the finder refused, 2 if cap
// is too small, 3 if the member pair lists are not in partner order.
extern "C" int cp_find(int64_t n_sys, const int64_t *offsets, const double *x, const double *y, const double *z,
                       const double *m, double G, double dt, double theta_c, double theta_s, int64_t cap,
                       int64_t *pairs, int32_t *cluster, int32_t *kc, int64_t *meta) {
  nb::CloseSet cs;
  if (!nb::find_close_set(n_sys, offsets, x, y, z, m, G, dt, theta_c, theta_s, cs).empty()) return 1;
  meta[0] = cs.n_pairs;
  meta[1] = static_cast<int64_t>(cs.cl_k.size());
  meta[2] = static_cast<int64_t>(cs.mem_body.size());
  meta[3] = cs.k_max;
  if (static_cast<int64_t>(cs.pr_a.size()) > cap) return 2;
  for (size_t q = 0; q < cs.pr_a.size(); ++q) {
    pairs[2 * q] = cs.mem_body[cs.pr_a[q]];
    pairs[2 * q + 1] = cs.mem_body[cs.pr_b[q]];
  }
  const int64_t N = offsets[n_sys];
  for (int64_t p = 0; p < N; ++p) cluster[p] = -1, kc[p] = 0;
  for (size_t c = 0; c + 1 < cs.cl_off.size(); ++c)
    for (int32_t i = cs.cl_off[c]; i < cs.cl_off[c + 1]; ++i) {
      cluster[cs.mem_body[i]] = static_cast<int32_t>(c);
      kc[cs.mem_body[i]] = cs.cl_k[c];
      int64_t last = -1;
      for (int32_t e = cs.mp_off[i]; e < cs.mp_off[i + 1]; ++e) {
        const int32_t q = cs.mp_pair[e];
        const int64_t other = cs.mem_body[cs.pr_a[q]] == cs.mem_body[i] ? cs.mem_body[cs.pr_b[q]] : cs.mem_body[cs.pr_a[q]];
        if (other <= last) return 3;
        last = other;
      }
    }
  return 0;
}
