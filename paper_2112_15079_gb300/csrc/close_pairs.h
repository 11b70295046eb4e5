// Close pairs and their clusters for close-encounter handling (host side).
// Plain C++ without CUDA, so the library and a CPU test build the same code.
//
// A pair of bodies p < j of one system is close when its two-body angular
// frequency w = sqrt(G (m_p + m_j) / d^3) gives w |dt| > theta_c, tested as
//   G (m_p + m_j) dt^2 > theta_c^2 d^3,   d^2 = dx^2 + dy^2 + dz^2,
//   (dx, dy, dz) = r_j - r_p,
// in FP64 in that order.  Bodies joined by close pairs form a cluster; a
// cluster takes k = max over its members of ceil(w_max |dt| / theta_s)
// sub-steps per step (at least 1; w_max: the member's fastest pair).
//
// The search avoids the all-pairs loop on large systems.  A close pair has
// d^3 < (m_p + m_j) K <= 2 max(m_p, m_j) K with K = G dt^2 / theta_c^2, so:
// the 64 heaviest bodies of the system are tested against every body, and
// the others against the bodies in the neighbouring cells of a grid whose
// cell is as wide as the largest such radius among them.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

namespace nb {

struct CloseSet {
  int64_t n_pairs = 0;
  int32_t k_max = 0;
  // Cluster c: members mem_body[cl_off[c] .. cl_off[c + 1]) in ascending
  // body order, k sub-steps cl_k[c].  Clusters are ordered by their first
  // body.
  std::vector<int32_t> cl_off{0}, cl_k, mem_body;
  // Pairs of cluster c: pr_off[c] .. pr_off[c + 1]; pair q joins members
  // pr_a[q] and pr_b[q] (indices into mem_body), body of a < body of b.
  std::vector<int32_t> pr_off{0}, pr_a, pr_b;
  // Member i's pairs: mp_pair[mp_off[i] .. mp_off[i + 1]), in ascending
  // order of the partner's body index.
  std::vector<int32_t> mp_off{0}, mp_pair;
};

// The close-pair test for p < j (see above); w receives the frequency.
inline bool close_pair(const double *x, const double *y, const double *z, const double *m, int64_t p, int64_t j,
                       double G, double dt2, double theta_c2, double &w) {
  const double dx = x[j] - x[p], dy = y[j] - y[p], dz = z[j] - z[p];
  const double d2 = dx * dx + dy * dy + dz * dz;
  const double d3 = d2 * std::sqrt(d2);
  if (!(G * (m[p] + m[j]) * dt2 > theta_c2 * d3)) return false;
  w = std::sqrt(G * (m[p] + m[j]) / d3);
  return true;
}

// Fill `out` for the systems [offsets[s], offsets[s + 1]).  Returns "" or the
// reason the set cannot be made (a cluster would need more than max_k
// sub-steps).
inline std::string find_close_set(int64_t n_sys, const int64_t *offsets, const double *x, const double *y,
                                  const double *z, const double *m, double G, double dt, double theta_c,
                                  double theta_s, CloseSet &out, int64_t max_k = 1000000) {
  out = CloseSet{};
  const double dt2 = dt * dt, tc2 = theta_c * theta_c, adt = std::fabs(dt);
  const double K = G * dt2 / tc2;
  std::vector<std::pair<int64_t, int64_t>> pairs;
  std::vector<double> pw;  // frequency of each pair
  auto test = [&](int64_t p, int64_t j) {
    double w = 0.0;
    if (close_pair(x, y, z, m, p, j, G, dt2, tc2, w)) {
      pairs.emplace_back(p, j);
      pw.push_back(w);
    }
  };
  for (int64_t s = 0; s < n_sys; ++s) {
    const int64_t b = offsets[s], e = offsets[s + 1], n = e - b;
    if (n <= 4096) {
      for (int64_t p = b; p < e; ++p)
        for (int64_t j = p + 1; j < e; ++j) test(p, j);
      continue;
    }
    // the 64 heaviest bodies (ties: lower index) against every body
    std::vector<int64_t> idx(static_cast<size_t>(n));
    std::iota(idx.begin(), idx.end(), b);
    const size_t nh = 64;
    std::partial_sort(idx.begin(), idx.begin() + nh, idx.end(),
                      [&](int64_t u, int64_t v) { return m[u] > m[v] || (m[u] == m[v] && u < v); });
    std::vector<char> heavy(static_cast<size_t>(n), 0);
    for (size_t i = 0; i < nh; ++i) heavy[idx[i] - b] = 1;
    for (size_t i = 0; i < nh; ++i) {
      const int64_t h = idx[i];
      for (int64_t j = b; j < e; ++j) {
        if (j == h || (heavy[j - b] && j < h)) continue;  // a heavy pair once, from its lower index
        test(std::min(h, j), std::max(h, j));
      }
    }
    // the rest among themselves, on a grid
    double mmax = 0.0, cmax = 0.0;
    for (int64_t p = b; p < e; ++p) {
      if (heavy[p - b]) continue;
      mmax = std::max(mmax, m[p]);
      cmax = std::max({cmax, std::fabs(x[p]), std::fabs(y[p]), std::fabs(z[p])});
    }
    if (!(mmax > 0.0)) continue;
    double cell = std::cbrt(2.0 * mmax * K) * 1.001;
    if (!(cell > 0.0) || !std::isfinite(cell)) continue;
    cell = std::max(cell, cmax * 1e-15);  // cell indices stay far inside int64
    std::unordered_map<uint64_t, std::vector<int64_t>> grid;
    auto ci = [&](double v) { return static_cast<int64_t>(std::floor(v / cell)); };
    auto key = [](int64_t i, int64_t j, int64_t k) {
      return static_cast<uint64_t>(i) * 0x9E3779B97F4A7C15ull ^ static_cast<uint64_t>(j) * 0xC2B2AE3D27D4EB4Full ^
             static_cast<uint64_t>(k) * 0x165667B19E3779F9ull;
    };
    for (int64_t p = b; p < e; ++p)
      if (!heavy[p - b]) grid[key(ci(x[p]), ci(y[p]), ci(z[p]))].push_back(p);
    std::vector<int64_t> cand;
    for (int64_t p = b; p < e; ++p) {
      if (heavy[p - b]) continue;
      const int64_t i0 = ci(x[p]), j0 = ci(y[p]), k0 = ci(z[p]);
      cand.clear();
      for (int64_t di = -1; di <= 1; ++di)
        for (int64_t dj = -1; dj <= 1; ++dj)
          for (int64_t dk = -1; dk <= 1; ++dk) {
            const auto it = grid.find(key(i0 + di, j0 + dj, k0 + dk));
            if (it == grid.end()) continue;
            for (int64_t j : it->second)
              if (j > p) cand.push_back(j);
          }
      std::sort(cand.begin(), cand.end());  // hash collisions may list a body twice
      cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
      for (int64_t j : cand) test(p, j);
    }
  }
  out.n_pairs = static_cast<int64_t>(pairs.size());
  if (pairs.empty()) return "";
  // clusters: union-find over the pairs
  const int64_t N = offsets[n_sys];
  std::vector<int64_t> parent(static_cast<size_t>(N));
  std::iota(parent.begin(), parent.end(), 0);
  auto find = [&](int64_t i) {
    while (parent[i] != i) {
      parent[i] = parent[parent[i]];
      i = parent[i];
    }
    return i;
  };
  std::vector<double> wmax(static_cast<size_t>(N), 0.0);
  for (size_t q = 0; q < pairs.size(); ++q) {
    const int64_t p = pairs[q].first, j = pairs[q].second;
    parent[find(p)] = find(j);
    wmax[p] = std::max(wmax[p], pw[q]);
    wmax[j] = std::max(wmax[j], pw[q]);
  }
  // members grouped by cluster, clusters by their first body
  std::vector<int64_t> members;
  for (const auto &pq : pairs) {
    members.push_back(pq.first);
    members.push_back(pq.second);
  }
  std::sort(members.begin(), members.end());
  members.erase(std::unique(members.begin(), members.end()), members.end());
  std::vector<int64_t> first_of_root(static_cast<size_t>(N), -1);
  for (int64_t p : members)
    if (first_of_root[find(p)] < 0) first_of_root[find(p)] = p;
  std::stable_sort(members.begin(), members.end(),
                   [&](int64_t u, int64_t v) { return first_of_root[find(u)] < first_of_root[find(v)]; });
  std::vector<int32_t> slot(static_cast<size_t>(N), -1);  // member index of each body
  for (size_t i = 0; i < members.size(); ++i) {
    const int64_t p = members[i];
    slot[p] = static_cast<int32_t>(i);
    out.mem_body.push_back(static_cast<int32_t>(p));
    const bool last = i + 1 == members.size() || find(members[i + 1]) != find(p);
    if (last) out.cl_off.push_back(static_cast<int32_t>(i + 1));
  }
  const size_t nc = out.cl_off.size() - 1;
  out.cl_k.assign(nc, 1);
  for (size_t c = 0; c < nc; ++c)
    for (int32_t i = out.cl_off[c]; i < out.cl_off[c + 1]; ++i) {
      const double kd = std::ceil(wmax[out.mem_body[i]] * adt / theta_s);
      if (!(kd <= static_cast<double>(max_k)))
        return "a close pair would need more than " + std::to_string(max_k) + " sub-steps per step";
      out.cl_k[c] = std::max(out.cl_k[c], std::max(1, static_cast<int32_t>(kd)));
    }
  for (int32_t k : out.cl_k) out.k_max = std::max(out.k_max, k);
  // pairs by cluster (ordered by member indices), and each member's pairs by partner body
  std::vector<size_t> order(pairs.size());
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](size_t u, size_t v) {
    const int32_t au = slot[pairs[u].first], av = slot[pairs[v].first];
    return au < av || (au == av && slot[pairs[u].second] < slot[pairs[v].second]);
  });
  std::vector<int32_t> cluster_of(members.size());
  for (size_t c = 0; c < nc; ++c)
    for (int32_t i = out.cl_off[c]; i < out.cl_off[c + 1]; ++i) cluster_of[i] = static_cast<int32_t>(c);
  std::vector<std::vector<std::pair<int64_t, int32_t>>> mine(members.size());  // (partner body, pair)
  size_t q = 0;
  for (size_t c = 0; c < nc; ++c) {
    while (q < order.size() && cluster_of[slot[pairs[order[q]].first]] == static_cast<int32_t>(c)) {
      const auto &pq = pairs[order[q]];
      const int32_t id = static_cast<int32_t>(out.pr_a.size());
      out.pr_a.push_back(slot[pq.first]);
      out.pr_b.push_back(slot[pq.second]);
      mine[slot[pq.first]].emplace_back(pq.second, id);
      mine[slot[pq.second]].emplace_back(pq.first, id);
      ++q;
    }
    out.pr_off.push_back(static_cast<int32_t>(out.pr_a.size()));
  }
  for (auto &v : mine) {
    std::sort(v.begin(), v.end());
    for (const auto &e : v) out.mp_pair.push_back(e.second);
    out.mp_off.push_back(static_cast<int32_t>(out.mp_pair.size()));
  }
  return "";
}

}  // namespace nb
