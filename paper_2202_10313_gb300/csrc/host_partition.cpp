// Weighted partitioning for distributed runs (Sec. V-C) and the face-local exchange plan.
//
// Element weights follow the paper: an element of cluster l (0-based) is updated
// 2^(N_c-1-l) times per macro step, and that is its weight. Faces are weighted by their
// communication volume per macro step: a face between clusters l_a and l_b carries one
// message per update of each side, 2^(N_c-1-l_a) + 2^(N_c-1-l_b). The paper hands these
// weights to a graph partitioner on the dual graph; here a recursive coordinate bisection
// of the element centroids at the weighted median (longest extent first) produces balanced
// parts, and a greedy boundary pass then moves elements across the cut where that lowers
// the face-weighted cut without breaking the balance tolerance.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "host_partition.h"

namespace lts {

namespace {

int64_t elem_weight(int32_t cl, int nc) { return int64_t(1) << (nc - 1 - cl); }

void rcb(const std::vector<double>& cen, const std::vector<int64_t>& w, std::vector<int64_t>& idx, size_t lo,
         size_t hi, int p0, int p1, std::vector<int32_t>& part) {
  if (hi <= lo) return;
  if (p1 - p0 == 1) {
    for (size_t i = lo; i < hi; ++i) part[idx[i]] = p0;
    return;
  }
  const int pl = (p1 - p0) / 2;
  double bmin[3] = {1e300, 1e300, 1e300}, bmax[3] = {-1e300, -1e300, -1e300};
  int64_t total = 0;
  for (size_t i = lo; i < hi; ++i) {
    const int64_t k = idx[i];
    for (int d = 0; d < 3; ++d) {
      bmin[d] = std::min(bmin[d], cen[3 * k + d]);
      bmax[d] = std::max(bmax[d], cen[3 * k + d]);
    }
    total += w[k];
  }
  int ax = 0;
  for (int d = 1; d < 3; ++d)
    if (bmax[d] - bmin[d] > bmax[ax] - bmin[ax]) ax = d;
  std::stable_sort(idx.begin() + lo, idx.begin() + hi, [&](int64_t a, int64_t b) {
    const double ca = cen[3 * a + ax], cb = cen[3 * b + ax];
    return ca < cb || (ca == cb && a < b);
  });
  // first position where the left side reaches its share of the weight
  const double target = (double)total * pl / (p1 - p0);
  int64_t acc = 0;
  size_t mid = lo;
  while (mid < hi && (double)(acc + w[idx[mid]]) <= target) acc += w[idx[mid++]];
  if (mid < hi && target - (double)acc > (double)(acc + w[idx[mid]]) - target) acc += w[idx[mid++]];
  rcb(cen, w, idx, lo, mid, p0, p0 + pl, part);
  rcb(cen, w, idx, mid, hi, p0 + pl, p1, part);
}

}  // namespace

void partition_elements(const Mesh& m, const std::vector<int32_t>& cluster, int nc, int n_parts,
                        std::vector<int32_t>& part, PartitionStats* stats) {
  const int64_t K = m.K;
  part.assign(K, 0);
  std::vector<int64_t> w(K);
  for (int64_t k = 0; k < K; ++k) w[k] = elem_weight(cluster[k], nc);
  if (n_parts > 1) {
    std::vector<double> cen(3 * K, 0.0);
    for (int64_t k = 0; k < K; ++k)
      for (int v = 0; v < 4; ++v)
        for (int d = 0; d < 3; ++d) cen[3 * k + d] += 0.25 * m.xyz[3 * m.tet[4 * k + v] + d];
    std::vector<int64_t> idx(K);
    std::iota(idx.begin(), idx.end(), 0);
    rcb(cen, w, idx, 0, K, 0, n_parts, part);
    // greedy boundary refinement, in element order, a few passes
    std::vector<int64_t> load(n_parts, 0);
    int64_t total = 0;
    for (int64_t k = 0; k < K; ++k) {
      load[part[k]] += w[k];
      total += w[k];
    }
    const double cap = 1.03 * (double)total / n_parts;
    for (int pass = 0; pass < 4; ++pass) {
      int64_t moved = 0;
      for (int64_t k = 0; k < K; ++k) {
        const int32_t p = part[k];
        // face-weighted connection of k to every part it touches
        int32_t cand[4];
        int64_t conn[4];
        int nc_ = 0;
        int64_t own = 0;
        for (int f = 0; f < 4; ++f) {
          const int64_t nb = m.nbr[4 * k + f];
          if (nb < 0) continue;
          const int64_t fw = w[k] + w[nb];
          if (part[nb] == p) {
            own += fw;
            continue;
          }
          int s = 0;
          while (s < nc_ && cand[s] != part[nb]) ++s;
          if (s == nc_) {
            cand[nc_] = part[nb];
            conn[nc_++] = 0;
          }
          conn[s] += fw;
        }
        int best = -1;
        int64_t gain = 0;
        for (int s = 0; s < nc_; ++s) {
          const int64_t g = conn[s] - own;
          if (g > gain && (double)(load[cand[s]] + w[k]) <= cap) {
            gain = g;
            best = s;
          }
        }
        if (best >= 0) {
          load[p] -= w[k];
          load[cand[best]] += w[k];
          part[k] = cand[best];
          ++moved;
        }
      }
      if (moved == 0) break;
    }
  }
  if (!stats) return;
  std::vector<int64_t> load(n_parts, 0);
  int64_t total = 0;
  for (int64_t k = 0; k < K; ++k) {
    load[part[k]] += w[k];
    total += w[k];
  }
  const double mean = (double)total / n_parts;
  stats->max_load = (double)*std::max_element(load.begin(), load.end()) / mean;
  stats->min_load = (double)*std::min_element(load.begin(), load.end()) / mean;
  stats->total_weight = (double)total;
  stats->cut_faces = 0;
  stats->msgs_per_macro = 0;
  stats->buffer_msgs_per_macro = 0;
  for (int64_t k = 0; k < K; ++k) {
    // faces of k whose neighbour lies in another part: k receives one message per update
    int32_t seen_part[4];
    int64_t seen_rate[4];
    int ns = 0;
    for (int f = 0; f < 4; ++f) {
      const int64_t nb = m.nbr[4 * k + f];
      if (nb < 0 || part[nb] == part[k]) continue;
      stats->cut_faces += 1;
      stats->msgs_per_macro += w[k];
      // the sender side of the same face: nb sends to part[k]; without compression nb would
      // send its buffer once per receiving part and receiver step
      int s = 0;
      while (s < ns && seen_part[s] != part[nb]) ++s;
      if (s == ns) {
        seen_part[ns] = part[nb];
        seen_rate[ns++] = 0;
      }
      seen_rate[s] = std::max(seen_rate[s], w[nb]);
    }
    for (int s = 0; s < ns; ++s) stats->buffer_msgs_per_macro += seen_rate[s];
  }
}

void cut_faces(const Mesh& m, const std::vector<int32_t>& part, const std::vector<int32_t>& cluster,
               std::vector<CutFace>& out) {
  out.clear();
  for (int64_t k = 0; k < m.K; ++k)
    for (int f = 0; f < 4; ++f) {
      const int64_t nb = m.nbr[4 * k + f];
      if (nb < 0 || part[nb] == part[k]) continue;
      CutFace c;
      c.recv_elem = k;
      c.recv_face = f;
      c.send_elem = nb;
      c.send_face = m.nbr_face[4 * k + f];
      c.orient = m.nbr_orient[4 * k + f];
      c.recv_part = part[k];
      c.send_part = part[nb];
      c.recv_cluster = cluster[k];
      out.push_back(c);
    }
  // message order: by (receiving part, sending part), then receiver cluster, element, face
  std::stable_sort(out.begin(), out.end(), [](const CutFace& a, const CutFace& b) {
    if (a.recv_part != b.recv_part) return a.recv_part < b.recv_part;
    if (a.send_part != b.send_part) return a.send_part < b.send_part;
    if (a.recv_cluster != b.recv_cluster) return a.recv_cluster < b.recv_cluster;
    if (a.recv_elem != b.recv_elem) return a.recv_elem < b.recv_elem;
    return a.recv_face < b.recv_face;
  });
}

}  // namespace lts
