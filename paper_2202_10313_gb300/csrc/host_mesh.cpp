// Element geometry, face matching and the (j, h) neighbour relation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "host.h"

namespace lts {

namespace {
const int kFaceV[4][3] = {{0, 2, 1}, {0, 1, 3}, {0, 3, 2}, {1, 2, 3}};

struct FaceRec {
  int64_t key[3];   // sorted vertex keys
  int32_t kind;     // 0 interior, 3 periodic
  int64_t elem;
  int8_t face;
  bool operator<(const FaceRec& o) const {
    return std::tie(kind, key[0], key[1], key[2], elem, face) <
           std::tie(o.kind, o.key[0], o.key[1], o.key[2], o.elem, o.face);
  }
  bool same_face(const FaceRec& o) const {
    return kind == o.kind && key[0] == o.key[0] && key[1] == o.key[1] && key[2] == o.key[2];
  }
};
}  // namespace

int build_mesh(Mesh& m, Error& err) {
  const int64_t K = m.K;
  m.detJ.assign(K, 0.0);
  m.J.assign(9 * K, 0.0);
  m.Jinv.assign(9 * K, 0.0);
  m.x0.assign(3 * K, 0.0);
  m.normal.assign(12 * K, 0.0);
  m.area.assign(4 * K, 0.0);
  m.dins.assign(K, 0.0);
  for (int64_t k = 0; k < K; ++k) {
    const double* v[4];
    for (int a = 0; a < 4; ++a) {
      int64_t id = m.tet[4 * k + a];
      if (id < 0 || id >= m.nv) { err = {-1, "vertex id out of range"}; return -1; }
      v[a] = &m.xyz[3 * id];
    }
    double* J = &m.J[9 * k];
    for (int d = 0; d < 3; ++d)
      for (int c = 0; c < 3; ++c) J[d * 3 + c] = v[c + 1][d] - v[0][d];
    double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                 J[2] * (J[3] * J[7] - J[4] * J[6]);
    if (!(det > 0.0)) { err = {-2, "tetrahedron " + std::to_string(k) + " has non-positive orientation"}; return -1; }
    m.detJ[k] = det;
    // inverse: Jinv[c][d] = dxi_c/dx_d (cofactor / det)
    double* Ji = &m.Jinv[9 * k];
    Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det;
    Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
    Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
    Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
    Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
    Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
    Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det;
    Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
    Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
    for (int d = 0; d < 3; ++d) m.x0[3 * k + d] = v[0][d];
    double asum = 0.0;
    for (int f = 0; f < 4; ++f) {
      const double* a = v[kFaceV[f][0]];
      const double* b = v[kFaceV[f][1]];
      const double* c = v[kFaceV[f][2]];
      double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
      double ln = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
      m.area[4 * k + f] = 0.5 * ln;
      for (int d = 0; d < 3; ++d) m.normal[12 * k + 3 * f + d] = cr[d] / ln;
      asum += 0.5 * ln;
    }
    m.dins[k] = 6.0 * (det / 6.0) / asum;
  }
  // vertex keys for periodic matching: position modulo the box
  std::vector<int64_t> pkey;
  if (m.periodic) {
    std::map<std::tuple<double, double, double>, int64_t> tab;
    pkey.resize(m.nv);
    for (int64_t i = 0; i < m.nv; ++i) {
      double c[3];
      for (int d = 0; d < 3; ++d) {
        double L = m.period[d];
        double x = std::fmod(m.xyz[3 * i + d], L);
        if (x < 0) x += L;
        if (x == L) x = 0.0;
        c[d] = x;
      }
      auto key = std::make_tuple(c[0], c[1], c[2]);
      auto it = tab.find(key);
      if (it == tab.end()) it = tab.emplace(key, (int64_t)tab.size()).first;
      pkey[i] = it->second;
    }
  }
  std::vector<FaceRec> recs;
  recs.reserve(4 * K);
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      int32_t bc = m.bc[4 * k + f];
      if (bc == 1 || bc == 2) continue;
      if (bc != 0 && bc != 3) { err = {-1, "bad face code"}; return -1; }
      if (bc == 3 && !m.periodic) { err = {-2, "periodic face without a period"}; return -1; }
      FaceRec r;
      r.kind = bc;
      r.elem = k;
      r.face = (int8_t)f;
      for (int a = 0; a < 3; ++a) {
        int64_t id = m.tet[4 * k + kFaceV[f][a]];
        r.key[a] = (bc == 3) ? pkey[id] : id;
      }
      std::sort(r.key, r.key + 3);
      recs.push_back(r);
    }
  std::sort(recs.begin(), recs.end());
  m.nbr.assign(4 * K, -1);
  m.nbr_face.assign(4 * K, -1);
  m.nbr_orient.assign(4 * K, -1);
  auto vkey = [&](int64_t k, int f, int a) {
    int64_t id = m.tet[4 * k + kFaceV[f][a]];
    return m.bc[4 * k + f] == 3 ? pkey[id] : id;
  };
  for (size_t i = 0; i < recs.size();) {
    size_t j = i;
    while (j < recs.size() && recs[j].same_face(recs[i])) ++j;
    if (j - i != 2) { err = {-2, "face shared by " + std::to_string(j - i) + " elements"}; return -1; }
    const FaceRec& A = recs[i];
    const FaceRec& Bf = recs[i + 1];
    for (int side = 0; side < 2; ++side) {
      const FaceRec& e = side ? Bf : A;
      const FaceRec& g = side ? A : Bf;
      int64_t ek[3], gk[3];
      for (int a = 0; a < 3; ++a) { ek[a] = vkey(e.elem, e.face, a); gk[a] = vkey(g.elem, g.face, a); }
      int h = -1;
      for (int a = 0; a < 3; ++a)
        if (gk[a] == ek[0]) h = a;
      if (h < 0 || gk[(h + 2) % 3] != ek[1] || gk[(h + 1) % 3] != ek[2]) {
        err = {-2, "inconsistent face orientation"};
        return -1;
      }
      m.nbr[4 * e.elem + e.face] = g.elem;
      m.nbr_face[4 * e.elem + e.face] = g.face;
      m.nbr_orient[4 * e.elem + e.face] = (int8_t)h;
    }
    i = j;
  }
  return 0;
}

int64_t locate(const Mesh& m, const double x[3], double xi_out[3]) {
  const double tol = 1e-12;
  for (int64_t k = 0; k < m.K; ++k) {
    const double* Ji = &m.Jinv[9 * k];
    const double* x0 = &m.x0[3 * k];
    double dx[3] = {x[0] - x0[0], x[1] - x0[1], x[2] - x0[2]};
    double xi[3];
    for (int c = 0; c < 3; ++c) xi[c] = Ji[c * 3 + 0] * dx[0] + Ji[c * 3 + 1] * dx[1] + Ji[c * 3 + 2] * dx[2];
    if (xi[0] >= -tol && xi[1] >= -tol && xi[2] >= -tol && 1.0 - xi[0] - xi[1] - xi[2] >= -tol) {
      for (int c = 0; c < 3; ++c) xi_out[c] = xi[c];
      return k;
    }
  }
  return -1;
}

}  // namespace lts
