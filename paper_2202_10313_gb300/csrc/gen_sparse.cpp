// Build-time generator of the sparse operator products of k_predict_sp (ahead-of-time
// specialisation, the GPU counterpart of the paper's generated sparse kernels, Sec. IV-A
// "all sparsity" and Sec. IV-B).
//
// The reference operators of one order are fixed numbers: the stiffness matrices K_c and
// the face matrices F~_i (Sec. III-A) in the orthonormal basis, computed here in FP64 by
// the library's own exact polynomial integration (host_basis.cpp) and rounded to FP32 as
// the device tables are. Their entries that vanish in exact arithmetic (the integration
// leaves them at <= 1e-10 of the largest; every true entry is >= 1e-3 of it) are left out,
// and every remaining entry becomes an immediate operand of a fused multiply-add. One GPU
// thread holds one row (one quantity of one element) of the operand in registers and
// forms all products of that row; the products are split into NPART parts of nearly equal
// multiply-add count, and a warp executes one part, so every thread of a warp runs the same
// straight-line code (no divergence) and no operator entry is read from memory. A part is a
// contiguous run of the outputs ordered by mode, so its outputs share most of their inputs
// and a thread loads only the inputs its part uses.
//
// Emitted, per order O and part count P (O = 3, 4, 5 with P = 1, 2, 4):
//   sp_time_o{O}(part, variant, x, y): Y_c[b] = sum_k x[k] K_c[b][k]        (time kernel,
//       d^{d+1}Q from d^dQ; K_c[b][k] != 0 only for deg b < deg k). Variant v takes only
//       the modes k < nbasis(O - v) and outputs b < nbasis(O - 1 - v) (the elastic time
//       kernel's degree truncation at derivative v; v = 0 is the full product).
//   sp_vol_o{O}(part, x, y, g): Z_c[b] = sum_k x[k] K_c[k][b] (volume kernel) and
//       G_i[f] = sum_k x[k] F~_i[k][f] (local face traces), from the same row.
//   sp_proj_o{O}(part, x, y): P_i[b] = sum_f x[i F + f] F^_i[f][b] (projection of one row of
//       the four faces' interface states, F^_i = F~_i^T in the orthonormal face basis).
//   sp_ntrace_o{O}(j, x, y): G_j[f] = sum_k x[k] F~_j[k][f] of one row of a neighbour's
//       buffer on the face j that each thread asks for (neighbour kernel).
// and for the reverse predict pass of the discrete adjoint (k_adj_pred_sp):
//   sp_trace_o{O}(part, x, g): G_i[f] = sum_k x[k] F~_i[k][f] alone (the traces of sp_vol).
//   sp_tproj_o{O}(part, x, y): y[b] = sum_i sum_f x[i F + f] F~_i[b][f] (the transposed face
//       traces of the four faces, summed).
//   sp_kvol_o{O}(part, variant, x, y): Z_c[b] = sum_k x[k] K_c[k][b] for 1 <= b < nbasis(O - v)
//       (the reverse time kernel at level v; K_c[k][b] != 0 only for deg k < deg b, so the
//       inputs are k < nbasis(O - 1 - v)).
// x[k * XP] is the thread's row, y[(c B + b) XP] (or y[(i B + b) XP]) and g[(i F + f) XP]
// the outputs (XP the pair stride of the staging arrays, a template parameter so that
// every address is an immediate offset). Every output the kernel reads is written
// (identically zero ones as 0); Z_c[0], which vanishes for every c, is not.
//
// Usage: gen_sparse <out.cuh>      writes the header
//        gen_sparse --list <order> lists every product term, one line each:
//        "<kind> <part> <output> <input> <value>", kind t (time kernel, output c B + b, full
//        variant), v (volume, output c B + b), g (face trace, output i F + f), p (face
//        projection, output i B + b, input i F + f), n (neighbour face trace, output j F + f),
//        s (summed transposed traces, output b, input i F + f) or k (reverse time kernel,
//        output c B + b, full variant); for checks against other operators.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "host.h"

namespace {

struct Out {
  char kind;                             // t, v, g, p, n
  int id;                                // output index within its kind
  std::string dst;                       // store expression
  std::vector<std::pair<int, float>> t;  // (input index, value), ascending input
};

using Parts = std::vector<std::vector<int>>;

// Parts of nearly equal multiply-add count (a store counts as one), each a contiguous run
// of the outputs in the given order.
Parts partition(const std::vector<Out>& outs, int nparts, const std::vector<int>& order) {
  size_t total = 0;
  for (int o : order) total += outs[o].t.size() + 1;
  Parts parts(nparts);
  size_t acc = 0;
  int p = 0;
  for (int o : order) {
    const size_t w = outs[o].t.size() + 1;
    // move on when this output would take the part further past its share than short of it
    if (p + 1 < nparts && acc + w / 2 > (size_t)(p + 1) * total / nparts) ++p;
    parts[p].push_back(o);
    acc += w;
  }
  return parts;
}

int nb(int o) { return o * (o + 1) * (o + 2) / 6; }

// All products of one order: time-kernel variants, volume + face traces, face projection.
struct Products {
  int O = 0, B = 0, F = 0, nparts = 1;
  std::vector<std::vector<Out>> time;    // per variant
  std::vector<Parts> time_parts;
  std::vector<Out> vol;                  // Z_c (b >= 1) then G_i
  Parts vol_parts;
  std::vector<Out> proj;
  Parts proj_parts;
  std::vector<std::vector<Out>> ntrace;  // per face j: the F outputs G_j[f]
  std::vector<Out> trace;                // G_i alone
  Parts trace_parts;
  std::vector<Out> tproj;                // sum over faces of the transposed traces
  Parts tproj_parts;
  std::vector<std::vector<Out>> kvol;    // reverse time kernel, per level
  std::vector<Parts> kvol_parts;
  size_t time_terms = 0, vol_terms = 0, face_terms = 0;

  void build(int order, int np) {
    O = order;
    nparts = np;
    lts::RefOps ops;
    ops.build(O);
    B = ops.B;
    F = ops.F;
    double kmax = 0.0, fmax = 0.0;
    for (int c = 0; c < 3; ++c)
      for (double v : ops.K[c]) kmax = std::max(kmax, std::fabs(v));
    for (int i = 0; i < 4; ++i)
      for (double v : ops.Ft[i]) fmax = std::max(fmax, std::fabs(v));
    auto nzk = [&](double v) { return std::fabs(v) > 1e-7 * kmax; };
    auto nzf = [&](double v) { return std::fabs(v) > 1e-7 * fmax; };
    auto dst = [](const char* arr, int idx) {
      char d[64];
      std::snprintf(d, sizeof d, "%s[%d * XP]", arr, idx);
      return std::string(d);
    };
    // time kernel variants; outputs (c, b) ordered by mode b, then c
    for (int v = 0; v <= O - 2; ++v) {
      const int kend = nb(O - v), bend = nb(O - 1 - v);
      std::vector<Out> outs;
      std::vector<int> ord;
      for (int b = 0; b < bend; ++b)
        for (int c = 0; c < 3; ++c) {
          Out u{'t', c * B + b, dst("y", c * B + b), {}};
          for (int k = 0; k < kend; ++k)
            if (nzk(ops.K[c][b * B + k])) u.t.push_back({k, (float)ops.K[c][b * B + k]});
          if (v == 0) time_terms += u.t.size();
          ord.push_back((int)outs.size());
          outs.push_back(u);
        }
      time_parts.push_back(partition(outs, nparts, ord));
      time.push_back(outs);
    }
    // volume (by mode b, then c) and face traces (by face mode f, then face i)
    std::vector<int> ord;
    for (int b = 0; b < B; ++b)
      for (int c = 0; c < 3; ++c) {
        Out u{'v', c * B + b, dst("y", c * B + b), {}};
        for (int k = 0; k < B; ++k)
          if (nzk(ops.K[c][k * B + b])) u.t.push_back({k, (float)ops.K[c][k * B + b]});
        vol_terms += u.t.size();
        if (b == 0) {   // the constant mode has no derivative: Z_c[0] = 0, not read
          if (!u.t.empty()) throw std::runtime_error("K_c[k][0] must vanish");
          continue;
        }
        ord.push_back((int)vol.size());
        vol.push_back(u);
      }
    for (int m = 0; m < F; ++m)
      for (int i = 0; i < 4; ++i) {
        Out u{'g', i * F + m, dst("g", i * F + m), {}};
        for (int k = 0; k < B; ++k)
          if (nzf(ops.Ft[i][k * F + m])) u.t.push_back({k, (float)ops.Ft[i][k * F + m]});
        face_terms += u.t.size();
        ord.push_back((int)vol.size());
        vol.push_back(u);
      }
    vol_parts = partition(vol, nparts, ord);
    // face projection, outputs (i, b) by face, then mode: F^_i[f][b] = F~_i[b][f]
    ord.clear();
    for (int i = 0; i < 4; ++i)
      for (int b = 0; b < B; ++b) {
        Out u{'p', i * B + b, dst("y", i * B + b), {}};
        for (int m = 0; m < F; ++m)
          if (nzf(ops.Ft[i][b * F + m])) u.t.push_back({i * F + m, (float)ops.Ft[i][b * F + m]});
        ord.push_back((int)proj.size());
        proj.push_back(u);
      }
    proj_parts = partition(proj, nparts, ord);
    // face traces of a neighbour's buffer on its face j (one face per thread, chosen at run
    // time): G_j[f] = sum_k x[k] F~_j[k][f]
    for (int j = 0; j < 4; ++j) {
      std::vector<Out> outs;
      for (int m = 0; m < F; ++m) {
        Out u{'n', j * F + m, dst("y", m), {}};
        for (int k = 0; k < B; ++k)
          if (nzf(ops.Ft[j][k * F + m])) u.t.push_back({k, (float)ops.Ft[j][k * F + m]});
        outs.push_back(u);
      }
      ntrace.push_back(outs);
    }
    // adjoint products: the face traces alone (as in vol, by face mode then face)
    ord.clear();
    for (const Out& u : vol)
      if (u.kind == 'g') {
        ord.push_back((int)trace.size());
        trace.push_back(u);
      }
    trace_parts = partition(trace, nparts, ord);
    // y[b] = sum_{i, f} x[i F + f] F~_i[b][f], by mode
    ord.clear();
    for (int b = 0; b < B; ++b) {
      Out u{'s', b, dst("y", b), {}};
      for (int i = 0; i < 4; ++i)
        for (int m = 0; m < F; ++m)
          if (nzf(ops.Ft[i][b * F + m])) u.t.push_back({i * F + m, (float)ops.Ft[i][b * F + m]});
      ord.push_back((int)tproj.size());
      tproj.push_back(u);
    }
    tproj_parts = partition(tproj, nparts, ord);
    // Z_c[b] = sum_k x[k] K_c[k][b], 1 <= b < nbasis(O - v), by mode then c
    for (int v = 0; v <= O - 2; ++v) {
      std::vector<Out> outs;
      std::vector<int> o2;
      for (int b = 1; b < nb(O - v); ++b)
        for (int c = 0; c < 3; ++c) {
          Out u{'k', c * B + b, dst("y", c * B + b), {}};
          for (int k = 0; k < B; ++k)
            if (nzk(ops.K[c][k * B + b])) {
              if (k >= nb(O - 1 - v)) throw std::runtime_error("K_c[k][b] must vanish for deg k >= deg b");
              u.t.push_back({k, (float)ops.K[c][k * B + b]});
            }
          o2.push_back((int)outs.size());
          outs.push_back(u);
        }
      kvol_parts.push_back(partition(outs, nparts, o2));
      kvol.push_back(outs);
    }
  }
};

std::string flt(float v) {
  char b[64];
  std::snprintf(b, sizeof b, "%a", (double)v);
  return std::string(b) + "f";
}

// Straight-line body of one part: loads of the needed inputs, then one fma chain per
// output (terms in ascending input index, the order of the dense kernels), then its store.
void emit_part(FILE* f, const std::vector<Out>& outs, const std::vector<int>& part) {
  std::vector<int> need;
  for (int o : part)
    for (auto& t : outs[o].t) need.push_back(t.first);
  std::sort(need.begin(), need.end());
  need.erase(std::unique(need.begin(), need.end()), need.end());
  for (int k : need) std::fprintf(f, "    const float x%d = x[%d * XP];\n", k, k);
  for (int o : part) {
    const Out& u = outs[o];
    if (u.t.empty()) {   // identically zero output that the kernel reads
      std::fprintf(f, "    %s = 0.f;\n", u.dst.c_str());
      continue;
    }
    std::fprintf(f, "    {\n      float a = x%d * %s;\n", u.t[0].first, flt(u.t[0].second).c_str());
    for (size_t i = 1; i < u.t.size(); ++i)
      std::fprintf(f, "      a = fmaf(x%d, %s, a);\n", u.t[i].first, flt(u.t[i].second).c_str());
    std::fprintf(f, "      %s = a;\n    }\n", u.dst.c_str());
  }
}

void emit_dispatch(FILE* f, const char* name, const char* args, const char* call_args,
                   const std::vector<Parts>& parts_of_variant, const std::vector<std::vector<Out>>& outs_of_variant,
                   bool has_variant) {
  const int nv = (int)parts_of_variant.size();
  for (int v = 0; v < nv; ++v) {
    const auto& parts = parts_of_variant[v];
    for (size_t p = 0; p < parts.size(); ++p) {
      std::fprintf(f, "template <int XP>\n__device__ __forceinline__ void %s_v%d_p%zu(%s) {\n", name, v, p, args);
      emit_part(f, outs_of_variant[v], parts[p]);
      std::fprintf(f, "}\n");
    }
  }
  std::fprintf(f, "template <int XP>\n__device__ __forceinline__ void %s(int part%s, %s) {\n", name,
               has_variant ? ", int variant" : "", args);
  for (int v = 0; v < nv; ++v) {
    if (has_variant) std::fprintf(f, "  if (variant == %d) {\n", v);
    std::fprintf(f, "  switch (part) {\n");
    for (size_t p = 0; p < parts_of_variant[v].size(); ++p)
      std::fprintf(f, "    case %zu: %s_v%d_p%zu<XP>(%s); break;\n", p, name, v, p, call_args);
    std::fprintf(f, "    default: break;\n  }\n");
    if (has_variant) std::fprintf(f, "  return;\n  }\n");
  }
  std::fprintf(f, "}\n");
}

// sp_ntrace_o{O}(j, x, y): G_j[f] = sum_k x[k] F~_j[k][f] for the face j the thread asks for
// (j < 0: none). A warp computes the faces that any of its lanes asks for (warp-uniform
// branches; every lane of the warp must call it) and each lane stores its own face's F
// outputs y[f * XP].
void emit_ntrace(FILE* f, int O, const Products& P) {
  std::fprintf(f, "template <int XP>\n__device__ __forceinline__ void sp_ntrace_o%d(int j, const float* __restrict__ x, "
               "float* __restrict__ y) {\n", O);
  std::vector<int> need;
  for (auto& outs : P.ntrace)
    for (auto& u : outs)
      for (auto& t : u.t) need.push_back(t.first);
  std::sort(need.begin(), need.end());
  need.erase(std::unique(need.begin(), need.end()), need.end());
  for (int k : need) std::fprintf(f, "  const float x%d = x[%d * XP];\n", k, k);
  for (int j = 0; j < 4; ++j) {
    std::fprintf(f, "  if (__any_sync(0xffffffffu, j == %d)) {\n", j);
    const auto& outs = P.ntrace[j];
    for (size_t m = 0; m < outs.size(); ++m) {
      const Out& u = outs[m];
      if (u.t.empty()) {
        std::fprintf(f, "    const float a%zu = 0.f;\n", m);
        continue;
      }
      std::fprintf(f, "    float a%zu = x%d * %s;\n", m, u.t[0].first, flt(u.t[0].second).c_str());
      for (size_t i = 1; i < u.t.size(); ++i)
        std::fprintf(f, "    a%zu = fmaf(x%d, %s, a%zu);\n", m, u.t[i].first, flt(u.t[i].second).c_str(), m);
    }
    std::fprintf(f, "    if (j == %d) {\n", j);
    for (size_t m = 0; m < outs.size(); ++m) std::fprintf(f, "      %s = a%zu;\n", outs[m].dst.c_str(), m);
    std::fprintf(f, "    }\n  }\n");
  }
  std::fprintf(f, "}\n");
}

void emit_order(FILE* f, int O, int nparts) {
  Products P;
  P.build(O, nparts);
  std::fprintf(f, "// ---- order %d (B = %d, F = %d), %d parts\n", O, P.B, P.F, nparts);
  std::fprintf(f, "// multiply-adds per row: time kernel %zu (full variant), volume %zu, face traces %zu\n",
               P.time_terms, P.vol_terms, P.face_terms);
  std::fprintf(f, "constexpr int kSpTimeTerms_o%d = %zu, kSpVolTerms_o%d = %zu, kSpFaceTerms_o%d = %zu;\n", O,
               P.time_terms, O, P.vol_terms, O, P.face_terms);
  char nm[64];
  std::snprintf(nm, sizeof nm, "sp_time_o%d", O);
  emit_dispatch(f, nm, "const float* __restrict__ x, float* __restrict__ y", "x, y", P.time_parts, P.time, true);
  std::snprintf(nm, sizeof nm, "sp_vol_o%d", O);
  emit_dispatch(f, nm, "const float* __restrict__ x, float* __restrict__ y, float* __restrict__ g", "x, y, g",
                {P.vol_parts}, {P.vol}, false);
  std::snprintf(nm, sizeof nm, "sp_proj_o%d", O);
  emit_dispatch(f, nm, "const float* __restrict__ x, float* __restrict__ y", "x, y", {P.proj_parts}, {P.proj}, false);
  emit_ntrace(f, O, P);
  std::snprintf(nm, sizeof nm, "sp_trace_o%d", O);
  emit_dispatch(f, nm, "const float* __restrict__ x, float* __restrict__ g", "x, g", {P.trace_parts}, {P.trace},
                false);
  std::snprintf(nm, sizeof nm, "sp_tproj_o%d", O);
  emit_dispatch(f, nm, "const float* __restrict__ x, float* __restrict__ y", "x, y", {P.tproj_parts}, {P.tproj},
                false);
  std::snprintf(nm, sizeof nm, "sp_kvol_o%d", O);
  emit_dispatch(f, nm, "const float* __restrict__ x, float* __restrict__ y", "x, y", P.kvol_parts, P.kvol, true);
}

int parts_of(int O) { return O == 5 ? 4 : (O == 4 ? 2 : 1); }

int list_terms(int O) {
  Products P;
  P.build(O, parts_of(O));
  auto list = [](const std::vector<Out>& outs, const Parts& parts) {
    for (size_t p = 0; p < parts.size(); ++p)
      for (int o : parts[p])
        for (auto& x : outs[o].t)
          std::printf("%c %zu %d %d %.9e\n", outs[o].kind, p, outs[o].id, x.first, (double)x.second);
  };
  list(P.time[0], P.time_parts[0]);
  list(P.vol, P.vol_parts);
  list(P.proj, P.proj_parts);
  for (auto& outs : P.ntrace) {
    std::vector<int> all(outs.size());
    for (size_t i = 0; i < all.size(); ++i) all[i] = (int)i;
    list(outs, Parts{all});
  }
  list(P.tproj, P.tproj_parts);
  list(P.kvol[0], P.kvol_parts[0]);
  return 0;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc == 3 && std::strcmp(argv[1], "--list") == 0) {
    const int O = std::atoi(argv[2]);
    if (O < 3 || O > 5) return 2;
    return list_terms(O);
  }
  if (argc != 2) {
    std::fprintf(stderr, "usage: gen_sparse <out.cuh> | gen_sparse --list <order>\n");
    return 2;
  }
  FILE* f = std::fopen(argv[1], "w");
  if (!f) {
    std::perror(argv[1]);
    return 1;
  }
  std::fprintf(f, "// Generated at build time by gen_sparse.cpp from the reference operators: do not edit.\n");
  std::fprintf(f, "#pragma once\nnamespace ltssp {\n");
  for (int O = 3; O <= 5; ++O) emit_order(f, O, parts_of(O));
  std::fprintf(f, "}  // namespace ltssp\n");
  return std::fclose(f) == 0 ? 0 : 1;
}
