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
// straight-line code (no divergence) and no operator entry is read from memory.
//
// Emitted, per order O and part count P (O = 3, 4, 5 with P = 1, 2, 4):
//   sp_time_o{O}(part, variant, x, y): Y_c[b] = sum_k x[k] K_c[b][k]        (time kernel,
//       d^{d+1}Q from d^dQ; K_c[b][k] != 0 only for deg b < deg k). Variant v takes only
//       the modes k < nbasis(O - v) and outputs b < nbasis(O - 1 - v) (the elastic time
//       kernel's degree truncation at derivative v; v = 0 is the full product).
//   sp_vol_o{O}(part, x, y, g): Z_c[b] = sum_k x[k] K_c[k][b] (volume kernel) and
//       G_i[f] = sum_k x[k] F~_i[k][f] (local face traces), from the same row.
// x[k * XP] is the thread's row, y[(c B + b) XP], g[(i F + f) XP] the outputs (XP the pair
// stride of the staging arrays, a template parameter so that every address is an
// immediate offset). Every output the kernel reads is written (identically zero ones as
// 0); Z_c[0], which vanishes for every c, is not.
//
// Usage: gen_sparse <out.cuh>
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
  std::string dst;                       // store expression (relative to y or g)
  std::vector<std::pair<int, float>> t;  // (k, value), ascending k
};

std::string flt(float v) {
  char b[64];
  std::snprintf(b, sizeof b, "%a", (double)v);
  return std::string(b) + "f";
}

// Greedy balance: outputs in descending term count, each to the part with the fewest terms.
std::vector<std::vector<int>> partition(const std::vector<Out>& outs, int nparts) {
  std::vector<int> order(outs.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return outs[a].t.size() > outs[b].t.size(); });
  std::vector<std::vector<int>> parts(nparts);
  std::vector<size_t> load(nparts, 0);
  for (int o : order) {
    int best = 0;
    for (int p = 1; p < nparts; ++p)
      if (load[p] < load[best]) best = p;
    parts[best].push_back(o);
    load[best] += outs[o].t.size();
  }
  for (auto& p : parts) std::sort(p.begin(), p.end());
  return parts;
}

// Straight-line body of one part: loads of the needed row entries, then one fma chain per
// output (terms in ascending k, the order of the dense kernels), then its store.
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
                   const std::vector<std::vector<std::vector<int>>>& parts_of_variant,
                   const std::vector<std::vector<Out>>& outs_of_variant, bool has_variant) {
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

void emit_order(FILE* f, int O, int nparts) {
  lts::RefOps ops;
  ops.build(O);
  const int B = ops.B, F = ops.F;
  double kmax = 0.0, fmax = 0.0;
  for (int c = 0; c < 3; ++c)
    for (double v : ops.K[c]) kmax = std::max(kmax, std::fabs(v));
  for (int i = 0; i < 4; ++i)
    for (double v : ops.Ft[i]) fmax = std::max(fmax, std::fabs(v));
  auto nzk = [&](double v) { return std::fabs(v) > 1e-7 * kmax; };
  auto nzf = [&](double v) { return std::fabs(v) > 1e-7 * fmax; };
  auto nb = [](int o) { return o * (o + 1) * (o + 2) / 6; };
  std::fprintf(f, "// ---- order %d (B = %d, F = %d), %d parts\n", O, B, F, nparts);
  // time kernel variants
  std::vector<std::vector<Out>> tv;
  std::vector<std::vector<std::vector<int>>> tp;
  size_t terms0 = 0;
  for (int v = 0; v <= O - 2; ++v) {
    const int kend = nb(O - v), bend = nb(O - 1 - v);
    std::vector<Out> outs;
    for (int c = 0; c < 3; ++c)
      for (int b = 0; b < bend; ++b) {
        Out u;
        char d[64];
        std::snprintf(d, sizeof d, "y[%d * XP]", c * B + b);
        u.dst = d;
        for (int k = 0; k < kend; ++k) {
          const double val = ops.K[c][b * B + k];
          if (nzk(val)) u.t.push_back({k, (float)val});
        }
        outs.push_back(u);
      }
    if (v == 0)
      for (auto& u : outs) terms0 += u.t.size();
    tp.push_back(partition(outs, nparts));
    tv.push_back(outs);
  }
  // volume + face traces
  std::vector<Out> vo;
  size_t vterms = 0, gterms = 0;
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < B; ++b) {
      Out u;
      char d[64];
      std::snprintf(d, sizeof d, "y[%d * XP]", c * B + b);
      u.dst = d;
      for (int k = 0; k < B; ++k) {
        const double val = ops.K[c][k * B + b];
        if (nzk(val)) u.t.push_back({k, (float)val});
      }
      vterms += u.t.size();
      if (b == 0) {   // the constant mode has no derivative: Z_c[0] = 0, not read
        if (!u.t.empty()) throw std::runtime_error("K_c[k][0] must vanish");
        continue;
      }
      vo.push_back(u);
    }
  for (int i = 0; i < 4; ++i)
    for (int m = 0; m < F; ++m) {
      Out u;
      char d[64];
      std::snprintf(d, sizeof d, "g[%d * XP]", i * F + m);
      u.dst = d;
      for (int k = 0; k < B; ++k) {
        const double val = ops.Ft[i][k * F + m];
        if (nzf(val)) u.t.push_back({k, (float)val});
      }
      gterms += u.t.size();
      vo.push_back(u);
    }
  std::fprintf(f, "// time-kernel product: %zu multiply-adds per row (full variant); volume %zu, face traces %zu\n",
               terms0, vterms, gterms);
  std::fprintf(f, "constexpr int kSpTimeTerms_o%d = %zu, kSpVolTerms_o%d = %zu, kSpFaceTerms_o%d = %zu;\n", O,
               terms0, O, vterms, O, gterms);
  char nm[64];
  std::snprintf(nm, sizeof nm, "sp_time_o%d", O);
  emit_dispatch(f, nm, "const float* __restrict__ x, float* __restrict__ y", "x, y", tp, tv, true);
  std::vector<std::vector<std::vector<int>>> vp{partition(vo, nparts)};
  std::vector<std::vector<Out>> vv{vo};
  std::snprintf(nm, sizeof nm, "sp_vol_o%d", O);
  emit_dispatch(f, nm, "const float* __restrict__ x, float* __restrict__ y, float* __restrict__ g", "x, y, g", vp, vv,
                false);
}

}  // namespace

// gen_sparse --list O: one line per product term, "<kind> <part> <output> <k> <value>" with
// kind t (time kernel, output c*B + b, full variant), v (volume, output c*B + b) or g (face
// trace, output i*F + f), for checking the generated products against other operators.
int list_terms(int O, int nparts) {
  lts::RefOps ops;
  ops.build(O);
  const int B = ops.B, F = ops.F;
  double kmax = 0.0, fmax = 0.0;
  for (int c = 0; c < 3; ++c)
    for (double v : ops.K[c]) kmax = std::max(kmax, std::fabs(v));
  for (int i = 0; i < 4; ++i)
    for (double v : ops.Ft[i]) fmax = std::max(fmax, std::fabs(v));
  std::vector<Out> t, v;
  std::vector<int> tid, vid;
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < B; ++b) {
      Out u, w;
      for (int k = 0; k < B; ++k) {
        if (std::fabs(ops.K[c][b * B + k]) > 1e-7 * kmax) u.t.push_back({k, (float)ops.K[c][b * B + k]});
        if (std::fabs(ops.K[c][k * B + b]) > 1e-7 * kmax) w.t.push_back({k, (float)ops.K[c][k * B + b]});
      }
      if (b < (O - 1) * O * (O + 1) / 6) {   // outputs of the full time variant: deg b <= O-2
        t.push_back(u);
        tid.push_back(c * B + b);
      }
      if (b > 0) {
        v.push_back(w);
        vid.push_back(c * B + b);
      }
    }
  const size_t nv = v.size();
  for (int i = 0; i < 4; ++i)
    for (int m = 0; m < F; ++m) {
      Out u;
      for (int k = 0; k < B; ++k)
        if (std::fabs(ops.Ft[i][k * F + m]) > 1e-7 * fmax) u.t.push_back({k, (float)ops.Ft[i][k * F + m]});
      v.push_back(u);
      vid.push_back(i * F + m);
    }
  const auto tp = partition(t, nparts), vp = partition(v, nparts);
  for (int p = 0; p < nparts; ++p) {
    for (int o : tp[p])
      for (auto& x : t[o].t) std::printf("t %d %d %d %.9e\n", p, tid[o], x.first, (double)x.second);
    for (int o : vp[p])
      for (auto& x : v[o].t) std::printf("%c %d %d %d %.9e\n", (size_t)o < nv ? 'v' : 'g', p, vid[o], x.first, (double)x.second);
  }
  return 0;
}

int main(int argc, char** argv) {
  if (argc == 3 && std::strcmp(argv[1], "--list") == 0) {
    const int O = std::atoi(argv[2]);
    if (O < 3 || O > 5) return 2;
    return list_terms(O, O == 5 ? 4 : (O == 4 ? 2 : 1));
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
  emit_order(f, 3, 1);
  emit_order(f, 4, 2);
  emit_order(f, 5, 4);
  std::fprintf(f, "}  // namespace ltssp\n");
  return std::fclose(f) == 0 ? 0 : 1;
}
