// C ABI of the solver: set-up tables, device state and the clustered-LTS schedule.
#include <algorithm>
#include <array>
#include <thread>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ader_lts.h"
#include "host.h"
#include "host_flux.h"
#include "host_partition.h"
#include "launch.h"

using ltsdev::DevOps;
using ltsdev::DevState;
using ltsdev::Launchers;
using ltsdev::PhaseArgs;
using ltsdev::RecvItem;
using ltsdev::SrcItem;

namespace ltsdev {
bool get_launchers(int order, int m, bool fused, Launchers* out) {
  if (m != 0 && m != 3) return false;
  switch (order) {
    case 3: *out = launchers_o3(m, fused); return true;
    case 4: *out = launchers_o4(m, fused); return true;
    case 5: *out = launchers_o5(m, fused); return true;
    default: return false;
  }
}
}  // namespace ltsdev

namespace {

struct Source {
  int64_t elem;          // original index
  int sim;               // fused simulation it drives
  double xi[3];
  double m6[6];
  double f0, t0, m0;
  std::vector<double> phi;
};

struct Receiver {
  int64_t elem;
  double xi[3];
  double dt;
  std::vector<double> phi;
  std::vector<double> t;       // sample times
  std::vector<int64_t> slot;   // device output slot of each sample
};

struct Status {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg) { throw Status{code, msg}; }

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(LTS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct GraphKey {
  const void *seis, *ritems, *sitems, *block;
  int contraction, ctas_p, ctas_n, suppress, parts, tile;
  long long wait;
  size_t n_r, n_s;
};

struct MacroGraph {
  cudaGraphExec_t exec = nullptr;
  GraphKey key{};
  int launches = 0;
};

struct lts_solver {
  int order = 0, nmech = 0, device = 0;
  int nsim = 1;                             // fused simulations
  int contraction = LTS_CONTRACT_FP32;
  int ctas_predict = 0, ctas_neighbour = 0;  // resident CTAs per SM the grids are sized for (0: occupancy)
  int tile = 1;                              // tile variant of the sparse engine's neighbour kernel
  long long wait_cycles = ltsdev::TC_WAIT_CYCLES;   // bound of the tensor-core completion waits
  int suppress_commit = 0;                          // failure-path test: waits run out
  // emulated partitioned run (Sec. V-C): cut faces receive face-local messages
  int n_parts = 1;
  std::vector<int32_t> part;
  std::vector<int64_t> cut_beg;             // cut faces by receiver cluster (device order), nc+1
  int64_t n_cut = 0;
  int* d_cut = nullptr;                     // [3][n_cut]: sender element, code, receiver cluster
  float* d_msg = nullptr;                   // [n_cut][nsim][9][F]
  int64_t msg_bytes = 0;                    // face-local message bytes produced so far
  // macro steps replayed from CUDA graphs (one per parity of the macro-step index)
  bool use_graphs = true;
  MacroGraph graphs[2];
  cudaStream_t capture_stream = nullptr;
  std::string err;
  Launchers L{};
  lts::RefOps ops;
  lts::Mesh mesh;
  lts::Material mat;
  bool has_mesh = false, has_mat = false, ready = false;
  std::vector<double> lam, mu, omega;       // per element / per mechanism
  std::vector<double> ylam, ymu;            // [K][m]
  std::vector<Source> sources;
  std::vector<Receiver> receivers;
  // clusters
  int nc = 1;
  double lambda = 1.0, dt_min = 0.0, delta = 0.0, speedup = 1.0;
  std::vector<int32_t> cluster;             // original order
  std::vector<int64_t> perm, iperm;         // perm[new] = old, iperm[old] = new
  std::vector<int64_t> cbeg;                // cluster ranges (internal order), nc+1
  int64_t s_now = 0;
  int64_t launches = 0;
  int64_t h2d_bytes = 0, d2h_bytes = 0;      // copies issued by advance / read calls
  // device
  void* block = nullptr;
  bool own_block = false;
  size_t block_bytes = 0;
  void* bound = nullptr;
  size_t bound_bytes = 0;
  DevOps dops{};
  DevState dst{};
  double* d_emat = nullptr;
  double* d_partial = nullptr;
  int* d_err = nullptr;                     // set by a kernel whose bounded wait gave up
  float* d_recv_phi = nullptr;
  float* d_src_phi = nullptr;
  int n_partial = 1024;
  // growable library-owned scratch
  float* d_seis = nullptr;
  size_t seis_cap = 0, seis_used = 0;
  RecvItem* d_ritems = nullptr;
  size_t ritems_cap = 0;
  SrcItem* d_sitems = nullptr;
  size_t sitems_cap = 0;
  int num_sms = 0;
  uint64_t adj_budget = 0;   // bytes for the LTS adjoint's phase inputs (0: half the free memory)
  std::vector<double> adj_src_grad;   // dJ/dm6 per source from the last adjoint sweep
  // profiling: event pairs around each predict / neighbour launch, read lazily
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<int> ev_kind;
  std::vector<int64_t> ev_elems;
};

namespace {

int run(lts_t* h, const std::function<void()>& fn) {
  if (!h) return LTS_ERR_ARG;
  try {
    h->err.clear();
    fn();
    return LTS_OK;
  } catch (const Status& s) {
    h->err = s.msg;
    return s.code;
  } catch (const std::bad_alloc&) {
    h->err = "host allocation failed";
    return LTS_ERR_OOM;
  } catch (const std::exception& e) {
    h->err = e.what();
    return LTS_ERR_ARG;
  }
}

// Face-basis maps of the three orientations h: the neighbour matrices factor as F-_{j,h} =
// F~_j R_h, R_h[f'][f] = int psi_f(chi) psi_f'(chi'(chi, h)) (the trace on the neighbour's face
// j, re-expanded in the local face parametrisation; an affine map of the triangle keeps
// polynomial degree, so R_h is block diagonal by degree and orthogonal). Solved here from the
// normal equations of F~_0 R_h = F-_{0,h} in FP64 and checked on every face j.
void face_orientation_maps(const lts::RefOps& ops, std::vector<float>& out) {
  const int B = ops.B, F = ops.F;
  std::vector<double> A(F * F), rhs(F * F);
  for (int h = 0; h < 3; ++h) {
    for (int p = 0; p < F; ++p)
      for (int q = 0; q < F; ++q) {
        double a = 0.0, r = 0.0;
        for (int k = 0; k < B; ++k) {
          a += ops.Ft[0][k * F + p] * ops.Ft[0][k * F + q];
          r += ops.Ft[0][k * F + p] * ops.Fb[h][k * F + q];
        }
        A[p * F + q] = a;
        rhs[p * F + q] = r;
      }
    // Gauss-Jordan with partial pivoting on [A | rhs] (A is symmetric positive definite)
    std::vector<double> M = A, R = rhs;
    for (int c = 0; c < F; ++c) {
      int piv = c;
      for (int r = c + 1; r < F; ++r)
        if (std::fabs(M[r * F + c]) > std::fabs(M[piv * F + c])) piv = r;
      for (int q = 0; q < F; ++q) {
        std::swap(M[c * F + q], M[piv * F + q]);
        std::swap(R[c * F + q], R[piv * F + q]);
      }
      const double d = M[c * F + c];
      if (std::fabs(d) < 1e-300) fail(LTS_ERR_ARG, "singular face trace matrix");
      for (int q = 0; q < F; ++q) {
        M[c * F + q] /= d;
        R[c * F + q] /= d;
      }
      for (int r = 0; r < F; ++r) {
        if (r == c) continue;
        const double f = M[r * F + c];
        if (f == 0.0) continue;
        for (int q = 0; q < F; ++q) {
          M[r * F + q] -= f * M[c * F + q];
          R[r * F + q] -= f * R[c * F + q];
        }
      }
    }
    double scale = 0.0, err = 0.0;
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < B; ++k)
        for (int q = 0; q < F; ++q) {
          double v = 0.0;
          for (int p = 0; p < F; ++p) v += ops.Ft[j][k * F + p] * R[p * F + q];
          scale = std::max(scale, std::fabs(ops.Fb[j * 3 + h][k * F + q]));
          err = std::max(err, std::fabs(v - ops.Fb[j * 3 + h][k * F + q]));
        }
    if (err > 1e-8 * scale) fail(LTS_ERR_ARG, "neighbour matrices do not factor through the face traces");
    for (int i = 0; i < F * F; ++i) out[h * F * F + i] = (float)R[i];
  }
}

struct Layout {
  size_t Q, B1, B2, B3, edata, ndata, nbr, ncode, meta, emat, partial, err, K, Ft, Fh, Fb, Rh, rphi, sphi, cut, msg,
      total;
};

// Element strides (floats) of Q and of the LTS buffers: [group][q][b][G] per element with
// the simulations of a group innermost; one simulation keeps the rows padded to 16 bytes.
int64_t q_stride(const lts_solver* h) {
  return h->nsim == 1 ? h->L.QS : (int64_t)h->L.NQ * h->L.B * h->nsim;
}
int64_t buf_stride(const lts_solver* h) { return h->nsim == 1 ? h->L.BUFS : (int64_t)9 * h->L.B * h->nsim; }

Layout layout_of(const lts_solver* h, int64_t K) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const Launchers& X = h->L;
  const size_t qs = (size_t)q_stride(h), bs = (size_t)buf_stride(h);
  L.Q = take(sizeof(float) * K * qs);
  L.B1 = take(sizeof(float) * K * bs);
  L.B2 = take(sizeof(float) * K * bs);
  L.B3 = take(sizeof(float) * K * bs);
  L.edata = take(sizeof(float) * K * ltsdev::ED);
  L.ndata = take(sizeof(float) * K * ltsdev::ND);
  L.nbr = take(sizeof(int) * K * 4);
  L.ncode = take(sizeof(int) * K * 4);
  L.meta = take(sizeof(int) * K);
  L.emat = take(sizeof(double) * K * 4);
  L.partial = take(sizeof(double) * h->n_partial);
  L.err = take(sizeof(int));
  L.K = take(sizeof(float) * 3 * X.B * X.B);
  L.Ft = take(sizeof(float) * 4 * X.B * X.F);
  L.Fh = take(sizeof(float) * 4 * X.F * X.B);
  L.Fb = take(sizeof(float) * 12 * X.B * X.F);
  L.Rh = take(sizeof(float) * 3 * X.F * X.F);
  L.rphi = take(sizeof(float) * std::max<size_t>(1, h->receivers.size()) * X.B);
  L.sphi = take(sizeof(float) * std::max<size_t>(1, h->sources.size()) * X.B);
  // cut faces of a partitioned run
  int64_t ncut = 0;
  if (h->n_parts > 1)
    for (int64_t k = 0; k < K; ++k)
      for (int f = 0; f < 4; ++f) {
        const int64_t nb = h->mesh.nbr[4 * k + f];
        if (nb >= 0 && h->part[nb] != h->part[k]) ++ncut;
      }
  L.cut = take(sizeof(int) * 3 * std::max<int64_t>(1, ncut));
  L.msg = take(sizeof(float) * 9 * X.F * h->nsim * std::max<int64_t>(1, ncut));
  L.total = off;
  return L;
}

void release_events(lts_solver* h) {
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  h->ev_pool.clear();
  h->ev_used = 0;
  h->ev_kind.clear();
  h->ev_elems.clear();
}

cudaEvent_t next_event(lts_solver* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    ck(cudaEventCreate(&e), "cudaEventCreate");
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

void release_graphs(lts_solver* h) {
  for (MacroGraph& g : h->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.launches = 0;
  }
}

void free_device(lts_solver* h) {
  release_graphs(h);
  if (h->own_block && h->block) cudaFree(h->block);
  h->block = nullptr;
  h->own_block = false;
  if (h->d_seis) cudaFree(h->d_seis);
  if (h->d_ritems) cudaFree(h->d_ritems);
  if (h->d_sitems) cudaFree(h->d_sitems);
  h->d_seis = nullptr;
  h->d_ritems = nullptr;
  h->d_sitems = nullptr;
  h->seis_cap = h->seis_used = h->ritems_cap = h->sitems_cap = 0;
  h->ready = false;
}

void setup_device(lts_solver* h) {
  const int64_t K = h->mesh.K;
  const Launchers& X = h->L;
  const int m = h->nmech;
  // ---- permutation: stable sort by cluster
  h->perm.resize(K);
  std::iota(h->perm.begin(), h->perm.end(), 0);
  std::stable_sort(h->perm.begin(), h->perm.end(),
                   [&](int64_t a, int64_t b) { return h->cluster[a] < h->cluster[b]; });
  h->iperm.resize(K);
  for (int64_t i = 0; i < K; ++i) h->iperm[h->perm[i]] = i;
  h->cbeg.assign(h->nc + 1, 0);
  for (int64_t i = 0; i < K; ++i) h->cbeg[h->cluster[i] + 1]++;
  for (int l = 0; l < h->nc; ++l) h->cbeg[l + 1] += h->cbeg[l];
  // ---- host tables in internal order
  std::vector<float> edata(K * ltsdev::ED, 0.f), ndata(K * ltsdev::ND, 0.f);
  std::vector<int> nbr(4 * K, -1), ncode(4 * K, 0), meta(K, 0);
  std::vector<double> emat(4 * K);
  const lts::Mesh& M = h->mesh;
  for (int64_t nk = 0; nk < K; ++nk) {
    const int64_t k = h->perm[nk];
    float* ed = &edata[nk * ltsdev::ED];
    float* nd = &ndata[nk * ltsdev::ND];
    for (int i = 0; i < 9; ++i) ed[i] = (float)M.Jinv[9 * k + i];
    const double rho = h->mat.rho[k];
    ed[9] = (float)h->lam[k];
    ed[10] = (float)h->mu[k];
    ed[11] = (float)(1.0 / rho);
    for (int l = 0; l < m; ++l) {
      ed[12 + 2 * l] = (float)(h->lam[k] * h->ylam[k * m + l]);
      ed[13 + 2 * l] = (float)(2.0 * h->mu[k] * h->ymu[k * m + l]);
    }
    nd[0] = ed[9];
    nd[1] = ed[10];
    nd[2] = ed[11];
    emat[4 * nk + 0] = h->lam[k];
    emat[4 * nk + 1] = h->mu[k];
    emat[4 * nk + 2] = rho;
    emat[4 * nk + 3] = M.detJ[k];
    const double zp = std::sqrt((h->lam[k] + 2.0 * h->mu[k]) * rho), zs = std::sqrt(h->mu[k] * rho);
    int flags = h->cluster[k];
    for (int f = 0; f < 4; ++f) {
      const int bc = M.bc[4 * k + f];
      const int64_t nb = M.nbr[4 * k + f];
      double zpo = zp, zso = zs;
      if (nb >= 0) {
        const double rn = h->mat.rho[nb];
        zpo = std::sqrt((h->lam[nb] + 2.0 * h->mu[nb]) * rn);
        zso = std::sqrt(h->mu[nb] * rn);
      }
      const double scale = -2.0 * M.area[4 * k + f] / M.detJ[k];
      float* lf = ed + 20 + 11 * f;
      float* nf = nd + 4 + 11 * f;
      for (int d = 0; d < 3; ++d) lf[d] = nf[d] = (float)M.normal[12 * k + 3 * f + d];
      double cl[8], cn[8];
      lts::face_coefficients_t<double>(bc, zp, zs, zpo, zso, scale, cl, cn);
      for (int q = 0; q < 8; ++q) {
        lf[3 + q] = (float)cl[q];
        nf[3 + q] = (float)cn[q];
      }
      if (nb >= 0) {
        nbr[4 * nk + f] = (int)h->iperm[nb];
        const int dc = h->cluster[nb] - h->cluster[k];
        const int rel = dc == 0 ? 0 : (dc < 0 ? 1 : 2);
        ncode[4 * nk + f] = (M.nbr_face[4 * k + f] * 3 + M.nbr_orient[4 * k + f]) | (rel << 8);
        if (dc < 0) flags |= ltsdev::FLAG_FINER;
        if (dc > 0) flags |= ltsdev::FLAG_COARSER;
      }
    }
    meta[nk] = flags;
  }
  // ---- operators (float)
  const int B = X.B, F = X.F;
  std::vector<float> hK(3 * B * B), hFt(4 * B * F), hFh(4 * F * B), hFb(12 * B * F);
  for (int c = 0; c < 3; ++c)
    for (int i = 0; i < B * B; ++i) hK[c * B * B + i] = (float)h->ops.K[c][i];
  for (int f = 0; f < 4; ++f)
    for (int k = 0; k < B; ++k)
      for (int q = 0; q < F; ++q) {
        hFt[(f * B + k) * F + q] = (float)h->ops.Ft[f][k * F + q];
        hFh[(f * F + q) * B + k] = (float)h->ops.Ft[f][k * F + q];
      }
  for (int jh = 0; jh < 12; ++jh)
    for (int i = 0; i < B * F; ++i) hFb[jh * B * F + i] = (float)h->ops.Fb[jh][i];
  std::vector<float> hRh(3 * F * F);
  face_orientation_maps(h->ops, hRh);
  std::vector<float> rphi(std::max<size_t>(1, h->receivers.size()) * B, 0.f);
  for (size_t r = 0; r < h->receivers.size(); ++r)
    for (int b = 0; b < B; ++b) rphi[r * B + b] = (float)h->receivers[r].phi[b];
  std::vector<float> sphi(std::max<size_t>(1, h->sources.size()) * B, 0.f);
  for (size_t s = 0; s < h->sources.size(); ++s)
    for (int b = 0; b < B; ++b) sphi[s * B + b] = (float)h->sources[s].phi[b];
  // ---- partitioned run: cut faces in device order (receiver cluster, then message order)
  std::vector<int> cut_host;
  h->n_cut = 0;
  h->cut_beg.assign(h->nc + 1, 0);
  if (h->n_parts > 1) {
    std::vector<lts::CutFace> cf;
    lts::cut_faces(M, h->part, h->cluster, cf);
    std::stable_sort(cf.begin(), cf.end(),
                     [](const lts::CutFace& a, const lts::CutFace& b) { return a.recv_cluster < b.recv_cluster; });
    h->n_cut = (int64_t)cf.size();
    cut_host.resize(3 * cf.size());
    for (size_t c = 0; c < cf.size(); ++c) {
      const lts::CutFace& x = cf[c];
      const int64_t nk = h->iperm[x.recv_elem];
      const int dc = h->cluster[x.send_elem] - h->cluster[x.recv_elem];
      const int rel = dc == 0 ? 0 : (dc < 0 ? 1 : 2);
      cut_host[c] = (int)h->iperm[x.send_elem];
      cut_host[cf.size() + c] = (x.send_face * 3 + x.orient) | (rel << 8);
      cut_host[2 * cf.size() + c] = x.recv_cluster;
      nbr[4 * nk + x.recv_face] = (int)c;
      ncode[4 * nk + x.recv_face] |= ltsdev::FACE_REMOTE;
      h->cut_beg[x.recv_cluster + 1]++;
    }
    for (int l = 0; l < h->nc; ++l) h->cut_beg[l + 1] += h->cut_beg[l];
  }
  // ---- device block
  free_device(h);
  Layout Lo = layout_of(h, K);
  if (h->bound) {
    if (h->bound_bytes < Lo.total) fail(LTS_ERR_OOM, "bound device block too small");
    h->block = h->bound;
    h->own_block = false;
  } else {
    cudaError_t e = cudaMalloc(&h->block, Lo.total);
    if (e != cudaSuccess) {
      h->block = nullptr;
      fail(LTS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->own_block = true;
  }
  h->block_bytes = Lo.total;
  char* base = static_cast<char*>(h->block);
  h->dst.Q = reinterpret_cast<float*>(base + Lo.Q);
  h->dst.B1 = reinterpret_cast<float*>(base + Lo.B1);
  h->dst.B2 = reinterpret_cast<float*>(base + Lo.B2);
  h->dst.B3 = reinterpret_cast<float*>(base + Lo.B3);
  h->dst.edata = reinterpret_cast<float*>(base + Lo.edata);
  h->dst.ndata = reinterpret_cast<float*>(base + Lo.ndata);
  h->dst.nbr = reinterpret_cast<int*>(base + Lo.nbr);
  h->dst.ncode = reinterpret_cast<int*>(base + Lo.ncode);
  h->dst.meta = reinterpret_cast<int*>(base + Lo.meta);
  h->d_emat = reinterpret_cast<double*>(base + Lo.emat);
  h->d_partial = reinterpret_cast<double*>(base + Lo.partial);
  h->d_err = reinterpret_cast<int*>(base + Lo.err);
  h->dops.K = reinterpret_cast<float*>(base + Lo.K);
  h->dops.Ft = reinterpret_cast<float*>(base + Lo.Ft);
  h->dops.Fh = reinterpret_cast<float*>(base + Lo.Fh);
  h->dops.Fb = reinterpret_cast<float*>(base + Lo.Fb);
  h->dops.Rh = reinterpret_cast<float*>(base + Lo.Rh);
  h->d_recv_phi = reinterpret_cast<float*>(base + Lo.rphi);
  h->d_src_phi = reinterpret_cast<float*>(base + Lo.sphi);
  h->d_cut = reinterpret_cast<int*>(base + Lo.cut);
  h->d_msg = reinterpret_cast<float*>(base + Lo.msg);
  h->dst.msg = h->d_msg;
  auto up = [&](const void* dst, const void* src, size_t bytes) {
    ck(cudaMemcpy(const_cast<void*>(dst), src, bytes, cudaMemcpyHostToDevice), "upload");
  };
  h->dst.qs = q_stride(h);
  h->dst.bs = buf_stride(h);
  h->dst.nsim = h->nsim;
  ck(cudaMemset(h->dst.Q, 0, sizeof(float) * K * h->dst.qs), "memset Q");
  ck(cudaMemset(h->dst.B1, 0, sizeof(float) * K * h->dst.bs), "memset B1");
  ck(cudaMemset(h->dst.B2, 0, sizeof(float) * K * h->dst.bs), "memset B2");
  ck(cudaMemset(h->dst.B3, 0, sizeof(float) * K * h->dst.bs), "memset B3");
  ck(cudaMemset(h->d_err, 0, sizeof(int)), "memset error word");
  up(h->dst.edata, edata.data(), sizeof(float) * edata.size());
  up(h->dst.ndata, ndata.data(), sizeof(float) * ndata.size());
  up(h->dst.nbr, nbr.data(), sizeof(int) * nbr.size());
  up(h->dst.ncode, ncode.data(), sizeof(int) * ncode.size());
  up(h->dst.meta, meta.data(), sizeof(int) * meta.size());
  up(h->d_emat, emat.data(), sizeof(double) * emat.size());
  up(h->dops.K, hK.data(), sizeof(float) * hK.size());
  up(h->dops.Ft, hFt.data(), sizeof(float) * hFt.size());
  up(h->dops.Fh, hFh.data(), sizeof(float) * hFh.size());
  up(h->dops.Fb, hFb.data(), sizeof(float) * hFb.size());
  up(h->dops.Rh, hRh.data(), sizeof(float) * hRh.size());
  up(h->d_recv_phi, rphi.data(), sizeof(float) * rphi.size());
  up(h->d_src_phi, sphi.data(), sizeof(float) * sphi.size());
  if (!cut_host.empty()) up(h->d_cut, cut_host.data(), sizeof(int) * cut_host.size());
  for (auto& r : h->receivers) {
    r.t.clear();
    r.slot.clear();
  }
  h->s_now = 0;
  h->ready = true;
}

void finish_clusters(lts_solver* h, double* lambda_out, double* speedup_out, int32_t* cluster_out) {
  const int64_t K = h->mesh.K;
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      int64_t nb = h->mesh.nbr[4 * k + f];
      if (nb >= 0 && std::abs(h->cluster[nb] - h->cluster[k]) > 1)
        fail(LTS_ERR_ARG, "face neighbours differ by more than one cluster");
    }
  h->speedup = lts::theoretical_speedup(h->cluster, h->lambda);
  h->delta = h->lambda * h->dt_min;
  if (h->device >= 0) setup_device(h);
  if (lambda_out) *lambda_out = h->lambda;
  if (speedup_out) *speedup_out = h->speedup;
  if (cluster_out) std::copy(h->cluster.begin(), h->cluster.end(), cluster_out);
}

void require_material(lts_solver* h) {
  if (!h->has_mesh) fail(LTS_ERR_STATE, "no mesh");
  if (!h->has_mat) fail(LTS_ERR_STATE, "no material");
}

void ensure_capacity(void** ptr, size_t* cap, size_t need, size_t elem) {
  if (need <= *cap) return;
  size_t nc = std::max(need, *cap * 2 + 16);
  void* p = nullptr;
  ck(cudaMalloc(&p, nc * elem), "cudaMalloc scratch");
  if (*ptr) {
    ck(cudaMemcpy(p, *ptr, *cap * elem, cudaMemcpyDeviceToDevice), "grow copy");
    cudaFree(*ptr);
  }
  *ptr = p;
  *cap = nc;
}

// Raises LTS_ERR_TIMEOUT if a kernel reported a bounded wait that gave up (the device
// must be synchronised); the report clears the word.
void check_device_error(lts_solver* h) {
  if (!h->d_err) return;
  int v = 0;
  ck(cudaMemcpy(&v, h->d_err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
  if (v != 0) {
    ck(cudaMemset(h->d_err, 0, sizeof(int)), "clear error word");
    fail(LTS_ERR_TIMEOUT, "a tensor-core completion wait gave up");
  }
}

double ricker(double t, double f0, double t0) {
  const double pi = 3.14159265358979323846;
  double a = pi * f0 * (t - t0);
  a *= a;
  return (1.0 - 2.0 * a) * std::exp(-a);
}

// One macro step (2^(N_c-1) finest steps from time level s_begin) as a fixed sequence of
// phases: per finest level, the neighbour passes of the clusters ending there, then the
// receivers and predict passes of the clusters starting there (Sec. V-B). The sequence, the
// grids and the work-item counts are the same for every macro step; only the parity of the
// coarsest cluster's step alternates (parity of the macro step) and the work-item values
// (source amplitudes, receiver sample times) change.
struct Phase {
  int kind;          // 0 neighbour, 1 predict
  int top;           // clusters 0..top
  int64_t s;
  int item_beg, item_end;
};

struct MacroPlan {
  std::vector<Phase> phases;
  std::vector<SrcItem> sitems;
  std::vector<double> sscale;   // per source item: -m0 (int s dt) / |det J| (amp = sscale m6)
  std::vector<RecvItem> ritems;
};

void plan_macro(lts_solver* h, int64_t s_begin, size_t& seis_need, MacroPlan& mp) {
  const int nc = h->nc;
  const int B = h->L.B;
  const int64_t s_end = s_begin + (int64_t(1) << (nc - 1));
  mp.phases.clear();
  mp.sitems.clear();
  mp.sscale.clear();
  mp.ritems.clear();
  std::vector<double> gx, gw;
  lts::gauss_jacobi(h->order, 0.0, gx, gw);
  auto top_cluster = [&](int64_t s) {
    int l = 0;
    while (l + 1 < nc && s % (int64_t(1) << (l + 1)) == 0) ++l;
    return l;
  };
  for (int64_t s = s_begin; s <= s_end; ++s) {
    if (s > s_begin) {
      Phase ph{0, top_cluster(s), s, (int)mp.sitems.size(), 0};
      for (size_t si = 0; si < h->sources.size(); ++si) {
        const Source& src = h->sources[si];
        const int l = h->cluster[src.elem];
        if (l > ph.top) continue;
        const double ta = (s - (int64_t(1) << l)) * h->delta, tb = s * h->delta;
        double integ = 0.0;
        for (int q = 0; q < h->order; ++q)
          integ += gw[q] * ricker(0.5 * (ta + tb) + 0.5 * (tb - ta) * gx[q], src.f0, src.t0);
        integ *= 0.5 * (tb - ta);
        SrcItem it{};
        it.elem = (int)h->iperm[src.elem];
        it.sim = src.sim;
        it.phi_off = (int)(si * B);
        for (int r = 0; r < 6; ++r) it.amp[r] = (float)(-src.m0 * src.m6[r] * integ / h->mesh.detJ[src.elem]);
        mp.sitems.push_back(it);
        mp.sscale.push_back(-src.m0 * integ / h->mesh.detJ[src.elem]);
      }
      ph.item_end = (int)mp.sitems.size();
      mp.phases.push_back(ph);
    }
    if (s < s_end) {
      Phase ph{1, top_cluster(s), s, (int)mp.ritems.size(), 0};
      for (size_t ri = 0; ri < h->receivers.size(); ++ri) {
        Receiver& rc = h->receivers[ri];
        const int l = h->cluster[rc.elem];
        if (l > ph.top) continue;
        const double ta = s * h->delta, tb = (s + (int64_t(1) << l)) * h->delta;
        RecvItem it{};
        it.elem = (int)h->iperm[rc.elem];
        it.sim = 0;
        it.phi_off = (int)(ri * B);
        it.n = 0;
        it.out_off = 0;
        int64_t j = std::max<int64_t>((int64_t)std::floor(ta / rc.dt) - 1, 0);
        for (; j * rc.dt < tb; ++j) {
          const double tj = j * rc.dt;
          if (tj < ta) continue;
          if (it.n == 8) fail(LTS_ERR_ARG, "more than 8 receiver samples in one element step");
          it.tau[it.n] = (float)(tj - ta);
          rc.t.push_back(tj);
          rc.slot.push_back((int64_t)seis_need);
          if (it.n == 0) it.out_off = (int)seis_need;
          ++seis_need;
          ++it.n;
        }
        // one item per simulation (also without samples: the item count of a phase is
        // fixed); sample slot j holds nsim x 9 values
        for (int f = 0; f < h->nsim; ++f) {
          it.sim = f;
          mp.ritems.push_back(it);
        }
      }
      ph.item_end = (int)mp.ritems.size();
      mp.phases.push_back(ph);
    }
  }
}

// Kernel arguments of one phase (Taylor coefficients per cluster, element range, step parities).
PhaseArgs phase_args(const lts_solver* h, const Phase& ph) {
  PhaseArgs pa{};
  for (int l = 0; l < h->nc; ++l) {
    const double dl = h->delta * std::ldexp(1.0, l);
    double fac = 1.0;
    for (int d = 0; d < h->order; ++d) {
      fac *= (d + 1);
      pa.coef[l][d] = (float)(std::pow(dl, d + 1) / fac);
      pa.hcoef[l][d] = (float)(std::pow(0.5 * dl, d + 1) / fac);
    }
  }
  for (int l = 0; l < 3; ++l) pa.omega[l] = l < (int)h->omega.size() ? (float)h->omega[l] : 0.f;
  pa.err = h->d_err;
  pa.wait = h->wait_cycles;
  pa.suppress = h->suppress_commit;
  pa.begin = 0;
  pa.end = (int)h->cbeg[ph.top + 1];
  for (int l = 0; l <= ph.top; ++l) {
    const int64_t n = ph.kind == 0 ? (ph.s >> l) - 1 : (ph.s >> l);
    pa.parity[l] = (int)(n & 1);
  }
  return pa;
}

// Enqueues the launches of one phase on `stream` (work items at the start of the item
// buffers); returns the number of kernels launched. Receivers are skipped when
// with_receivers is false (state-only replays).
int enqueue_phase(lts_solver* h, const Phase& ph, cudaStream_t stream, bool with_receivers = true) {
  const Launchers& X = h->L;
  const bool use_sp = h->contraction == LTS_CONTRACT_SPARSE;
  const bool use_tc = h->contraction == LTS_CONTRACT_TF32X3 || h->contraction == LTS_CONTRACT_TF32;
  const int passes = h->contraction == LTS_CONTRACT_TF32X3 ? 3 : 1;
  const int maxp = std::max(1, use_tc ? X.blocks_predict_tc : (use_sp ? X.blocks_predict_sp : X.blocks_predict));
  // the sparse engine's neighbour kernel reads every neighbour from local buffers: partitioned
  // runs (face-local messages) keep the gather-and-product neighbour kernel
  const bool use_nsp = use_sp && X.neighbour_sp[0] && h->n_parts <= 1;
  const int tv = h->tile & 1;
  const int maxn = std::max(1, use_nsp ? X.blocks_neighbour_sp[tv] : X.blocks_neighbour);
  const int grid_cap_p = h->num_sms * (h->ctas_predict > 0 ? std::min(h->ctas_predict, maxp) : maxp);
  const int grid_cap_n = h->num_sms * (h->ctas_neighbour > 0 ? std::min(h->ctas_neighbour, maxn) : maxn);
  const PhaseArgs pa = phase_args(h, ph);
  const int nelem = pa.end - pa.begin;
  if (nelem <= 0) return 0;
  int launches = 0;
  // NVTX range per phase while profiling (kind, finest level, clusters 0..top)
  struct Range {
    bool on;
    ~Range() {
      if (on) nvtxRangePop();
    }
  } range{h->profiling};
  if (range.on) {
    char name[64];
    std::snprintf(name, sizeof(name), "%s s=%lld clusters<=%d", ph.kind == 0 ? "neighbour" : "predict",
                  (long long)ph.s, ph.top);
    nvtxRangePushA(name);
  }
  // CTA batches: NE elements (one simulation) or one element and FG of its simulations
  const int ne_batch = ph.kind == 0 ? (use_nsp ? X.NEN_SP[tv] : X.NEN) : (use_sp ? X.NE_SP : X.NE);
  // sparse engine: batches of ne_batch slots (elements, or (element, simulation) pairs)
  const bool slots = ph.kind == 0 ? use_nsp : use_sp;
  const int nb = slots ? (int)(((int64_t)nelem * h->nsim + ne_batch - 1) / ne_batch)
                       : (X.FG > 1 ? nelem * (h->nsim / X.FG) : (nelem + ne_batch - 1) / ne_batch);
  if (with_receivers && ph.kind == 1 && ph.item_end > ph.item_beg) {
    X.receivers(h->dops, h->dst.Q, h->dst.qs, h->nsim, X.FG, h->dst.edata, h->d_recv_phi, h->d_ritems + ph.item_beg,
                h->d_seis, pa.omega, ph.item_end - ph.item_beg, stream);
    ++launches;
  }
  if (ph.kind == 0 && h->n_parts > 1 && h->cut_beg[ph.top + 1] > 0) {
    // the neighbours' partitions compute the face-local messages of the active cut faces
    const int nact = (int)h->cut_beg[ph.top + 1];
    X.pack(h->dops, h->dst, pa, h->d_cut, h->d_cut + h->n_cut, h->d_cut + 2 * h->n_cut, nact, h->d_msg, stream);
    ++launches;
  }
  if (h->profiling) ck(cudaEventRecord(next_event(h), stream), "event record");
  if (ph.kind == 0 && use_nsp)
    X.neighbour_sp[tv](h->dops, h->dst, pa, std::min(nb, grid_cap_n), stream);
  else if (ph.kind == 0)
    X.neighbour(h->dops, h->dst, pa, std::min(nb, grid_cap_n), stream);
  else if (use_tc)
    X.predict_tc(h->dops, h->dst, pa, std::min(nb, grid_cap_p), passes, h->d_err, h->wait_cycles, h->suppress_commit,
                 stream);
  else if (use_sp)
    X.predict_sp(h->dops, h->dst, pa, std::min(nb, grid_cap_p), stream);
  else
    X.predict(h->dops, h->dst, pa, std::min(nb, grid_cap_p), stream);
  ++launches;
  if (h->profiling) {
    ck(cudaEventRecord(next_event(h), stream), "event record");
    h->ev_kind.push_back(ph.kind == 1 ? 0 : 1);
    h->ev_elems.push_back(nelem);
  }
  if (ph.kind == 0 && ph.item_end > ph.item_beg) {
    X.sources(h->dst.Q, h->dst.qs, X.FG, h->d_src_phi, h->d_sitems + ph.item_beg, ph.item_end - ph.item_beg, stream);
    ++launches;
  }
  return launches;
}

// Enqueues the launches of one macro step on `stream`; returns the number of kernels.
int enqueue_macro(lts_solver* h, const MacroPlan& mp, cudaStream_t stream) {
  int launches = 0;
  for (const Phase& ph : mp.phases) launches += enqueue_phase(h, ph, stream);
  ck(cudaGetLastError(), "kernel launch");
  return launches;
}

// Face-local message bytes of one macro step of a partitioned run.
int64_t macro_msg_bytes(const lts_solver* h, const MacroPlan& mp) {
  int64_t b = 0;
  if (h->n_parts <= 1) return 0;
  for (const Phase& ph : mp.phases)
    if (ph.kind == 0 && h->cbeg[ph.top + 1] > 0)
      b += h->cut_beg[ph.top + 1] * h->nsim * 9 * (int64_t)h->L.F * (int64_t)sizeof(float);
  return b;
}

void advance_steps(lts_solver* h, int64_t n_finest, cudaStream_t stream) {
  if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
  struct Range {
    Range() { nvtxRangePushA("lts_advance"); }
    ~Range() { nvtxRangePop(); }
  } range;
  const int nc = h->nc;
  const int64_t period = int64_t(1) << (nc - 1);
  if (n_finest < 0 || n_finest % period != 0) fail(LTS_ERR_ARG, "n_finest must be a multiple of 2^(N_c-1)");
  if (n_finest == 0) return;
  const int64_t s0 = h->s_now, nmac = n_finest / period;
  // host plans of every macro step (receiver sample slots are assigned here)
  std::vector<MacroPlan> plans(nmac);
  size_t seis_need = h->seis_used;
  for (int64_t m = 0; m < nmac; ++m) plan_macro(h, s0 + m * period, seis_need, plans[m]);
  ensure_capacity(reinterpret_cast<void**>(&h->d_seis), &h->seis_cap, seis_need * 9 * h->nsim, sizeof(float));
  ensure_capacity(reinterpret_cast<void**>(&h->d_ritems), &h->ritems_cap, plans[0].ritems.size(), sizeof(RecvItem));
  ensure_capacity(reinterpret_cast<void**>(&h->d_sitems), &h->sitems_cap, plans[0].sitems.size(), sizeof(SrcItem));
  h->seis_used = seis_need;
  for (int64_t m = 0; m < nmac; ++m) {
    const MacroPlan& mp = plans[m];
    // this macro step's work items; stream-ordered after the previous macro step
    if (!mp.ritems.empty())
      ck(cudaMemcpyAsync(h->d_ritems, mp.ritems.data(), mp.ritems.size() * sizeof(RecvItem), cudaMemcpyHostToDevice,
                         stream),
         "upload receiver items");
    if (!mp.sitems.empty())
      ck(cudaMemcpyAsync(h->d_sitems, mp.sitems.data(), mp.sitems.size() * sizeof(SrcItem), cudaMemcpyHostToDevice,
                         stream),
         "upload source items");
    h->h2d_bytes += (int64_t)(mp.ritems.size() * sizeof(RecvItem) + mp.sitems.size() * sizeof(SrcItem));
    h->msg_bytes += macro_msg_bytes(h, mp);
    if (!h->use_graphs || h->profiling) {
      h->launches += enqueue_macro(h, mp, stream);
      continue;
    }
    // CUDA graph of the macro step, one per parity of the macro-step index, rebuilt when
    // anything its launches capture has changed
    const int par = (int)(((s0 / period) + m) & 1);
    GraphKey key{};
    key.seis = h->d_seis;
    key.ritems = h->d_ritems;
    key.sitems = h->d_sitems;
    key.block = h->block;
    key.contraction = h->contraction;
    key.ctas_p = h->ctas_predict;
    key.ctas_n = h->ctas_neighbour;
    key.tile = h->tile;
    key.wait = h->wait_cycles;
    key.suppress = h->suppress_commit;
    key.parts = h->n_parts;
    key.n_r = mp.ritems.size();
    key.n_s = mp.sitems.size();
    MacroGraph& g = h->graphs[par];
    if (!g.exec || std::memcmp(&g.key, &key, sizeof(GraphKey)) != 0) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
      if (!h->capture_stream) ck(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking), "capture stream");
      ck(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      int nl = 0;
      try {
        nl = enqueue_macro(h, mp, h->capture_stream);
      } catch (...) {
        cudaGraph_t tmp = nullptr;
        cudaStreamEndCapture(h->capture_stream, &tmp);
        if (tmp) cudaGraphDestroy(tmp);
        throw;
      }
      cudaGraph_t graph = nullptr;
      ck(cudaStreamEndCapture(h->capture_stream, &graph), "end capture");
      cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
      cudaGraphDestroy(graph);
      ck(e, "graph instantiate");
      g.key = key;
      g.launches = nl;
    }
    ck(cudaGraphLaunch(g.exec, stream), "graph launch");
    h->launches += g.launches;
  }
  h->s_now = s0 + n_finest;
}

// ------------------------------------------------------------------ discrete adjoint
struct DevBuf {
  void* p = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  template <typename T>
  T* get() const {
    return static_cast<T*>(p);
  }
  void alloc(size_t bytes) {
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      fail(LTS_ERR_OOM, "device allocation for the adjoint failed");
    }
  }
};

// Transposed copies of the operator tables for the adjoint kernels (their loops run over the
// other index of K_c, F~_i, F^_i and F-_{j,h} than the forward kernels' do).
struct AdjTables {
  DevBuf buf;
  const float *KT = nullptr, *FtT = nullptr, *FhT = nullptr, *FbT = nullptr;
};

void make_adj_tables(const lts_solver* h, AdjTables& T) {
  const int B = h->L.B, F = h->L.F;
  std::vector<float> K((size_t)3 * B * B), Ft((size_t)4 * B * F), Fh((size_t)4 * F * B), Fb((size_t)12 * B * F);
  auto down = [&](std::vector<float>& v, const float* src) {
    ck(cudaMemcpy(v.data(), src, sizeof(float) * v.size(), cudaMemcpyDeviceToHost), "download operators");
  };
  down(K, h->dops.K);
  down(Ft, h->dops.Ft);
  down(Fh, h->dops.Fh);
  down(Fb, h->dops.Fb);
  std::vector<float> all(K.size() + Ft.size() + Fh.size() + Fb.size());
  float* kt = all.data();
  float* ftt = kt + K.size();
  float* fht = ftt + Ft.size();
  float* fbt = fht + Fh.size();
  for (int c = 0; c < 3; ++c)
    for (int i = 0; i < B; ++i)
      for (int j = 0; j < B; ++j) kt[(c * B + j) * B + i] = K[(c * B + i) * B + j];
  for (int i = 0; i < 4; ++i)
    for (int b = 0; b < B; ++b)
      for (int f = 0; f < F; ++f) {
        ftt[(i * F + f) * B + b] = Ft[(i * B + b) * F + f];
        fht[(i * B + b) * F + f] = Fh[(i * F + f) * B + b];
      }
  for (int jh = 0; jh < 12; ++jh)
    for (int b = 0; b < B; ++b)
      for (int f = 0; f < F; ++f) fbt[(jh * F + f) * B + b] = Fb[(jh * B + b) * F + f];
  T.buf.alloc(sizeof(float) * all.size());
  ck(cudaMemcpy(T.buf.p, all.data(), sizeof(float) * all.size(), cudaMemcpyHostToDevice), "upload operators");
  const float* base = T.buf.get<float>();
  T.KT = base;
  T.FtT = base + (ftt - kt);
  T.FhT = base + (fht - kt);
  T.FbT = base + (fbt - kt);
}

// Material gradient from the correlations W (device, [internal element][AM_SIZE]): dJ/dp =
// sum <dM/dp, W> over the element's star matrices and face operators and over the operators
// of the neighbours' faces that look at it (they depend on this element's material through
// the Riemann state). One thread per element (original order); the derivatives are exact,
// by forward-mode dual numbers through the same closed forms the forward set-up evaluates
// (host_flux.h), contracted with W without forming the 9 x 9 matrices.
struct GradGeom {
  const double *jinv, *normal, *area, *detJ, *rho, *lam, *mu, *W;
  const int *bc, *nbr, *nbr_face;
  const long long* iperm;
  long long K;
};

__device__ lts::Dual grad_face_dot(const GradGeom& g, long long k, int face, int param) {
  using lts::Dual;
  auto mat = [&](long long e, int base, Dual* m) {
    m[0] = Dual(g.rho[e], param == base ? 1.0 : 0.0);
    m[1] = Dual(g.lam[e], param == base + 1 ? 1.0 : 0.0);
    m[2] = Dual(g.mu[e], param == base + 2 ? 1.0 : 0.0);
  };
  Dual own[3], oth[3];
  mat(k, 0, own);
  const Dual rinv = Dual(1.0) / own[0];
  const int bc = g.bc[4 * k + face];
  const long long nb = g.nbr[4 * k + face];
  if (nb >= 0)
    mat(nb, 3, oth);
  else
    for (int q = 0; q < 3; ++q) oth[q] = own[q];
  const Dual zp = lts::sqrt_t((own[1] + Dual(2.0) * own[2]) * own[0]), zs = lts::sqrt_t(own[2] * own[0]);
  const Dual zpo = nb >= 0 ? lts::sqrt_t((oth[1] + Dual(2.0) * oth[2]) * oth[0]) : zp;
  const Dual zso = nb >= 0 ? lts::sqrt_t(oth[2] * oth[0]) : zs;
  const Dual scale(-2.0 * g.area[4 * k + face] / g.detJ[k]);
  Dual cl[8], cn[8];
  lts::face_coefficients_t<Dual>(bc, zp, zs, zpo, zso, scale, cl, cn);
  const double* Wk = g.W + (size_t)g.iperm[k] * ltsdev::AM_SIZE;
  const double* n = g.normal + 12 * k + 3 * face;
  return lts::face_flux_dot<Dual>(n, cl, own[1], own[2], rinv, Wk + ltsdev::AM_LOC + face * 81) +
         lts::face_flux_dot<Dual>(n, cn, own[1], own[2], rinv, Wk + ltsdev::AM_NBR + face * 81);
}

__global__ void k_grad_contract(GradGeom g, double* grad) {
  using lts::Dual;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.K) return;
  const double* We = g.W + (size_t)g.iperm[e] * ltsdev::AM_SIZE;
  for (int p = 0; p < 3; ++p) {
    const Dual rho(g.rho[e], p == 0 ? 1.0 : 0.0), lam(g.lam[e], p == 1 ? 1.0 : 0.0), mu(g.mu[e], p == 2 ? 1.0 : 0.0);
    double acc = lts::star_dot<Dual>(g.jinv + 9 * e, lam, mu, Dual(1.0) / rho, We + ltsdev::AM_STAR).d;
    for (int i = 0; i < 4; ++i) {
      acc += grad_face_dot(g, e, i, p).d;
      const long long nb = g.nbr[4 * e + i];
      if (nb >= 0) acc += grad_face_dot(g, nb, g.nbr_face[4 * e + i], 3 + p).d;
    }
    grad[3 * e + p] = acc;
  }
}

// Explicit 9 x 9 operators of every element in FP32 (internal order): the star matrices S_c
// and, per face, the flux solvers A- (interior state) and A+ (exterior state), from the
// closed forms of the forward set-up (host_flux.h) evaluated in FP64. One thread per
// (element, task): task 0 the star matrices, task 1 + i face i.
__global__ void k_build_amat(GradGeom g, float* amat) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 5 * g.K) return;
  const long long k = t / 5;
  const int task = (int)(t % 5);
  float* out = amat + (size_t)g.iperm[k] * ltsdev::AM_SIZE;
  const double rho = g.rho[k], lam = g.lam[k], mu = g.mu[k], rinv = 1.0 / rho;
  if (task == 0) {
    double S[3][81];
    lts::star_matrices_t<double>(g.jinv + 9 * k, lam, mu, rinv, S);
    for (int c = 0; c < 3; ++c)
      for (int q = 0; q < 81; ++q) out[ltsdev::AM_STAR + c * 81 + q] = (float)S[c][q];
    return;
  }
  const int i = task - 1;
  const int bc = g.bc[4 * k + i];
  const long long nb = g.nbr[4 * k + i];
  const double zp = lts::sqrt_t((lam + 2.0 * mu) * rho), zs = lts::sqrt_t(mu * rho);
  const double zpo = nb >= 0 ? lts::sqrt_t((g.lam[nb] + 2.0 * g.mu[nb]) * g.rho[nb]) : zp;
  const double zso = nb >= 0 ? lts::sqrt_t(g.mu[nb] * g.rho[nb]) : zs;
  const double scale = -2.0 * g.area[4 * k + i] / g.detJ[k];
  double cl[8], cn[8], M[81];
  lts::face_coefficients_t<double>(bc, zp, zs, zpo, zso, scale, cl, cn);
  lts::face_flux_matrix<double>(g.normal + 12 * k + 3 * i, cl, lam, mu, rinv, M);
  for (int q = 0; q < 81; ++q) out[ltsdev::AM_LOC + i * 81 + q] = (float)M[q];
  lts::face_flux_matrix<double>(g.normal + 12 * k + 3 * i, cn, lam, mu, rinv, M);
  for (int q = 0; q < 81; ++q) out[ltsdev::AM_NBR + i * 81 + q] = (float)M[q];
}

// Geometry and material of every element on the device (original element order), for the
// operator build and the gradient contraction; the buffers live as long as `bufs`.
struct GeoBufs {
  DevBuf dbl, ints, perm;
};
GradGeom upload_geometry(const lts_solver* h, GeoBufs& bufs, cudaStream_t stream) {
  const lts::Mesh& M = h->mesh;
  const int64_t K = M.K;
  std::vector<int> bc(4 * K), nbr(4 * K), nface(4 * K);
  std::vector<long long> iperm(K);
  for (int64_t i = 0; i < 4 * K; ++i) {
    bc[i] = M.bc[i];
    nbr[i] = (int)M.nbr[i];
    nface[i] = M.nbr_face[i];
  }
  for (int64_t k = 0; k < K; ++k) iperm[k] = (long long)h->iperm[k];
  const size_t nd = (size_t)K * (9 + 12 + 4 + 1 + 3);
  bufs.dbl.alloc(sizeof(double) * nd);
  bufs.ints.alloc(sizeof(int) * 12 * K);
  bufs.perm.alloc(sizeof(long long) * K);
  double* geo = bufs.dbl.get<double>();
  int* in = bufs.ints.get<int>();
  auto up = [&](void* dst, const void* src, size_t bytes) {
    ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream), "adjoint geometry");
  };
  GradGeom g{};
  g.jinv = geo;
  g.normal = geo + 9 * K;
  g.area = geo + 21 * K;
  g.detJ = geo + 25 * K;
  g.rho = geo + 26 * K;
  g.lam = geo + 27 * K;
  g.mu = geo + 28 * K;
  g.bc = in;
  g.nbr = in + 4 * K;
  g.nbr_face = in + 8 * K;
  g.iperm = bufs.perm.get<long long>();
  g.K = K;
  up(const_cast<double*>(g.jinv), M.Jinv.data(), sizeof(double) * 9 * K);
  up(const_cast<double*>(g.normal), M.normal.data(), sizeof(double) * 12 * K);
  up(const_cast<double*>(g.area), M.area.data(), sizeof(double) * 4 * K);
  up(const_cast<double*>(g.detJ), M.detJ.data(), sizeof(double) * K);
  up(const_cast<double*>(g.rho), h->mat.rho.data(), sizeof(double) * K);
  up(const_cast<double*>(g.lam), h->lam.data(), sizeof(double) * K);
  up(const_cast<double*>(g.mu), h->mu.data(), sizeof(double) * K);
  up(in, bc.data(), sizeof(int) * 4 * K);
  up(in + 4 * K, nbr.data(), sizeof(int) * 4 * K);
  up(in + 8 * K, nface.data(), sizeof(int) * 4 * K);
  up(bufs.perm.p, iperm.data(), sizeof(long long) * K);
  // the host vectors must outlive the copies: the stream is synchronised before they go
  ck(cudaStreamSynchronize(stream), "synchronize");
  return g;
}

void contract_gradient(GradGeom g, const double* d_w, double* grad, cudaStream_t stream) {
  g.W = d_w;
  DevBuf d_grad;
  d_grad.alloc(sizeof(double) * 3 * g.K);
  const int threads = 128;
  k_grad_contract<<<(unsigned)((g.K + threads - 1) / threads), threads, 0, stream>>>(g, d_grad.get<double>());
  ck(cudaGetLastError(), "gradient contraction");
  ck(cudaMemcpyAsync(grad, d_grad.p, sizeof(double) * 3 * g.K, cudaMemcpyDeviceToHost, stream), "download gradient");
  ck(cudaStreamSynchronize(stream), "synchronize");
}


// Clustered-LTS branch of lts_misfit_gradient: samples at the macro-step boundaries, Q
// checkpoints every `every` macro steps, and per macro step a phase-by-phase recompute
// that keeps Q before each predict pass and the buffers before each neighbour pass for the
// reverse sweep (k_adj_pred / k_adj_nbr, phases in reverse order).
void adjoint_lts(lts_solver* h, int64_t n_macro, int64_t every, const double* data, double* misfit, double* grad,
                 double* synth_out, double* dq0, cudaStream_t stream, const DevBuf& d_amat, const DevBuf& d_fwd,
                 const DevBuf& d_back, const DevBuf& d_relem, const DevBuf& d_rphi, int nrec, const AdjTables& tabs,
                 const GradGeom& geo, const DevBuf& d_own, const std::vector<int64_t>& own_off) {
  const Launchers& X = h->L;
  const int64_t K = h->mesh.K;
  const int B = X.B, NB9 = 9 * B;
  const int64_t qs = h->dst.qs, bs = h->dst.bs;
  const int64_t period = int64_t(1) << (h->nc - 1);
  const int64_t ncp = (n_macro + every - 1) / every;
  const int64_t segm = std::min(every, n_macro);
  // fused runs: nsim simulations in groups of G; samples [time][sim][receiver][3], adjoints
  // [element][sim][9][B]
  const int nsim = h->nsim, G = nsim > 1 ? X.FG : 1;
  h->adj_src_grad.clear();   // set again only by a completed reverse sweep
  const int64_t ns = (int64_t)nsim * nrec * 3;   // sample values per sample time
  // the reverse sweep's state (adjoints, correlations, checkpoints) only when it runs
  const bool reverse = grad || dq0;
  DevBuf d_syn, d_res, d_lq, d_lb, d_w, d_cp, d_mac, d_qn;
  d_syn.alloc(sizeof(float) * (n_macro + 1) * ns);
  if (reverse) {
    d_res.alloc(sizeof(float) * (n_macro + 1) * ns);
    d_lq.alloc(sizeof(float) * K * nsim * NB9);
    d_lb.alloc(sizeof(float) * 3 * K * nsim * NB9);
    d_w.alloc(sizeof(double) * K * ltsdev::AM_SIZE);
    d_cp.alloc(sizeof(float) * ncp * K * qs);
    d_qn.alloc(sizeof(float) * K * qs);
  }
  // moment-tensor gradient: [source][6] and one pass's source items with their scales
  const int nsrc = (int)h->sources.size();
  DevBuf d_sg, d_sgi, d_sgc;
  d_sg.alloc(sizeof(double) * std::max(nsrc, 1) * 6);
  d_sgi.alloc(sizeof(SrcItem) * std::max(nsrc, 1));
  d_sgc.alloc(sizeof(double) * std::max(nsrc, 1));
  const size_t qbytes = sizeof(float) * K * qs;
  auto dcopy = [&](void* dst, const void* src, size_t bytes) {
    ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, stream), "adjoint copy");
  };
  float* cp = d_cp.get<float>();
  const int* relem = d_relem.get<int>();
  const float* rphi = d_rphi.get<float>();
  // ---- forward sweep: samples at the macro boundaries, checkpoints
  const int64_t s0 = h->s_now;
  std::vector<size_t> nrec_t(nrec);
  X.adj_sample(h->dst.Q, qs, nsim, G, relem, rphi, nrec, d_syn.get<float>(), stream);
  for (int64_t m = 0; m < n_macro; ++m) {
    if (reverse && m % every == 0) dcopy(cp + (m / every) * K * qs, h->dst.Q, qbytes);
    advance_steps(h, period, stream);
    X.adj_sample(h->dst.Q, qs, nsim, G, relem, rphi, nrec, d_syn.get<float>() + (m + 1) * ns, stream);
  }
  for (int r = 0; r < nrec; ++r) nrec_t[r] = h->receivers[r].t.size();
  const size_t seis_fwd = h->seis_used;
  if (reverse) dcopy(d_qn.p, h->dst.Q, qbytes);
  std::vector<float> syn((size_t)(n_macro + 1) * ns);
  ck(cudaMemcpyAsync(syn.data(), d_syn.p, sizeof(float) * syn.size(), cudaMemcpyDeviceToHost, stream), "samples");
  ck(cudaStreamSynchronize(stream), "synchronize");
  check_device_error(h);
  std::vector<float> res(syn.size());
  double J = 0.0;
  for (size_t q = 0; q < syn.size(); ++q) {
    const double r = (double)syn[q] - data[q];
    res[q] = (float)r;
    J += 0.5 * r * r;
  }
  if (misfit) *misfit = J;
  if (synth_out)
    for (size_t q = 0; q < syn.size(); ++q) synth_out[q] = syn[q];
  if (!grad && !dq0) return;       // misfit only: no reverse sweep
  ck(cudaMemcpyAsync(d_res.p, res.data(), sizeof(float) * res.size(), cudaMemcpyHostToDevice, stream), "residuals");
  // ---- reverse sweep
  ck(cudaMemsetAsync(d_lq.p, 0, sizeof(float) * K * nsim * NB9, stream), "memset");
  ck(cudaMemsetAsync(d_lb.p, 0, sizeof(float) * 3 * K * nsim * NB9, stream), "memset");
  ck(cudaMemsetAsync(d_w.p, 0, sizeof(double) * K * ltsdev::AM_SIZE, stream), "memset");
  ck(cudaMemsetAsync(d_sg.p, 0, sizeof(double) * std::max(nsrc, 1) * 6, stream), "memset");
  X.adj_source(d_lq.get<float>(), nsim, relem, rphi, d_res.get<float>() + n_macro * ns, nrec, stream);
  ltsdev::AdjLtsArgs aa{};
  aa.lq = d_lq.get<float>();
  aa.lb1 = d_lb.get<float>();
  aa.lb2 = aa.lb1 + K * nsim * NB9;
  aa.lb3 = aa.lb2 + K * nsim * NB9;
  aa.nsim = nsim;
  aa.G = G;
  aa.amat = d_amat.get<float>();
  aa.fwd = d_fwd.get<int>();
  aa.back = d_back.get<int>();
  aa.meta = h->dst.meta;
  aa.W = d_w.get<double>();
  aa.KT = tabs.KT;
  aa.FtT = tabs.FtT;
  aa.FhT = tabs.FhT;
  aa.FbT = tabs.FbT;
  aa.qs = qs;
  aa.bufs = bs;
  MacroPlan mp;
  // Phase layout of a macro step (the same for every macro step; the step indices are
  // relative) and the bytes each phase's reverse reads: Q of the active elements before a
  // predict pass, B1, B2, B3 of the buffer owners before a neighbour pass. Elements are in
  // cluster order, so both are prefixes.
  std::vector<Phase> lay;
  std::vector<size_t> snap_off, snap_len;
  size_t per_macro = 0;
  {
    size_t seis_need = h->seis_used;
    plan_macro(h, s0, seis_need, mp);
    for (int r = 0; r < nrec; ++r) {
      h->receivers[r].t.resize(nrec_t[r]);
      h->receivers[r].slot.resize(nrec_t[r]);
    }
    for (const Phase& ph : mp.phases) {
      Phase q = ph;
      q.s -= s0;
      lay.push_back(q);
      const int64_t n = ph.kind == 1 ? h->cbeg[ph.top + 1] : h->cbeg[std::min(ph.top + 2, h->nc)];
      const size_t len = ph.kind == 1 ? sizeof(float) * n * qs : 3 * sizeof(float) * n * bs;
      snap_off.push_back(per_macro);
      snap_len.push_back(len);
      per_macro += (len + 255) / 256 * 256;
    }
  }
  auto phase_at = [&](size_t pi, int64_t sb0) {
    Phase q = lay[pi];
    q.s += sb0;
    return q;
  };
  // reverse of one macro step from the phase inputs kept in `snap` (layout above)
  MacroPlan smp;   // the reversed macro step's source items
  auto reverse_macro = [&](int64_t m, const char* snap) {
    const int64_t sb0 = s0 + m * period;
    if (nsrc > 0) {
      size_t seis_need = h->seis_used;
      plan_macro(h, sb0, seis_need, smp);
      for (int r = 0; r < nrec; ++r) {
        h->receivers[r].t.resize(nrec_t[r]);
        h->receivers[r].slot.resize(nrec_t[r]);
      }
    }
    for (size_t pi = lay.size(); pi-- > 0;) {
      const Phase ph = phase_at(pi, sb0);
      if (nsrc > 0 && ph.kind == 0) {
        // the sources this neighbour pass added: lambda_Q is now the adjoint of Q after it
        const Phase& sp = smp.phases[pi];
        const int n = sp.item_end - sp.item_beg;
        if (n > 0) {
          ck(cudaMemcpyAsync(d_sgi.p, smp.sitems.data() + sp.item_beg, sizeof(SrcItem) * n, cudaMemcpyHostToDevice,
                             stream),
             "source items");
          ck(cudaMemcpyAsync(d_sgc.p, smp.sscale.data() + sp.item_beg, sizeof(double) * n, cudaMemcpyHostToDevice,
                             stream),
             "source scales");
          X.adj_src_grad(d_lq.get<float>(), nsim, d_sgi.get<SrcItem>(), d_sgc.get<double>(), n, h->d_src_phi,
                         d_sg.get<double>(), stream);
        }
      }
      const PhaseArgs pa = phase_args(h, ph);
      if (pa.end <= 0) continue;
      aa.end = pa.end;
      const float* base = reinterpret_cast<const float*>(snap + snap_off[pi]);
      if (ph.kind == 1) {
        aa.Qs = base;
        // the sparse engine's reverse predict (one or fused simulations); the other engines
        // take the dense-block kernel
        if (h->contraction == LTS_CONTRACT_SPARSE && X.adj_pred_sp)
          X.adj_pred_sp(aa, pa, pa.end, stream);
        else
          X.adj_pred(h->dops, aa, pa, pa.end, stream);
      } else {
        // a buffer owner differs by at most one cluster from the receivers it feeds, so
        // the owners of this pass are among the elements of clusters 0..top+1 (the buffer
        // snapshots' extent); one CTA for each that has an active receiver
        const int owners = (int)h->cbeg[std::min(ph.top + 2, h->nc)];
        aa.B1s = base;
        aa.B2s = base + (size_t)owners * bs;
        aa.B3s = base + 2 * (size_t)owners * bs;
        aa.bufs = bs;
        aa.owners = d_own.get<int>() + own_off[ph.top];
        X.adj_nbr(h->dops, aa, pa, (int)(own_off[ph.top + 1] - own_off[ph.top]), stream);
      }
    }
    X.adj_source(d_lq.get<float>(), nsim, relem, rphi, d_res.get<float>() + m * ns, nrec, stream);
  };
  // forward replay of macro step m, keeping every phase's inputs in `snap`
  auto replay_macro = [&](int64_t m, char* snap) {
    const int64_t sb0 = s0 + m * period;
    h->s_now = sb0;
    size_t seis_need = h->seis_used;
    plan_macro(h, sb0, seis_need, mp);
    ensure_capacity(reinterpret_cast<void**>(&h->d_sitems), &h->sitems_cap, mp.sitems.size(), sizeof(SrcItem));
    if (!mp.sitems.empty())
      ck(cudaMemcpyAsync(h->d_sitems, mp.sitems.data(), mp.sitems.size() * sizeof(SrcItem), cudaMemcpyHostToDevice,
                         stream),
         "upload source items");
    for (size_t pi = 0; pi < mp.phases.size(); ++pi) {
      const Phase& ph = mp.phases[pi];
      char* dst = snap + snap_off[pi];
      if (ph.kind == 1) {
        dcopy(dst, h->dst.Q, snap_len[pi]);
      } else {
        const size_t one = snap_len[pi] / 3;
        dcopy(dst, h->dst.B1, one);
        dcopy(dst + one, h->dst.B2, one);
        dcopy(dst + 2 * one, h->dst.B3, one);
      }
      enqueue_phase(h, ph, stream, false);
    }
    for (int r = 0; r < nrec; ++r) {
      h->receivers[r].t.resize(nrec_t[r]);
      h->receivers[r].slot.resize(nrec_t[r]);
    }
    h->seis_used = seis_fwd;
  };
  // The inputs of a whole segment's phases are kept when they fit in half the free device
  // memory: one forward replay per segment. Otherwise the segment's macro-boundary states are
  // kept and each macro step is replayed once more just before its reverse.
  size_t free_b = 0, total_b = 0;
  ck(cudaMemGetInfo(&free_b, &total_b), "memory info");
  const double budget = h->adj_budget ? (double)h->adj_budget : 0.5 * (double)free_b;
  const bool whole_segment = (double)segm * (double)per_macro <= budget;
  DevBuf d_snap;
  d_snap.alloc(whole_segment ? segm * per_macro : per_macro);
  char* snap = d_snap.get<char>();
  if (!whole_segment) d_mac.alloc(sizeof(float) * segm * K * qs);
  float* mac = d_mac.get<float>();
  for (int64_t sgi = ncp - 1; sgi >= 0; --sgi) {
    const int64_t m0 = sgi * every, m1 = std::min(m0 + every, n_macro);
    dcopy(h->dst.Q, cp + sgi * K * qs, qbytes);
    h->s_now = s0 + m0 * period;
    if (whole_segment) {
      for (int64_t m = m0; m < m1; ++m) replay_macro(m, snap + (m - m0) * per_macro);
      for (int64_t m = m1 - 1; m >= m0; --m) reverse_macro(m, snap + (m - m0) * per_macro);
      continue;
    }
    // macro-boundary states of the segment
    dcopy(mac, h->dst.Q, qbytes);
    for (int64_t m = m0; m + 1 < m1; ++m) {
      advance_steps(h, period, stream);
      dcopy(mac + (m + 1 - m0) * K * qs, h->dst.Q, qbytes);
    }
    for (int64_t m = m1 - 1; m >= m0; --m) {
      dcopy(h->dst.Q, mac + (m - m0) * K * qs, qbytes);
      replay_macro(m, snap);
      reverse_macro(m, snap);
    }
  }
  ck(cudaGetLastError(), "adjoint kernels");
  dcopy(h->dst.Q, d_qn.p, qbytes);
  h->s_now = s0 + n_macro * period;
  h->adj_src_grad.assign((size_t)nsrc * 6, 0.0);
  if (nsrc > 0)
    ck(cudaMemcpyAsync(h->adj_src_grad.data(), d_sg.p, sizeof(double) * nsrc * 6, cudaMemcpyDeviceToHost, stream),
       "source gradient");
  std::vector<float> lq;
  if (dq0) {
    lq.resize((size_t)K * nsim * NB9);
    ck(cudaMemcpyAsync(lq.data(), d_lq.p, sizeof(float) * lq.size(), cudaMemcpyDeviceToHost, stream), "adjoint state");
  }
  ck(cudaStreamSynchronize(stream), "synchronize");
  check_device_error(h);
  if (misfit) *misfit = J;
  if (synth_out)
    for (size_t q = 0; q < syn.size(); ++q) synth_out[q] = syn[q];
  if (dq0)   // [sim][element (original order)][9][B]
    for (int f = 0; f < nsim; ++f)
      for (int64_t k = 0; k < K; ++k)
        for (int q = 0; q < NB9; ++q)
          dq0[((size_t)f * K + k) * NB9 + q] = lq[((size_t)h->iperm[k] * nsim + f) * NB9 + q];
  if (grad) contract_gradient(geo, d_w.get<double>(), grad, stream);
}

}  // namespace

namespace ltsdev {
cudaError_t measure_peaks(cudaStream_t stream, double* out);   // peaks.cu
}

extern "C" {

int lts_create(int order, int n_mech, int n_fused, int device, lts_t** out) {
  const bool fused_ok = n_fused == 1 || (n_fused > 0 && n_fused <= LTS_MAX_FUSED && n_fused % LTS_FUSED_MULTIPLE == 0);
  if (!out || order < 3 || order > 5 || (n_mech != 0 && n_mech != 3) || !fused_ok) return LTS_ERR_ARG;
  lts_solver* h = nullptr;
  try {
    h = new lts_solver();
  } catch (...) {
    return LTS_ERR_OOM;
  }
  int rc = run(h, [&] {
    h->order = order;
    h->nmech = n_mech;
    h->device = device;
    h->nsim = n_fused;
    if (!ltsdev::get_launchers(order, n_mech, n_fused > 1, &h->L)) fail(LTS_ERR_ARG, "unsupported order / mechanisms");
    if (n_fused > 1 && n_fused % h->L.FG != 0) fail(LTS_ERR_ARG, "fused count not a multiple of the CTA group");
    // one simulation: the sparse-product kernels by default (the fastest FP32 engine there;
    // with fused simulations the dense-block kernels, whose slots keep the simulations of an
    // element in the innermost 16 bytes, are faster)
    if (h->L.predict_sp) h->contraction = LTS_CONTRACT_SPARSE;
    if (device >= 0) {
      ck(cudaSetDevice(device), "cudaSetDevice");
      ck(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device), "device attribute");
      ck(h->L.init(&h->L), "kernel attributes");
    }
    h->ops.build(order);
  });
  if (rc != LTS_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return LTS_OK;
}

void lts_destroy(lts_t* h) {
  if (!h) return;
  if (h->device >= 0) cudaSetDevice(h->device);
  free_device(h);
  release_events(h);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  delete h;
}

const char* lts_last_error(lts_t* h) { return h ? h->err.c_str() : "null handle"; }

int lts_set_mesh(lts_t* h, int64_t n_vert, const double* xyz, int64_t n_tet, const int64_t* tet, const int32_t* face_bc,
                 const double* period) {
  return run(h, [&] {
    if (n_vert <= 0 || n_tet <= 0 || !xyz || !tet || !face_bc) fail(LTS_ERR_ARG, "bad mesh arguments");
    if (n_tet > (int64_t(1) << 30)) fail(LTS_ERR_ARG, "too many elements");
    if (n_tet * h->nsim > INT32_MAX) fail(LTS_ERR_ARG, "too many (element, simulation) slots");
    lts::Mesh m;
    m.nv = n_vert;
    m.K = n_tet;
    m.xyz.assign(xyz, xyz + 3 * n_vert);
    m.tet.assign(tet, tet + 4 * n_tet);
    m.bc.assign(face_bc, face_bc + 4 * n_tet);
    if (period) {
      m.periodic = true;
      for (int d = 0; d < 3; ++d) {
        if (!(period[d] > 0.0)) fail(LTS_ERR_ARG, "period must be positive");
        m.period[d] = period[d];
      }
    }
    for (int32_t c : m.bc)
      if (c < 0 || c > 3) fail(LTS_ERR_ARG, "bad face code");
    lts::Error e{0, ""};
    if (lts::build_mesh(m, e) != 0) fail(e.code == -1 ? LTS_ERR_ARG : LTS_ERR_MESH, e.msg);
    free_device(h);
    h->mesh = std::move(m);
    h->has_mesh = true;
    h->part.clear();
    h->n_parts = 1;
    h->has_mat = false;
    h->sources.clear();
    h->receivers.clear();
  });
}

int lts_set_material(lts_t* h, const double* rho, const double* vp, const double* vs, const double* qp,
                     const double* qs, double f_min, double f_max) {
  return run(h, [&] {
    if (!h->has_mesh) fail(LTS_ERR_STATE, "no mesh");
    if (!rho || !vp || !vs) fail(LTS_ERR_ARG, "missing material arrays");
    const int64_t K = h->mesh.K;
    const int m = h->nmech;
    if (m > 0 && (!qp || !qs || !(f_min > 0.0) || !(f_max > f_min))) fail(LTS_ERR_ARG, "missing Q model");
    lts::Material mt;
    mt.rho.assign(rho, rho + K);
    mt.vp.assign(vp, vp + K);
    mt.vs.assign(vs, vs + K);
    h->lam.resize(K);
    h->mu.resize(K);
    for (int64_t k = 0; k < K; ++k) {
      if (!(rho[k] > 0.0) || !(vp[k] > 0.0) || !(vs[k] > 0.0)) fail(LTS_ERR_ARG, "non-positive material value");
      h->mu[k] = rho[k] * vs[k] * vs[k];
      h->lam[k] = rho[k] * vp[k] * vp[k] - 2.0 * h->mu[k];
    }
    h->omega.assign(m, 0.0);
    h->ylam.assign(K * m, 0.0);
    h->ymu.assign(K * m, 0.0);
    if (m > 0) {
      mt.qp.assign(qp, qp + K);
      mt.qs.assign(qs, qs + K);
      mt.f_min = f_min;
      mt.f_max = f_max;
      lts::relaxation_frequencies(m, f_min, f_max, h->omega.data());
      std::vector<double> ys(m), yp(m);
      for (int64_t k = 0; k < K; ++k) {
        if (!(qp[k] > 0.0) || !(qs[k] > 0.0)) fail(LTS_ERR_ARG, "non-positive Q");
        if (lts::fit_y(m, qs[k], h->omega.data(), ys.data()) != 0 ||
            lts::fit_y(m, qp[k], h->omega.data(), yp.data()) != 0)
          fail(LTS_ERR_ARG, "singular relaxation fit");
        for (int l = 0; l < m; ++l) {
          h->ymu[k * m + l] = ys[l];
          h->ylam[k * m + l] = ((h->lam[k] + 2.0 * h->mu[k]) * yp[l] - 2.0 * h->mu[k] * ys[l]) / h->lam[k];
        }
      }
    }
    free_device(h);
    h->mat = std::move(mt);
    h->has_mat = true;
  });
}

int lts_setup_clusters(lts_t* h, int n_clusters, double cfl, double lambda, int32_t* cluster_out, double* lambda_out,
                       double* speedup_out) {
  return run(h, [&] {
    require_material(h);
    if (n_clusters < 1 || n_clusters > ltsdev::MAXC || !(cfl > 0.0) || lambda > 1.0)
      fail(LTS_ERR_ARG, "bad cluster arguments");
    if (lambda > 0.0 && lambda <= 0.5) fail(LTS_ERR_ARG, "lambda must lie in (0.5, 1]");
    if (h->device >= 0) ck(cudaSetDevice(h->device), "cudaSetDevice");
    std::vector<double> dt;
    lts::cfl_time_steps(h->mesh, h->mat, h->order, cfl, dt);
    h->dt_min = *std::min_element(dt.begin(), dt.end());
    h->nc = n_clusters;
    if (lambda <= 0.0) {
      h->lambda = lts::search_lambda(h->mesh, dt, n_clusters, h->cluster, nullptr);
    } else {
      h->lambda = lambda;
      lts::assign_clusters(dt, lambda, n_clusters, h->cluster);
      lts::normalise_clusters(h->mesh, h->cluster);
    }
    finish_clusters(h, lambda_out, speedup_out, cluster_out);
  });
}

int lts_force_clusters(lts_t* h, int n_clusters, const int32_t* clusters, double cfl, double lambda) {
  return run(h, [&] {
    require_material(h);
    if (n_clusters < 1 || n_clusters > ltsdev::MAXC || !clusters || !(cfl > 0.0) || lambda > 1.0)
      fail(LTS_ERR_ARG, "bad cluster arguments");
    if (h->device >= 0) ck(cudaSetDevice(h->device), "cudaSetDevice");
    std::vector<double> dt;
    lts::cfl_time_steps(h->mesh, h->mat, h->order, cfl, dt);
    h->dt_min = *std::min_element(dt.begin(), dt.end());
    h->nc = n_clusters;
    h->lambda = lambda > 0.0 ? lambda : 1.0;
    h->cluster.assign(clusters, clusters + h->mesh.K);
    for (int32_t c : h->cluster)
      if (c < 0 || c >= n_clusters) fail(LTS_ERR_ARG, "cluster index out of range");
    finish_clusters(h, nullptr, nullptr, nullptr);
  });
}

int lts_state_bytes(lts_t* h, int n_clusters, int64_t* bytes) {
  return run(h, [&] {
    require_material(h);
    (void)n_clusters;
    if (!bytes) fail(LTS_ERR_ARG, "null output");
    *bytes = (int64_t)layout_of(h, h->mesh.K).total;
  });
}

int lts_bind_device_memory(lts_t* h, void* dev, int64_t bytes) {
  return run(h, [&] {
    if (dev && (reinterpret_cast<uintptr_t>(dev) % 256 != 0)) fail(LTS_ERR_ARG, "device block must be 256-byte aligned");
    free_device(h);
    h->bound = dev;
    h->bound_bytes = dev ? (size_t)bytes : 0;
  });
}

int lts_quadrature_points(lts_t* h, int64_t* n_per_elem, double* xyz_out) {
  return run(h, [&] {
    if (!h->has_mesh) fail(LTS_ERR_STATE, "no mesh");
    const int64_t np = (int64_t)h->ops.qp.size();
    if (n_per_elem) *n_per_elem = np;
    if (!xyz_out) return;
    const lts::Mesh& M = h->mesh;
    for (int64_t k = 0; k < M.K; ++k)
      for (int64_t p = 0; p < np; ++p)
        for (int d = 0; d < 3; ++d) {
          const auto& xi = h->ops.qp[p];
          xyz_out[(k * np + p) * 3 + d] =
              M.x0[3 * k + d] + M.J[9 * k + d * 3 + 0] * xi[0] + M.J[9 * k + d * 3 + 1] * xi[1] + M.J[9 * k + d * 3 + 2] * xi[2];
        }
  });
}

// Host DOF arrays are simulation-major, [F][n][N^q][B] (F = 1: [n][N^q][B]); on the device
// an element's row holds simulation groups of G = FG: [F/G][N^q][B][G].
static int64_t row_index(const lts_t* h, int r, int b, int f) {
  const int B = h->L.B, NQ = h->L.NQ, G = h->L.FG;
  return (int64_t)(f / G) * NQ * B * G + ((int64_t)r * B + b) * G + f % G;
}

static void pack_row(const lts_t* h, const double* dofs, int64_t n, int64_t i, float* row) {
  const int B = h->L.B, NQ = h->L.NQ, F = h->nsim;
  for (int f = 0; f < F; ++f)
    for (int r = 0; r < NQ; ++r)
      for (int b = 0; b < B; ++b) row[row_index(h, r, b, f)] = (float)dofs[((f * n + i) * NQ + r) * B + b];
}

static void unpack_row(const lts_t* h, const float* row, int64_t n, int64_t i, double* dofs) {
  const int B = h->L.B, NQ = h->L.NQ, F = h->nsim;
  for (int f = 0; f < F; ++f)
    for (int r = 0; r < NQ; ++r)
      for (int b = 0; b < B; ++b) dofs[((f * n + i) * NQ + r) * B + b] = row[row_index(h, r, b, f)];
}

static void upload_dofs(lts_t* h, const double* dofs) {
  const int64_t K = h->mesh.K, qs = h->dst.qs;
  std::vector<float> q((size_t)K * qs, 0.f);
  for (int64_t k = 0; k < K; ++k) pack_row(h, dofs, K, k, &q[h->iperm[k] * qs]);
  ck(cudaSetDevice(h->device), "cudaSetDevice");
  ck(cudaMemcpy(h->dst.Q, q.data(), q.size() * sizeof(float), cudaMemcpyHostToDevice), "upload Q");
}

int lts_project_initial(lts_t* h, const double* values) {
  return run(h, [&] {
    if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
    if (!values) fail(LTS_ERR_ARG, "null values");
    const int64_t K = h->mesh.K;
    const int B = h->L.B, NQ = h->L.NQ;
    const int64_t np = (int64_t)h->ops.qp.size();
    std::vector<double> phiq(np * B);
    for (int64_t p = 0; p < np; ++p) h->ops.eval(h->ops.qp[p].data(), &phiq[p * B]);
    std::vector<double> dofs((size_t)h->nsim * K * NQ * B, 0.0);
    for (int64_t k = 0; k < K; ++k)
      for (int64_t p = 0; p < np; ++p) {
        const double w = h->ops.qw[p];
        for (int r = 0; r < NQ; ++r) {
          const double v = w * values[(k * np + p) * NQ + r];
          for (int b = 0; b < B; ++b) dofs[(k * NQ + r) * B + b] += v * phiq[p * B + b];
        }
      }
    const size_t one = (size_t)K * NQ * B;
    for (int f = 1; f < h->nsim; ++f) std::copy(dofs.begin(), dofs.begin() + one, dofs.begin() + f * one);
    upload_dofs(h, dofs.data());
  });
}

int lts_set_dofs(lts_t* h, const double* dofs) {
  return run(h, [&] {
    if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
    if (!dofs) fail(LTS_ERR_ARG, "null dofs");
    upload_dofs(h, dofs);
  });
}

int lts_get_dofs(lts_t* h, double* dofs) {
  return run(h, [&] {
    if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
    if (!dofs) fail(LTS_ERR_ARG, "null dofs");
    const int64_t K = h->mesh.K, qs = h->dst.qs;
    std::vector<float> q((size_t)K * qs);
    ck(cudaSetDevice(h->device), "cudaSetDevice");
    ck(cudaDeviceSynchronize(), "synchronize");
    ck(cudaMemcpy(q.data(), h->dst.Q, q.size() * sizeof(float), cudaMemcpyDeviceToHost), "download Q");
    check_device_error(h);
    for (int64_t k = 0; k < K; ++k) unpack_row(h, &q[h->iperm[k] * qs], K, k, dofs);
  });
}

int lts_set_dofs_subset(lts_t* h, int64_t n, const int64_t* elems, const double* dofs) {
  return run(h, [&] {
    if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
    if (n < 0 || (n > 0 && (!elems || !dofs))) fail(LTS_ERR_ARG, "bad subset arguments");
    const int64_t qs = h->dst.qs;
    std::vector<float> row(qs, 0.f);
    ck(cudaSetDevice(h->device), "cudaSetDevice");
    ck(cudaDeviceSynchronize(), "synchronize");
    for (int64_t i = 0; i < n; ++i) {
      const int64_t k = elems[i];
      if (k < 0 || k >= h->mesh.K) fail(LTS_ERR_ARG, "element index out of range");
      pack_row(h, dofs, n, i, row.data());
      ck(cudaMemcpy(h->dst.Q + h->iperm[k] * qs, row.data(), qs * sizeof(float), cudaMemcpyHostToDevice), "upload");
    }
  });
}

int lts_get_dofs_subset(lts_t* h, int64_t n, const int64_t* elems, double* dofs) {
  return run(h, [&] {
    if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
    if (n < 0 || (n > 0 && (!elems || !dofs))) fail(LTS_ERR_ARG, "bad subset arguments");
    const int64_t qs = h->dst.qs;
    std::vector<float> row(qs);
    ck(cudaSetDevice(h->device), "cudaSetDevice");
    ck(cudaDeviceSynchronize(), "synchronize");
    check_device_error(h);
    for (int64_t i = 0; i < n; ++i) {
      const int64_t k = elems[i];
      if (k < 0 || k >= h->mesh.K) fail(LTS_ERR_ARG, "element index out of range");
      ck(cudaMemcpy(row.data(), h->dst.Q + h->iperm[k] * qs, qs * sizeof(float), cudaMemcpyDeviceToHost), "download");
      unpack_row(h, row.data(), n, i, dofs);
    }
  });
}

int lts_add_point_source(lts_t* h, int fused_idx, const double x[3], const double m6[6], double f0, double t0,
                         double m0) {
  return run(h, [&] {
    if (!h->has_mesh) fail(LTS_ERR_STATE, "no mesh");
    if (fused_idx < 0 || fused_idx >= h->nsim || !x || !m6) fail(LTS_ERR_ARG, "bad source arguments");
    Source s;
    s.sim = fused_idx;
    s.elem = lts::locate(h->mesh, x, s.xi);
    if (s.elem < 0) fail(LTS_ERR_ARG, "source outside the mesh");
    std::copy(m6, m6 + 6, s.m6);
    s.f0 = f0;
    s.t0 = t0;
    s.m0 = m0;
    s.phi.resize(h->L.B);
    h->ops.eval(s.xi, s.phi.data());
    h->sources.push_back(std::move(s));
    h->ready = false;
  });
}

int lts_add_receiver(lts_t* h, const double x[3], double dt_sample, int* id) {
  return run(h, [&] {
    if (!h->has_mesh) fail(LTS_ERR_STATE, "no mesh");
    if (!x || !(dt_sample > 0.0)) fail(LTS_ERR_ARG, "bad receiver arguments");
    Receiver r;
    r.elem = lts::locate(h->mesh, x, r.xi);
    if (r.elem < 0) fail(LTS_ERR_ARG, "receiver outside the mesh");
    r.dt = dt_sample;
    r.phi.resize(h->L.B);
    h->ops.eval(r.xi, r.phi.data());
    h->receivers.push_back(std::move(r));
    if (id) *id = (int)h->receivers.size() - 1;
    h->ready = false;
  });
}

int lts_advance_steps(lts_t* h, int64_t n_finest, void* cuda_stream) {
  return run(h, [&] {
    if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
    ck(cudaSetDevice(h->device), "cudaSetDevice");
    advance_steps(h, n_finest, static_cast<cudaStream_t>(cuda_stream));
  });
}

int lts_advance(lts_t* h, double t_end, void* cuda_stream) {
  return run(h, [&] {
    if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
    const int64_t period = int64_t(1) << (h->nc - 1);
    const double macro = h->delta * period;
    const double tnow = h->s_now * h->delta;
    const int64_t nmac = (int64_t)std::floor((t_end - tnow) / macro * (1.0 + 1e-9) + 1e-9);
    if (nmac <= 0) return;
    ck(cudaSetDevice(h->device), "cudaSetDevice");
    advance_steps(h, nmac * period, static_cast<cudaStream_t>(cuda_stream));
  });
}

int lts_get_seismogram(lts_t* h, int id, int fused_idx, double* t_out, double* v_out, int64_t cap, int64_t* n) {
  return run(h, [&] {
    if (id < 0 || id >= (int)h->receivers.size() || fused_idx < 0 || fused_idx >= h->nsim)
      fail(LTS_ERR_ARG, "bad receiver id");
    const Receiver& r = h->receivers[id];
    const int64_t ns = (int64_t)r.t.size();
    if (n) *n = ns;
    const int64_t m = std::min<int64_t>(ns, cap);
    if (m <= 0) return;
    ck(cudaSetDevice(h->device), "cudaSetDevice");
    ck(cudaDeviceSynchronize(), "synchronize");
    // the receiver's samples occupy increasing slots; copy the span they cover
    const int64_t lo = r.slot[0], hi = r.slot[m - 1] + 1, F = h->nsim;
    std::vector<float> buf((hi - lo) * 9 * F);
    ck(cudaMemcpy(buf.data(), h->d_seis + lo * 9 * F, buf.size() * sizeof(float), cudaMemcpyDeviceToHost),
       "download seismogram");
    check_device_error(h);
    h->d2h_bytes += (int64_t)(buf.size() * sizeof(float));
    for (int64_t i = 0; i < m; ++i) {
      if (t_out) t_out[i] = r.t[i];
      if (v_out)
        for (int q = 0; q < 9; ++q) v_out[i * 9 + q] = buf[((r.slot[i] - lo) * F + fused_idx) * 9 + q];
    }
  });
}

int lts_energy(lts_t* h, double* e) {
  return run(h, [&] {
    if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
    if (!e) fail(LTS_ERR_ARG, "null output");
    ck(cudaSetDevice(h->device), "cudaSetDevice");
    const int nb = h->n_partial;
    h->L.energy(h->dst.Q, h->dst.qs, h->nsim, h->L.FG, h->d_emat, (int)h->mesh.K, h->d_partial, nb, 0);
    ck(cudaGetLastError(), "energy kernel");
    std::vector<double> part(nb);
    ck(cudaMemcpy(part.data(), h->d_partial, nb * sizeof(double), cudaMemcpyDeviceToHost), "download energy");
    check_device_error(h);
    double s = 0.0;
    for (double v : part) s += v;
    *e = s;
    if (!std::isfinite(s)) fail(LTS_ERR_NONFINITE, "non-finite energy: the state holds NaN or Inf");
  });
}

int lts_checkpoint_save(lts_t* h, const char* path) {
  return run(h, [&] {
    if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
    const int64_t period = int64_t(1) << (h->nc - 1);
    if (h->s_now % period != 0) fail(LTS_ERR_STATE, "not at a macro-step boundary");
    if (!path) fail(LTS_ERR_ARG, "null path");
    ck(cudaSetDevice(h->device), "cudaSetDevice");
    ck(cudaDeviceSynchronize(), "synchronize");
    check_device_error(h);
    const int64_t K = h->mesh.K, qs = h->dst.qs;
    std::vector<float> q((size_t)K * qs);
    ck(cudaMemcpy(q.data(), h->dst.Q, q.size() * sizeof(float), cudaMemcpyDeviceToHost), "download Q");
    std::vector<float> seis((size_t)h->seis_used * 9 * h->nsim);
    if (!seis.empty())
      ck(cudaMemcpy(seis.data(), h->d_seis, seis.size() * sizeof(float), cudaMemcpyDeviceToHost), "download samples");
    FILE* f = std::fopen(path, "wb");
    if (!f) fail(LTS_ERR_ARG, std::string("cannot write ") + path);
    bool ok = true;
    auto put = [&](const void* p, size_t bytes) { ok = ok && std::fwrite(p, 1, bytes, f) == bytes; };
    const char magic[8] = {'L', 'T', 'S', 'C', 'K', 'P', 'T', '1'};
    const int64_t hdr[9] = {h->order, h->nmech, h->nsim, K, h->nc, qs, (int64_t)h->receivers.size(),
                            (int64_t)h->sources.size(), h->s_now};
    put(magic, 8);
    put(hdr, sizeof(hdr));
    put(&h->delta, sizeof(double));
    put(q.data(), q.size() * sizeof(float));
    for (const Receiver& r : h->receivers) {
      const int64_t n = (int64_t)r.t.size();
      put(&n, sizeof(n));
      put(r.t.data(), n * sizeof(double));
      for (int64_t i = 0; i < n; ++i) put(&seis[(size_t)r.slot[i] * 9 * h->nsim], 9 * h->nsim * sizeof(float));
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) fail(LTS_ERR_ARG, std::string("write failed: ") + path);
  });
}

int lts_checkpoint_load(lts_t* h, const char* path) {
  return run(h, [&] {
    if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
    if (!path) fail(LTS_ERR_ARG, "null path");
    FILE* f = std::fopen(path, "rb");
    if (!f) fail(LTS_ERR_ARG, std::string("cannot read ") + path);
    struct Close {
      FILE* f;
      ~Close() { std::fclose(f); }
    } close_f{f};
    auto get = [&](void* p, size_t bytes) {
      if (std::fread(p, 1, bytes, f) != bytes) fail(LTS_ERR_ARG, "truncated checkpoint");
    };
    char magic[8];
    get(magic, 8);
    if (std::memcmp(magic, "LTSCKPT1", 8) != 0) fail(LTS_ERR_ARG, "not a checkpoint file");
    int64_t hdr[9];
    get(hdr, sizeof(hdr));
    const int64_t K = h->mesh.K, qs = h->dst.qs;
    const int64_t want[8] = {h->order, h->nmech, h->nsim, K, h->nc, qs, (int64_t)h->receivers.size(),
                             (int64_t)h->sources.size()};
    for (int i = 0; i < 8; ++i)
      if (hdr[i] != want[i]) fail(LTS_ERR_ARG, "checkpoint written for a different set-up");
    double delta = 0.0;
    get(&delta, sizeof(double));
    if (delta != h->delta) fail(LTS_ERR_ARG, "checkpoint written with a different time step");
    std::vector<float> q((size_t)K * qs);
    get(q.data(), q.size() * sizeof(float));
    std::vector<std::vector<double>> ts(h->receivers.size());
    std::vector<float> seis;
    for (size_t r = 0; r < h->receivers.size(); ++r) {
      int64_t n = 0;
      get(&n, sizeof(n));
      if (n < 0 || n > (int64_t(1) << 40)) fail(LTS_ERR_ARG, "corrupt checkpoint");
      ts[r].resize(n);
      get(ts[r].data(), n * sizeof(double));
      const size_t off = seis.size();
      seis.resize(off + (size_t)n * 9 * h->nsim);
      get(seis.data() + off, (size_t)n * 9 * h->nsim * sizeof(float));
    }
    ck(cudaSetDevice(h->device), "cudaSetDevice");
    ck(cudaDeviceSynchronize(), "synchronize");
    ck(cudaMemcpy(h->dst.Q, q.data(), q.size() * sizeof(float), cudaMemcpyHostToDevice), "upload Q");
    const size_t nsamp = seis.size() / (9 * h->nsim);
    ensure_capacity(reinterpret_cast<void**>(&h->d_seis), &h->seis_cap, nsamp * 9 * h->nsim, sizeof(float));
    if (!seis.empty())
      ck(cudaMemcpy(h->d_seis, seis.data(), seis.size() * sizeof(float), cudaMemcpyHostToDevice), "upload samples");
    int64_t slot = 0;
    for (size_t r = 0; r < h->receivers.size(); ++r) {
      h->receivers[r].t = ts[r];
      h->receivers[r].slot.resize(ts[r].size());
      for (size_t i = 0; i < ts[r].size(); ++i) h->receivers[r].slot[i] = slot++;
    }
    h->seis_used = nsamp;
    h->s_now = hdr[8];
  });
}

int lts_info(lts_t* h, int* n_clusters_out, int64_t* cluster_elems, int64_t* updates_per_macro, double* dt_min,
             double* lambda, double* finest_dt, double* time_now, int64_t* launches) {
  return run(h, [&] {
    if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
    if (n_clusters_out) *n_clusters_out = h->nc;
    for (int l = 0; l < h->nc; ++l) {
      const int64_t ne = h->cbeg[l + 1] - h->cbeg[l];
      if (cluster_elems) cluster_elems[l] = ne;
      if (updates_per_macro) updates_per_macro[l] = ne * (int64_t(1) << (h->nc - 1 - l));
    }
    if (dt_min) *dt_min = h->dt_min;
    if (lambda) *lambda = h->lambda;
    if (finest_dt) *finest_dt = h->delta;
    if (time_now) *time_now = h->s_now * h->delta;
    if (launches) *launches = h->launches;
  });
}

int lts_set_profiling(lts_t* h, int enable) {
  return run(h, [&] {
    h->profiling = enable != 0;
    h->ev_used = 0;
    h->ev_kind.clear();
    h->ev_elems.clear();
  });
}

int lts_kernel_stats(lts_t* h, double* ms_out, int64_t* launches_out, int64_t* elems_out) {
  return run(h, [&] {
    double ms[2] = {0, 0};
    int64_t nl[2] = {0, 0}, ne[2] = {0, 0};
    if (h->ev_used > 0) ck(cudaEventSynchronize(h->ev_pool[h->ev_used - 1]), "event sync");
    for (size_t i = 0; i < h->ev_kind.size(); ++i) {
      float t = 0.f;
      ck(cudaEventElapsedTime(&t, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]), "cudaEventElapsedTime");
      ms[h->ev_kind[i]] += t;
      nl[h->ev_kind[i]] += 1;
      ne[h->ev_kind[i]] += h->ev_elems[i];
    }
    for (int i = 0; i < 2; ++i) {
      if (ms_out) ms_out[i] = ms[i];
      if (launches_out) launches_out[i] = nl[i];
      if (elems_out) elems_out[i] = ne[i];
    }
    h->ev_used = 0;
    h->ev_kind.clear();
    h->ev_elems.clear();
  });
}

int lts_launch_config(lts_t* h, int* ctas_per_sm, int* threads) {
  return run(h, [&] {
    const Launchers& X = h->L;
    const bool tc = X.predict_tc != nullptr;
    // the predict and neighbour kernels of the handle's engine (sparse: with its tile variant)
    const bool sp = h->contraction == LTS_CONTRACT_SPARSE && X.predict_sp;
    const bool nsp = sp && X.neighbour_sp[0] && h->n_parts <= 1;
    const int tv = h->tile & 1;
    if (ctas_per_sm) {
      ctas_per_sm[0] = sp ? X.blocks_predict_sp : X.blocks_predict;
      ctas_per_sm[1] = nsp ? X.blocks_neighbour_sp[tv] : X.blocks_neighbour;
      ctas_per_sm[2] = tc ? X.blocks_predict_tc : 0;
    }
    if (threads) {
      threads[0] = sp ? X.NT_SP : X.NT;
      threads[1] = nsp ? X.NTN_SP[tv] : X.NTN;
      threads[2] = tc ? X.NT : 0;
    }
  });
}

int lts_autotune(lts_t* h, int allow_tf32, void* cuda_stream, int* chosen, double* best_ms, double* table, int cap,
                 int* n_out) {
  return run(h, [&] {
    if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
    if (cap < 0 || (cap > 0 && !table)) fail(LTS_ERR_ARG, "bad table arguments");
    ck(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const Launchers& X = h->L;
    const int64_t K = h->mesh.K;
    const size_t qbytes = sizeof(float) * K * h->dst.qs, bbytes = sizeof(float) * K * h->dst.bs;
    void* snap = nullptr;
    if (cudaMalloc(&snap, qbytes + 3 * bbytes) != cudaSuccess) {
      cudaGetLastError();
      fail(LTS_ERR_OOM, "no device memory for the autotune snapshot");
    }
    struct Free {
      void* p;
      ~Free() { cudaFree(p); }
    } free_snap{snap};
    char* sp = static_cast<char*>(snap);
    float* dev[4] = {h->dst.Q, h->dst.B1, h->dst.B2, h->dst.B3};
    const size_t sz[4] = {qbytes, bbytes, bbytes, bbytes};
    auto copy_state = [&](bool save) {
      size_t off = 0;
      for (int i = 0; i < 4; ++i) {
        ck(cudaMemcpyAsync(save ? static_cast<void*>(sp + off) : static_cast<void*>(dev[i]),
                           save ? static_cast<const void*>(dev[i]) : static_cast<const void*>(sp + off), sz[i],
                           cudaMemcpyDeviceToDevice, stream),
           "autotune state copy");
        off += sz[i];
      }
    };
    // host-side state that a trial step changes
    const int64_t s0 = h->s_now, l0 = h->launches, hb0 = h->h2d_bytes;
    const size_t seis0 = h->seis_used;
    std::vector<size_t> nrec(h->receivers.size());
    for (size_t i = 0; i < nrec.size(); ++i) nrec[i] = h->receivers[i].t.size();
    auto restore_host = [&] {
      h->s_now = s0;
      h->launches = l0;
      h->h2d_bytes = hb0;
      h->seis_used = seis0;
      for (size_t i = 0; i < nrec.size(); ++i) {
        h->receivers[i].t.resize(nrec[i]);
        h->receivers[i].slot.resize(nrec[i]);
      }
    };
    const bool prof = h->profiling;
    h->profiling = false;
    // candidates: engine x predict CTAs/SM x neighbour CTAs/SM (the occupancy maximum and
    // one fewer)
    std::vector<std::array<int, 4>> cand;
    std::vector<int> engines{LTS_CONTRACT_FP32};
    if (X.predict_sp) engines.push_back(LTS_CONTRACT_SPARSE);
    if (X.predict_tc) engines.push_back(LTS_CONTRACT_TF32X3);
    if (X.predict_tc && allow_tf32) engines.push_back(LTS_CONTRACT_TF32);
    for (int eng : engines) {
      const int mp = std::max(1, eng == LTS_CONTRACT_FP32     ? X.blocks_predict
                                 : eng == LTS_CONTRACT_SPARSE ? X.blocks_predict_sp
                                                              : X.blocks_predict_tc);
      const bool nsp = eng == LTS_CONTRACT_SPARSE && X.neighbour_sp[0] && h->n_parts <= 1;
      for (int tv = 0; tv < (nsp ? 2 : 1); ++tv) {
        const int mn = std::max(1, nsp ? X.blocks_neighbour_sp[tv] : X.blocks_neighbour);
        for (int cp = mp; cp >= std::max(1, mp - 1); --cp)
          for (int cn = mn; cn >= std::max(1, mn - 1); --cn) cand.push_back({eng, cp, cn, tv});
      }
    }
    cudaEvent_t ev[2];
    ck(cudaEventCreate(&ev[0]), "cudaEventCreate");
    ck(cudaEventCreate(&ev[1]), "cudaEventCreate");
    struct Ev {
      cudaEvent_t* e;
      ~Ev() {
        cudaEventDestroy(e[0]);
        cudaEventDestroy(e[1]);
      }
    } free_ev{ev};
    copy_state(true);
    const int64_t period = int64_t(1) << (h->nc - 1);
    double best = 1e300;
    int bi = 0;
    // trial -1 warms caches and clocks with the first candidate and is not counted
    for (int i = -1; i < (int)cand.size(); ++i) {
      const auto& c = cand[std::max(i, 0)];
      h->contraction = c[0];
      h->ctas_predict = c[1];
      h->ctas_neighbour = c[2];
      h->tile = c[3];
      ck(cudaEventRecord(ev[0], stream), "event record");
      advance_steps(h, period, stream);
      ck(cudaEventRecord(ev[1], stream), "event record");
      ck(cudaEventSynchronize(ev[1]), "event sync");
      float ms = 0.f;
      ck(cudaEventElapsedTime(&ms, ev[0], ev[1]), "event time");
      check_device_error(h);
      copy_state(false);
      restore_host();
      if (i < 0) continue;
      if (i < cap) {
        table[5 * i + 0] = c[0];
        table[5 * i + 1] = c[1];
        table[5 * i + 2] = c[2];
        table[5 * i + 3] = c[3];
        table[5 * i + 4] = ms;
      }
      if (ms < best) {
        best = ms;
        bi = i;
      }
    }
    ck(cudaStreamSynchronize(stream), "synchronize");
    h->profiling = prof;
    h->contraction = cand[bi][0];
    h->ctas_predict = cand[bi][1];
    h->ctas_neighbour = cand[bi][2];
    h->tile = cand[bi][3];
    if (chosen)
      for (int i = 0; i < 4; ++i) chosen[i] = cand[bi][i];
    if (best_ms) *best_ms = best;
    if (n_out) *n_out = (int)cand.size();
  });
}

int lts_partition(lts_t* h, int n_parts, int32_t* part_out, double* stats_out) {
  return run(h, [&] {
    require_material(h);
    if ((int64_t)h->cluster.size() != h->mesh.K) fail(LTS_ERR_STATE, "clusters not set up");
    if (n_parts < 1 || n_parts > h->mesh.K) fail(LTS_ERR_ARG, "bad part count");
    std::vector<int32_t> part;
    lts::PartitionStats st;
    lts::partition_elements(h->mesh, h->cluster, h->nc, n_parts, part, &st);
    if (part_out) std::copy(part.begin(), part.end(), part_out);
    if (stats_out) {
      const double v[6] = {st.max_load, st.min_load, st.total_weight, st.cut_faces, st.msgs_per_macro,
                           st.buffer_msgs_per_macro};
      std::copy(v, v + 6, stats_out);
    }
  });
}

int lts_cut_faces(lts_t* h, const int32_t* part, int64_t cap, int64_t* faces, int64_t* n) {
  return run(h, [&] {
    require_material(h);
    if ((int64_t)h->cluster.size() != h->mesh.K) fail(LTS_ERR_STATE, "clusters not set up");
    if (!part || cap < 0 || (cap > 0 && !faces)) fail(LTS_ERR_ARG, "bad arguments");
    std::vector<int32_t> p(part, part + h->mesh.K);
    for (int32_t x : p)
      if (x < 0) fail(LTS_ERR_ARG, "negative part index");
    std::vector<lts::CutFace> cf;
    lts::cut_faces(h->mesh, p, h->cluster, cf);
    if (n) *n = (int64_t)cf.size();
    for (int64_t c = 0; c < std::min<int64_t>(cap, (int64_t)cf.size()); ++c) {
      const lts::CutFace& x = cf[c];
      const int64_t v[8] = {x.recv_elem, x.recv_face, x.send_elem, x.send_face, x.orient, x.recv_part, x.send_part,
                            x.recv_cluster};
      std::copy(v, v + 8, faces + 8 * c);
    }
  });
}

int lts_set_partition(lts_t* h, int n_parts, const int32_t* part) {
  return run(h, [&] {
    require_material(h);
    if (n_parts > 1) {
      if (!part) fail(LTS_ERR_ARG, "null part array");
      for (int64_t k = 0; k < h->mesh.K; ++k)
        if (part[k] < 0 || part[k] >= n_parts) fail(LTS_ERR_ARG, "part index out of range");
      h->part.assign(part, part + h->mesh.K);
      h->n_parts = n_parts;
    } else {
      h->part.clear();
      h->n_parts = 1;
    }
    if (h->device >= 0 && (int64_t)h->cluster.size() == h->mesh.K) {
      ck(cudaSetDevice(h->device), "cudaSetDevice");
      setup_device(h);
    }
  });
}

int lts_exchange_bytes(lts_t* h, int64_t* bytes) {
  return run(h, [&] {
    if (!bytes) fail(LTS_ERR_ARG, "null output");
    *bytes = h->msg_bytes;
  });
}

int lts_set_finest_dt(lts_t* h, double dt) {
  return run(h, [&] {
    if ((int64_t)h->cluster.size() != h->mesh.K) fail(LTS_ERR_STATE, "clusters not set up");
    if (!(dt > 0.0)) fail(LTS_ERR_ARG, "time step must be positive");
    h->delta = dt;
    release_graphs(h);
  });
}

int lts_misfit_gradient(lts_t* h, int64_t n_steps, int64_t every, const double* data, double* misfit, double* grad,
                        double* synth_out, double* dq0, void* cuda_stream) {
  return run(h, [&] {
    if (!h->ready) fail(LTS_ERR_STATE, "clusters not set up");
    const Launchers& X = h->L;
    // a partitioned run on one GPU is bitwise the unpartitioned one; its reverse sweep reads
    // the owners' buffer snapshots directly (a multi-GPU build would send the transposed face
    // messages back over the cut)
    if (h->nmech != 0 || !X.adj_pred) fail(LTS_ERR_ARG, "the adjoint covers the elastic equations");
    const int64_t period = int64_t(1) << (h->nc - 1);
    if (h->nc > 1 && n_steps % period != 0) fail(LTS_ERR_ARG, "n_steps must be a multiple of the macro step");
    const int nrec = (int)h->receivers.size();
    if (nrec < 1 || n_steps < 1 || every < 1 || !data) fail(LTS_ERR_ARG, "bad adjoint arguments");
    ck(cudaSetDevice(h->device), "cudaSetDevice");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const int64_t K = h->mesh.K;
    const int B = X.B;
    // ---- face links (internal order)
    std::vector<int> fwd(8 * K, -1), back(8 * K, 0);
    for (int64_t k = 0; k < K; ++k) {
      const int64_t nk = h->iperm[k];
      for (int i = 0; i < 4; ++i) {
        const int64_t nb = h->mesh.nbr[4 * k + i];
        if (nb < 0) continue;
        const int ip = h->mesh.nbr_face[4 * k + i];
        fwd[8 * nk + 2 * i] = (int)h->iperm[nb];
        fwd[8 * nk + 2 * i + 1] = ip * 3 + h->mesh.nbr_orient[4 * k + i];
        back[8 * nk + 2 * i] = ip;
        back[8 * nk + 2 * i + 1] = i * 3 + h->mesh.nbr_orient[4 * nb + ip];
      }
    }
    // per cluster level t, the buffer owners of a neighbour pass whose highest cluster is t
    // that have a receiver in clusters 0..t (internal order, ascending)
    std::vector<int> own;
    std::vector<int64_t> own_off(1, 0);
    for (int t = 0; t < h->nc; ++t) {
      const int64_t nown = h->cbeg[std::min(t + 2, h->nc)], nact = h->cbeg[t + 1];
      for (int64_t kn = 0; kn < nown; ++kn)
        for (int i = 0; i < 4; ++i) {
          const int k = fwd[8 * kn + 2 * i];
          if (k >= 0 && k < nact) {
            own.push_back((int)kn);
            break;
          }
        }
      own_off.push_back((int64_t)own.size());
    }
    std::vector<int> relem(nrec);
    std::vector<float> rphi((size_t)nrec * B);
    for (int r = 0; r < nrec; ++r) {
      relem[r] = (int)h->iperm[h->receivers[r].elem];
      for (int b = 0; b < B; ++b) rphi[(size_t)r * B + b] = (float)h->receivers[r].phi[b];
    }
    // ---- device buffers; the explicit operators (reverse sweep only) are built on the device
    DevBuf d_amat, d_fwd, d_back, d_relem, d_rphi, d_own;
    GeoBufs geo_bufs;
    GradGeom geo{};
    if (grad || dq0) {
      geo = upload_geometry(h, geo_bufs, stream);
      d_amat.alloc(sizeof(float) * K * ltsdev::AM_SIZE);
      const long long nt = 5 * K;
      k_build_amat<<<(unsigned)((nt + 127) / 128), 128, 0, stream>>>(geo, d_amat.get<float>());
      ck(cudaGetLastError(), "operator build");
    }
    d_fwd.alloc(sizeof(int) * fwd.size());
    d_back.alloc(sizeof(int) * back.size());
    d_relem.alloc(sizeof(int) * nrec);
    d_rphi.alloc(sizeof(float) * rphi.size());
    auto up = [&](void* dst, const void* src, size_t bytes) {
      ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream), "adjoint upload");
    };
    up(d_fwd.p, fwd.data(), sizeof(int) * fwd.size());
    up(d_back.p, back.data(), sizeof(int) * back.size());
    d_own.alloc(sizeof(int) * own.size());
    up(d_own.p, own.data(), sizeof(int) * own.size());
    up(d_relem.p, relem.data(), sizeof(int) * nrec);
    up(d_rphi.p, rphi.data(), sizeof(float) * rphi.size());
    AdjTables tabs;
    make_adj_tables(h, tabs);
    // the phase-level sweep for every cluster count (one cluster: a macro step is one step)
    adjoint_lts(h, n_steps / period, every, data, misfit, grad, synth_out, dq0, stream, d_amat, d_fwd, d_back,
                d_relem, d_rphi, nrec, tabs, geo, d_own, own_off);
  });
}

int lts_set_graphs(lts_t* h, int enable) {
  return run(h, [&] {
    h->use_graphs = enable != 0;
    if (!h->use_graphs) release_graphs(h);
  });
}

int lts_adjoint_source_gradient(lts_t* h, double* out) {
  return run(h, [&] {
    if (!out) fail(LTS_ERR_ARG, "out is NULL");
    if (h->adj_src_grad.size() != h->sources.size() * 6)
      fail(LTS_ERR_STATE, "no adjoint sweep with the current sources");
    std::copy(h->adj_src_grad.begin(), h->adj_src_grad.end(), out);
  });
}

int lts_measure_peaks(lts_t* h, void* cuda_stream, double* out) {
  return run(h, [&] {
    if (!out) fail(LTS_ERR_ARG, "out is NULL");
    const cudaError_t e = ltsdev::measure_peaks(static_cast<cudaStream_t>(cuda_stream), out);
    if (e == cudaErrorTimeout) fail(LTS_ERR_TIMEOUT, "tensor-core peak probe did not complete within its bound");
    if (e != cudaSuccess) fail(LTS_ERR_CUDA, std::string("peak probes: ") + cudaGetErrorString(e));
  });
}

int lts_set_adjoint_memory(lts_t* h, uint64_t bytes) {
  return run(h, [&] { h->adj_budget = bytes; });
}

int lts_set_wait_limit(lts_t* h, int64_t cycles, int suppress_commit) {
  return run(h, [&] {
    if (cycles <= 0) fail(LTS_ERR_ARG, "wait limit must be positive");
    h->wait_cycles = cycles;
    h->suppress_commit = suppress_commit != 0;
  });
}

int lts_set_tile(lts_t* h, int tile) {
  return run(h, [&] {
    if (tile != 0 && tile != 1) fail(LTS_ERR_ARG, "tile variant must be 0 or 1");
    h->tile = tile;
  });
}

int lts_set_contraction(lts_t* h, int mode) {
  return run(h, [&] {
    if (mode != LTS_CONTRACT_FP32 && mode != LTS_CONTRACT_TF32X3 && mode != LTS_CONTRACT_TF32 &&
        mode != LTS_CONTRACT_SPARSE)
      fail(LTS_ERR_ARG, "unknown contraction mode");
    if ((mode == LTS_CONTRACT_TF32X3 || mode == LTS_CONTRACT_TF32) && !h->L.predict_tc)
      fail(LTS_ERR_ARG, "no tensor-core kernel for this shape");
    if (mode == LTS_CONTRACT_SPARSE && !h->L.predict_sp) fail(LTS_ERR_ARG, "no sparse kernel for this shape");
    h->contraction = mode;
  });
}

int lts_transfer_bytes(lts_t* h, int64_t* h2d, int64_t* d2h) {
  return run(h, [&] {
    if (h2d) *h2d = h->h2d_bytes;
    if (d2h) *d2h = h->d2h_bytes;
  });
}

int lts_reference_operators(int order, double* K, double* Ft, double* Fb) {
  if (order < 3 || order > 5) return LTS_ERR_ARG;
  try {
    lts::RefOps ops;
    ops.build(order);
    const int B = ops.B, F = ops.F;
    for (int c = 0; c < 3 && K; ++c) std::copy(ops.K[c].begin(), ops.K[c].end(), K + c * B * B);
    for (int f = 0; f < 4 && Ft; ++f) std::copy(ops.Ft[f].begin(), ops.Ft[f].end(), Ft + f * B * F);
    for (int jh = 0; jh < 12 && Fb; ++jh) std::copy(ops.Fb[jh].begin(), ops.Fb[jh].end(), Fb + jh * B * F);
  } catch (...) {
    return LTS_ERR_OOM;
  }
  return LTS_OK;
}

int lts_eval_basis(int order, int64_t n, const double* xi, double* out) {
  if (order < 3 || order > 5 || n < 0 || (n > 0 && (!xi || !out))) return LTS_ERR_ARG;
  try {
    lts::RefOps ops;
    ops.build(order);
    for (int64_t i = 0; i < n; ++i) ops.eval(xi + 3 * i, out + i * ops.B);
  } catch (...) {
    return LTS_ERR_OOM;
  }
  return LTS_OK;
}

int lts_quadrature_rule(int order, int64_t* n, double* xi, double* w) {
  if (order < 3 || order > 5 || !n) return LTS_ERR_ARG;
  try {
    lts::RefOps ops;
    ops.build(order);
    *n = (int64_t)ops.qp.size();
    for (size_t p = 0; p < ops.qp.size(); ++p) {
      if (xi)
        for (int d = 0; d < 3; ++d) xi[3 * p + d] = ops.qp[p][d];
      if (w) w[p] = ops.qw[p];
    }
  } catch (...) {
    return LTS_ERR_OOM;
  }
  return LTS_OK;
}

}  // extern "C"
