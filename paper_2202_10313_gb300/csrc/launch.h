// Launch wrappers of the kernels, one table per (order, mechanisms, fused group) instantiation.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "kernels_sp.cuh"
#include "kernels_tc.cuh"
#include "kernels_adj.cuh"
#include "kernels_adj_sp.cuh"

namespace ltsdev {

struct Launchers {
  int B, F, NQ, QS, BUFS, NE, NT, NEN, NTN;
  int FG;                                    // simulations per CTA in fused mode (1: single)
  size_t smem_predict, smem_neighbour;
  int blocks_predict, blocks_neighbour;      // resident CTAs per SM (filled by init)
  cudaError_t (*init)(Launchers*);
  void (*predict)(const DevOps&, const DevState&, const PhaseArgs&, int grid, cudaStream_t);
  void (*neighbour)(const DevOps&, const DevState&, const PhaseArgs&, int grid, cudaStream_t);
  // tensor-core predict + local kernel (nullptr where the shape has no tensor-core path);
  // passes 3: split-tf32 products, 1: tf32; err: device word set when a bounded wait gave up
  void (*predict_tc)(const DevOps&, const DevState&, const PhaseArgs&, int grid, int passes, int* err,
                     long long wait_cycles, int suppress_commit, cudaStream_t);
  size_t smem_predict_tc;
  int blocks_predict_tc;
  // predict + local kernel with generated sparse products (slots: elements, or (element,
  // simulation) pairs of fused simulations)
  void (*predict_sp)(const DevOps&, const DevState&, const PhaseArgs&, int grid, cudaStream_t);
  size_t smem_predict_sp;
  int blocks_predict_sp, NE_SP, NT_SP;
  // neighbour kernel of the same engine (face traces and orientation maps; no partition), in
  // two tile variants: 8 elements per CTA (two CTAs per SM) or 4 (four CTAs per SM)
  void (*neighbour_sp[2])(const DevOps&, const DevState&, const PhaseArgs&, int grid, cudaStream_t);
  size_t smem_neighbour_sp[2];
  int blocks_neighbour_sp[2], NEN_SP[2], NTN_SP[2];
  // fg: simulation group size of the layout (FG of the fused instantiation, 1 for one simulation)
  void (*receivers)(const DevOps&, const float* Q, long long qs, int nsim, int fg, const float* edata,
                    const float* phi, const RecvItem* items, float* out, const float* omega, int n, cudaStream_t);
  void (*sources)(float* Q, long long qs, int fg, const float* phi, const SrcItem* items, int n, cudaStream_t);
  // discrete adjoint of the elastic GTS loop (one simulation, no mechanisms; else nullptr)
  void (*adj_sample)(const float* Q, long long qs, int nsim, int G, const int* elem, const float* phi, int nrec,
                     float* out, cudaStream_t);
  void (*adj_source)(float* lam, int nsim, const int* elem, const float* phi, const float* res, int nrec,
                     cudaStream_t);
  void (*adj_src_grad)(const float* lam, int nsim, const SrcItem* items, const double* c, int n, const float* phi,
                       double* g, cudaStream_t);
  void (*adj_pred)(const DevOps&, const AdjLtsArgs&, const PhaseArgs&, int nelem, cudaStream_t);
  // the same with generated sparse products (one or fused simulations)
  void (*adj_pred_sp)(const AdjLtsArgs&, const PhaseArgs&, int nelem, cudaStream_t);
  void (*adj_nbr)(const DevOps&, const AdjLtsArgs&, const PhaseArgs&, int K, cudaStream_t);
  // face-local messages of a partitioned run (one simulation)
  void (*pack)(const DevOps&, const DevState&, const PhaseArgs&, const int* send_elem, const int* send_code,
               const int* recv_cluster, int n, float* msg, cudaStream_t);
  void (*energy)(const float* Q, long long qs, int nsim, int fg, const double* emat, int K, double* partial,
                 int nblocks, cudaStream_t);
};

template <int O, int M, int FG>
struct Impl {
  using C = Cfg<O, M, FG>;
  // Dynamic shared memory limit; max_carveout also asks for the largest shared-memory
  // carveout (the CUDA-core kernels keep the default: their gathers live on L1).
  template <typename K>
  static cudaError_t smem_attrs(K kernel, size_t bytes, bool max_carveout) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess || !max_carveout) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  }
  static cudaError_t init(Launchers* L) {
    cudaError_t e = smem_attrs(k_predict_local<O, M, FG>, L->smem_predict, false);
    if (e != cudaSuccess) return e;
    e = smem_attrs(k_neighbour<O, M, FG>, L->smem_neighbour, false);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L->blocks_predict, k_predict_local<O, M, FG>, C::NT,
                                                      L->smem_predict);
    if (e != cudaSuccess) return e;
    if constexpr (TcCfg<O, M, FG>::SUPPORTED) {
      e = smem_attrs(k_predict_tc<O, M, FG>, L->smem_predict_tc, true);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L->blocks_predict_tc, k_predict_tc<O, M, FG>, C::NT,
                                                        L->smem_predict_tc);
      if (e != cudaSuccess) return e;
      // the occupancy query answers one CTA for this kernel although registers and shared
      // memory admit two; the persistent grid is sized for two (CTAs are independent and
      // two fit the 512 tensor-memory columns)
      L->blocks_predict_tc = 2;
    }
    {
      constexpr bool FU = FG > 1;
      e = smem_attrs(k_predict_sp<O, M, FU>, L->smem_predict_sp, true);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L->blocks_predict_sp, k_predict_sp<O, M, FU>,
                                                        SpCfg<O, M, FU>::NT, L->smem_predict_sp);
      if (e != cudaSuccess) return e;
      e = smem_attrs(k_neighbour_sp<O, M, 8, FU>, L->smem_neighbour_sp[0], true);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L->blocks_neighbour_sp[0], k_neighbour_sp<O, M, 8, FU>,
                                                        SpnCfg<O, M, 8>::NT, L->smem_neighbour_sp[0]);
      if (e != cudaSuccess) return e;
      e = smem_attrs(k_neighbour_sp<O, M, 4, FU>, L->smem_neighbour_sp[1], true);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L->blocks_neighbour_sp[1], k_neighbour_sp<O, M, 4, FU>,
                                                        SpnCfg<O, M, 4>::NT, L->smem_neighbour_sp[1]);
      if (e != cudaSuccess) return e;
    }
    if constexpr (M == 0) {
      e = cudaFuncSetAttribute(k_adj_pred<O>, cudaFuncAttributeMaxDynamicSharedMemorySize, AdjPredCfg<O>::SMEM_BYTES);
      if (e != cudaSuccess) return e;
      e = smem_attrs(k_adj_pred_sp<O>, AdjSpCfg<O>::TOTAL * sizeof(float), true);
      if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L->blocks_neighbour, k_neighbour<O, M, FG>, C::NTN,
                                                         L->smem_neighbour);
  }
  static void predict(const DevOps& o, const DevState& s, const PhaseArgs& p, int grid, cudaStream_t st) {
    k_predict_local<O, M, FG><<<grid, C::NT, C::P_TOTAL * sizeof(float), st>>>(o, s, p);
  }
  static void neighbour(const DevOps& o, const DevState& s, const PhaseArgs& p, int grid, cudaStream_t st) {
    k_neighbour<O, M, FG><<<grid, C::NTN, C::N_TOTAL * sizeof(float), st>>>(o, s, p);
  }
  static void predict_sp(const DevOps& o, const DevState& s, const PhaseArgs& p, int grid, cudaStream_t st) {
    using S = SpCfg<O, M, (FG > 1)>;
    k_predict_sp<O, M, (FG > 1)><<<grid, S::NT, S::TOTAL * sizeof(float), st>>>(o, s, p);
  }
  template <int NE>
  static void neighbour_sp(const DevOps& o, const DevState& s, const PhaseArgs& p, int grid, cudaStream_t st) {
    k_neighbour_sp<O, M, NE, (FG > 1)>
        <<<grid, SpnCfg<O, M, NE>::NT, SpnCfg<O, M, NE>::TOTAL * sizeof(float), st>>>(o, s, p);
  }
  static void predict_tc(const DevOps& o, const DevState& s, const PhaseArgs& p, int grid, int passes, int* err,
                         long long wait_cycles, int suppress_commit, cudaStream_t st) {
    if constexpr (TcCfg<O, M, FG>::SUPPORTED)
      k_predict_tc<O, M, FG><<<grid, C::NT, TcCfg<O, M, FG>::SMEM_BYTES, st>>>(o, s, p, passes, err, wait_cycles,
                                                                               suppress_commit);
  }
  static void receivers(const DevOps& o, const float* Q, long long qs, int nsim, int fg, const float* ed,
                        const float* phi, const RecvItem* it, float* out, const float* om, int n, cudaStream_t st) {
    k_receivers<O, M><<<n, rup(C::B, 32), 0, st>>>(o, Q, qs, nsim, fg, ed, phi, it, out, om[0], om[1], om[2]);
  }
  static void sources(float* Q, long long qs, int fg, const float* phi, const SrcItem* it, int n, cudaStream_t st) {
    k_sources<O, M><<<1, 128, 0, st>>>(Q, qs, fg, phi, it, n);
  }
  static void pack(const DevOps& o, const DevState& s, const PhaseArgs& p, const int* se, const int* sc,
                   const int* rc, int n, float* msg, cudaStream_t st) {
    const int threads = 128, nt = n * s.nsim * C::F;   // one thread per (cut face, simulation, face mode)
    k_pack_faces<O, M><<<(nt + threads - 1) / threads, threads, 0, st>>>(o, s, p, se, sc, rc, n, FG, msg);
  }
  static void adj_sample(const float* Q, long long qs, int nsim, int G, const int* elem, const float* phi, int nrec,
                         float* out, cudaStream_t st) {
    k_adj_sample<O><<<(3 * nrec * nsim + 127) / 128, 128, 0, st>>>(Q, qs, nsim, G, elem, phi, nrec, out);
  }
  static void adj_source(float* lam, int nsim, const int* elem, const float* phi, const float* res, int nrec,
                         cudaStream_t st) {
    k_adj_source<O><<<1, 64, 0, st>>>(lam, nsim, elem, phi, res, nrec);
  }
  static void adj_src_grad(const float* lam, int nsim, const SrcItem* items, const double* c, int n,
                           const float* phi, double* g, cudaStream_t st) {
    if (n > 0) k_adj_src_grad<O><<<(6 * n + 127) / 128, 128, 0, st>>>(lam, nsim, items, c, n, phi, g);
  }
  // persistent: at most one CTA per SM, each CTA's element groups take elements in turn
  static void adj_pred(const DevOps& o, const AdjLtsArgs& a, const PhaseArgs& p, int n, cudaStream_t st) {
    using A = AdjPredCfg<O>;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int ctas = (n + A::G - 1) / A::G;
    const int grid = ctas < nsm ? ctas : nsm;
    if (grid > 0) k_adj_pred<O><<<grid, A::THREADS, A::SMEM_BYTES, st>>>(o, a, p);
  }
  // two CTAs per SM, each taking batches of NE elements in turn
  static void adj_pred_sp(const AdjLtsArgs& a, const PhaseArgs& p, int n, cudaStream_t st) {
    using A = AdjSpCfg<O>;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int nb = (n + A::NE - 1) / A::NE;
    const int grid = nb < 2 * nsm ? nb : 2 * nsm;
    if (grid > 0) k_adj_pred_sp<O><<<grid, A::NT, A::TOTAL * sizeof(float), st>>>(a, p);
  }
  static void adj_nbr(const DevOps& o, const AdjLtsArgs& a, const PhaseArgs& p, int K, cudaStream_t st) {
    if (K > 0) k_adj_nbr<O><<<K, AdjNT<O>::value, 0, st>>>(o, a, p);
  }
  static void energy(const float* Q, long long qs, int nsim, int fg, const double* emat, int K, double* partial,
                     int nblocks, cudaStream_t st) {
    k_energy<O, M><<<nblocks, 256, 0, st>>>(Q, qs, nsim, fg, emat, K, partial);
  }
  static Launchers make() {
    Launchers L{};
    L.FG = FG;
    L.B = C::B;
    L.F = C::F;
    L.NQ = C::NQ;
    L.QS = C::QS;
    L.BUFS = C::BUFS;
    L.NE = C::NE;
    L.NT = C::NT;
    L.NEN = C::NEN;
    L.NTN = C::NTN;
    L.smem_predict = C::P_TOTAL * sizeof(float);
    L.smem_neighbour = C::N_TOTAL * sizeof(float);
    L.init = &init;
    L.predict = &predict;
    if constexpr (TcCfg<O, M, FG>::SUPPORTED) {
      L.predict_tc = &predict_tc;
      L.smem_predict_tc = TcCfg<O, M, FG>::SMEM_BYTES;
    }
    {
      L.predict_sp = &predict_sp;
      L.smem_predict_sp = SpCfg<O, M, (FG > 1)>::TOTAL * sizeof(float);
      L.NE_SP = SpCfg<O, M, (FG > 1)>::NE;
      L.NT_SP = SpCfg<O, M, (FG > 1)>::NT;
      L.neighbour_sp[0] = &neighbour_sp<8>;
      L.neighbour_sp[1] = &neighbour_sp<4>;
      L.smem_neighbour_sp[0] = SpnCfg<O, M, 8>::TOTAL * sizeof(float);
      L.smem_neighbour_sp[1] = SpnCfg<O, M, 4>::TOTAL * sizeof(float);
      L.NEN_SP[0] = 8;
      L.NEN_SP[1] = 4;
      L.NTN_SP[0] = SpnCfg<O, M, 8>::NT;
      L.NTN_SP[1] = SpnCfg<O, M, 4>::NT;
    }
    L.neighbour = &neighbour;
    L.receivers = &receivers;
    L.sources = &sources;
    L.pack = &pack;
    // the adjoint covers the elastic equations (one or fused simulations)
    if constexpr (M == 0) {
      L.adj_sample = &adj_sample;
      L.adj_source = &adj_source;
      L.adj_src_grad = &adj_src_grad;
      L.adj_pred = &adj_pred;
      L.adj_pred_sp = &adj_pred_sp;
      L.adj_nbr = &adj_nbr;
    }
    L.energy = &energy;
    return L;
  }
};

// defined in kernels_o{3,4,5}.cu; fused selects the fused-simulation instantiation
Launchers launchers_o3(int m, bool fused);
Launchers launchers_o4(int m, bool fused);
Launchers launchers_o5(int m, bool fused);

}  // namespace ltsdev
