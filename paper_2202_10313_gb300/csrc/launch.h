// Launch wrappers of the kernels, one table per (order, mechanisms, fused group) instantiation.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace ltsdev {

struct Launchers {
  int B, F, NQ, QS, BUFS, NE, NT, NEN;
  int FG;                                    // simulations per CTA in fused mode (1: single)
  size_t smem_predict, smem_neighbour;
  int blocks_predict, blocks_neighbour;      // resident CTAs per SM (filled by init)
  cudaError_t (*init)(Launchers*);
  void (*predict)(const DevOps&, const DevState&, const PhaseArgs&, int grid, cudaStream_t);
  void (*neighbour)(const DevOps&, const DevState&, const PhaseArgs&, int grid, cudaStream_t);
  // fg: simulation group size of the layout (FG of the fused instantiation, 1 for one simulation)
  void (*receivers)(const DevOps&, const float* Q, long long qs, int nsim, int fg, const float* edata,
                    const float* phi, const RecvItem* items, float* out, const float* omega, int n, cudaStream_t);
  void (*sources)(float* Q, long long qs, int fg, const float* phi, const SrcItem* items, int n, cudaStream_t);
  void (*energy)(const float* Q, long long qs, int nsim, int fg, const double* emat, int K, double* partial,
                 int nblocks, cudaStream_t);
};

template <int O, int M, int FG>
struct Impl {
  using C = Cfg<O, M, FG>;
  static cudaError_t init(Launchers* L) {
    cudaError_t e = cudaFuncSetAttribute(k_predict_local<O, M, FG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L->smem_predict);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_neighbour<O, M, FG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)L->smem_neighbour);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L->blocks_predict, k_predict_local<O, M, FG>, C::NT,
                                                      L->smem_predict);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&L->blocks_neighbour, k_neighbour<O, M, FG>, C::NTN,
                                                         L->smem_neighbour);
  }
  static void predict(const DevOps& o, const DevState& s, const PhaseArgs& p, int grid, cudaStream_t st) {
    k_predict_local<O, M, FG><<<grid, C::NT, C::P_TOTAL * sizeof(float), st>>>(o, s, p);
  }
  static void neighbour(const DevOps& o, const DevState& s, const PhaseArgs& p, int grid, cudaStream_t st) {
    k_neighbour<O, M, FG><<<grid, C::NTN, C::N_TOTAL * sizeof(float), st>>>(o, s, p);
  }
  static void receivers(const DevOps& o, const float* Q, long long qs, int nsim, int fg, const float* ed,
                        const float* phi, const RecvItem* it, float* out, const float* om, int n, cudaStream_t st) {
    k_receivers<O, M><<<n, rup(C::B, 32), 0, st>>>(o, Q, qs, nsim, fg, ed, phi, it, out, om[0], om[1], om[2]);
  }
  static void sources(float* Q, long long qs, int fg, const float* phi, const SrcItem* it, int n, cudaStream_t st) {
    k_sources<O, M><<<1, 128, 0, st>>>(Q, qs, fg, phi, it, n);
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
    L.smem_predict = C::P_TOTAL * sizeof(float);
    L.smem_neighbour = C::N_TOTAL * sizeof(float);
    L.init = &init;
    L.predict = &predict;
    L.neighbour = &neighbour;
    L.receivers = &receivers;
    L.sources = &sources;
    L.energy = &energy;
    return L;
  }
};

// defined in kernels_o{3,4,5}.cu; fused selects the fused-simulation instantiation
Launchers launchers_o3(int m, bool fused);
Launchers launchers_o4(int m, bool fused);
Launchers launchers_o5(int m, bool fused);

}  // namespace ltsdev
