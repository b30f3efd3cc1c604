// Discrete adjoint of the clustered-LTS time loop, elastic equations, one or fused
// simulations (one cluster is the global-time-stepping case: a macro step is one step).
//
// One step of an element maps Q to Q' = Q + V(T) + S_L(T) + S_N(X of the face neighbours),
// with D_0 = Q, D_{d+1} = sum_c S_c D_d K_c^T (S_c the star matrices of the time kernel),
// T = sum_d c_d D_d, V = -sum_c S_c T K_c, S_L = sum_i A-_i (T F~_i) F^_i and
// S_N = sum_i A+_i (X_i F-_{j,h}) F^_i (A-_i, A+_i the 9 x 9 flux solvers of face i, X_i the
// neighbour's buffer that the cluster relation selects). For the adjoint lambda = dJ/dQ'
// the reverse passes below compute, per element,
//   mu = dJ/dT = -sum_c S_c^T lambda K_c^T + sum_i ((A-_i^T lambda) F^_i^T) F~_i^T
//        + the adjoints of the buffers the step wrote,
//   G_{O-1} = c_{O-1} mu, G_d = c_d mu + sum_c S_c^T G_{d+1} K_c,   dJ/dQ = lambda + G_0,
// the transposed neighbour fluxes into the adjoints of the buffers they read, and the
// per-element correlations that the material derivatives of S_c, A-_i, A+_i are contracted
// with once the loop is done:
//   W_c  += sum_{d<O-1} G_{d+1} (D_d K_c^T)^T - lambda (T K_c)^T,
//   W-_i += lambda (T F~_i F^_i)^T,   W+_i += lambda_k (X F-_{j,h} F^_i)^T.
// The matrices are explicit (FP32, built on the host from the same closed forms as the
// forward kernels' star and flux code); CUDA cores.
#pragma once
#include "kernels.cuh"

namespace ltsdev {

constexpr int AM_STAR = 0;       // S_c, c = 0..2: [out][in]
constexpr int AM_LOC = 243;      // A-_i, i = 0..3
constexpr int AM_NBR = 567;      // A+_i, i = 0..3
constexpr int AM_SIZE = 891;     // floats per element (also the size of the correlations W)

// Threads per element group: one warp up to order 4, two at order 5 (every phase needs at
// least one thread per mode column).
template <int O>
struct AdjNT {
  static constexpr int value = (nbasis(O) <= 32) ? 32 : 64;
};

// Transposed copies of the operator tables, so that every loop over a table reads it with
// consecutive threads on consecutive entries:
//   KT[c][j][i] = K[c][i][j],  FtT[i][f][b] = F~_i[b][f],  FhT[i][b][f] = F^_i[f][b],
//   FbT[jh][f][b] = F-_{jh}[b][f].
// v[r] = sum_{j < N} src[r * LD + j] * tab[j * ts + t] for the 9 rows r: each table entry is
// loaded once and the rows accumulate in registers.
template <int N, int LD>
__device__ __forceinline__ void rows9(const float* src, const float* __restrict__ tab, int ts, int t, float v[9]) {
#pragma unroll
  for (int r = 0; r < 9; ++r) v[r] = 0.f;
#pragma unroll 4
  for (int j = 0; j < N; ++j) {
    const float w = __ldg(tab + j * ts + t);
#pragma unroll
    for (int r = 0; r < 9; ++r) v[r] = fmaf(src[r * LD + j], w, v[r]);
  }
}

// Velocity at the receivers from Q^n: out[f][r][q] = sum_b Q_f[elem_r][6+q][b] phi_r[b] for
// the nsim simulations of an (elastic) state in groups of G (simulation f of element k, row
// q, mode b at k qs + (f / G) 9 B G + (q B + b) G + f % G; G = 1 for one simulation).
template <int O>
__global__ void k_adj_sample(const float* Q, long long qs, int nsim, int G, const int* elem, const float* phi,
                             int nrec, float* out) {
  constexpr int B = nbasis(O);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * nrec * nsim) return;
  const int f = t / (3 * nrec), r = (t / 3) % nrec, q = t % 3;
  const float* row = Q + (size_t)elem[r] * qs + (size_t)(f / G) * (9 * B * G) + f % G + (size_t)(6 + q) * B * G;
  float v = 0.f;
  for (int b = 0; b < B; ++b) v = fmaf(row[(size_t)b * G], phi[r * B + b], v);
  out[t] = v;
}

// The misfit's source: lambda_f[elem_r][6+q][b] += res[f][r][q] phi_r[b], lambda laid out
// [element][simulation][9][B] (receivers in order, so receivers that share an element add
// in a fixed order).
template <int O>
__global__ void k_adj_source(float* lam, int nsim, const int* elem, const float* phi, const float* res, int nrec) {
  constexpr int B = nbasis(O);
  const int b = threadIdx.x;
  if (b >= B) return;
  for (int f = 0; f < nsim; ++f)
    for (int r = 0; r < nrec; ++r)
      for (int q = 0; q < 3; ++q)
        lam[((size_t)elem[r] * nsim + f) * 9 * B + (6 + q) * B + b] += res[(f * nrec + r) * 3 + q] * phi[r * B + b];
}


// Moment-tensor gradient of the point sources one neighbour pass added:
// g[src][r] += c_s sum_b lambda_f[elem][r][b] phi_src[b], with c_s = -m0 (int s dt) / |det J|
// of item s and lambda the adjoint of Q after the pass ([element][simulation][9][B]). One
// thread per (item, stress component); a pass holds at most one item per source, so every
// entry has one writer.
template <int O>
__global__ void k_adj_src_grad(const float* lam, int nsim, const SrcItem* items, const double* c, int n,
                               const float* phi, double* g) {
  constexpr int B = nbasis(O);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 6 * n) return;
  const int s = t / 6, r = t % 6;
  const SrcItem it = items[s];
  const float* row = lam + ((size_t)it.elem * nsim + it.sim) * 9 * B + (size_t)r * B;
  float v = 0.f;
  for (int b = 0; b < B; ++b) v = fmaf(row[b], phi[it.phi_off + b], v);
  g[(size_t)(it.phi_off / B) * 6 + r] += c[s] * (double)v;
}

// ------------------------------------------------------------------ clustered LTS adjoint
// The LTS state is (Q, B1, B2, B3). Taken backwards, a neighbour pass of cluster l (step n)
// that added S_N(X_i) to Q_k sends ((A+_i^T lambda_Q_k) F^_i^T) F-_{j,h}^T to the adjoint
// of the buffer it read (B1 same cluster, B3 the neighbour finer, B2 / B1 - B2 the
// neighbour coarser in the first / second half); a predict pass that wrote B1 = T,
// B2 = T(dt/2) (finer neighbour), B3 = T or B3 += T (coarser neighbour, even / odd n) and
// added V(T) + S_L(T) to Q collects mu = V^T + S_L^T + lambda_B1 (+ lambda_B3) and
// mu_half = lambda_B2, resets the buffer adjoints it overwrote (lambda_B3 survives an
// accumulation) and runs the transposed time kernel with both Taylor weights.
struct AdjLtsArgs {
  const float* Qs;                    // Q before this predict pass (element stride qs)
  const float *B1s, *B2s, *B3s;       // buffers before this neighbour pass (element stride bufs)
  float* lq;                          // [K][9B] adjoint of Q
  float *lb1, *lb2, *lb3;             // [K][9B] adjoints of B1, B2, B3
  const float* amat;
  const int* fwd;
  const int* back;
  const int* meta;
  double* W;                          // [K][AM_SIZE], per-pass sums in FP32 added in FP64
  const float *KT, *FtT, *FhT, *FbT;  // transposed operator tables (see AdjTables)
  long long qs, bufs;
  int end;                            // active elements [0, end)
  // simulations of a fused run, in groups of G in the state and buffer snapshots (element k,
  // simulation f, row r, mode b at k qs + (f / G) 9 B G + (r B + b) G + f % G; one
  // simulation: nsim = G = 1); the adjoints are [element][simulation][9][B] and W sums the
  // simulations' correlations
  int nsim, G;
};

// y += S x (TR = false) or y += S^T x (TR = true) for an elastic star matrix S (row-major
// [out][in]). It couples the six stresses only to the three velocities and the velocities
// only to the stresses, so its other 45 entries are zero and skipped.
template <bool TR>
__device__ __forceinline__ void star_acc(const float* S, const float x[9], float y[9]) {
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int s = 6; s < 9; ++s) y[r] = fmaf(TR ? S[s * 9 + r] : S[r * 9 + s], x[s], y[r]);
#pragma unroll
  for (int r = 6; r < 9; ++r)
#pragma unroll
    for (int s = 0; s < 6; ++s) y[r] = fmaf(TR ? S[s * 9 + r] : S[r * 9 + s], x[s], y[r]);
}

// dst[q] = src[q] for q < N by a CTA of NT threads: every load is issued before the first
// store, so the element's copies are in flight together.
template <int N, int NT>
__device__ __forceinline__ void stage(float* dst, const float* __restrict__ src, int t) {
  constexpr int R = (N + NT - 1) / NT;
  float v[R];
#pragma unroll
  for (int j = 0; j < R; ++j)
    if (t + j * NT < N) v[j] = __ldg(src + t + j * NT);
#pragma unroll
  for (int j = 0; j < R; ++j)
    if (t + j * NT < N) dst[t + j * NT] = v[j];
}

// dst[q] = src[q G] for q < N (one simulation of a fused block), loads issued first.
template <int N, int NT>
__device__ __forceinline__ void stage_strided(float* dst, const float* __restrict__ src, int G, int t) {
  constexpr int R = (N + NT - 1) / NT;
  float v[R];
#pragma unroll
  for (int j = 0; j < R; ++j)
    if (t + j * NT < N) v[j] = __ldg(src + (size_t)(t + j * NT) * G);
#pragma unroll
  for (int j = 0; j < R; ++j)
    if (t + j * NT < N) dst[t + j * NT] = v[j];
}

// acc[i][j] += sum_{j' < n} X[(r0 + i) * LD + j'] * Y[(s0 + j) * LD + j'] for a 3 x 3 tile.
template <int LD>
__device__ __forceinline__ void tile33(const float* X, const float* Y, int r0, int s0, int n, float acc[3][3]) {
  for (int j = 0; j < n; ++j) {
    float x[3], y[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      x[i] = X[(r0 + i) * LD + j];
      y[i] = Y[(s0 + i) * LD + j];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int q = 0; q < 3; ++q) acc[i][q] = fmaf(x[i], y[q], acc[i][q]);
  }
}

// Shared-memory plan of k_adj_pred, a persistent kernel: the operator tables (K_c^T, K_c,
// F~_i, F^_i^T, F~_i^T) once per CTA, then one region per element group. A group is one warp
// (orders 3-4) or two (order 5) and takes the CTA's elements in turn; G groups fill the
// shared memory (at most 128 registers a thread, 15 named barriers for two-warp groups).
template <int O>
struct AdjPredCfg {
  static constexpr int B = nbasis(O), F = nface(O), NB9 = 9 * B, NT = AdjNT<O>::value;
  static constexpr int NSCR = (3 * NB9 > 108 * F) ? 3 * NB9 : 108 * F;
  static constexpr int ELEM = rup(AM_SIZE + (4 + O) * NB9 + NSCR, 4);   // sM, sL, sT, sG[2], sD[O], scratch
  static constexpr int TAB = rup(6 * B * B + 12 * B * F, 4);
  static constexpr int G_SMEM = (227 * 1024 / 4 - TAB) / ELEM;
  static constexpr int G_REG = 65536 / (128 * NT);
  static constexpr int G_BAR = (NT == 32) ? 32 : 15;
  static constexpr int G0 = G_SMEM < G_REG ? G_SMEM : G_REG;
  static constexpr int G = G0 < G_BAR ? G0 : G_BAR;
  static constexpr int THREADS = G * NT;
  static constexpr int SMEM_BYTES = 4 * (TAB + G * ELEM);
  static_assert(G >= 1 && SMEM_BYTES <= 227 * 1024, "k_adj_pred shared-memory plan");
};

// Barrier of one element group: the warp itself, or a named barrier over its two warps.
template <int NT>
__device__ __forceinline__ void gsync(int g) {
  if constexpr (NT == 32)
    __syncwarp();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "n"(NT) : "memory");
}

// rows9 with the table in shared memory.
template <int N, int LD>
__device__ __forceinline__ void rows9s(const float* src, const float* tab, int ts, int t, float v[9]) {
#pragma unroll
  for (int r = 0; r < 9; ++r) v[r] = 0.f;
#pragma unroll 4
  for (int j = 0; j < N; ++j) {
    const float w = tab[j * ts + t];
#pragma unroll
    for (int r = 0; r < 9; ++r) v[r] = fmaf(src[r * LD + j], w, v[r]);
  }
}

// Reverse of a predict pass over the active elements [0, end).
//
// Degree structure used throughout (exact): K_c[i][j] vanishes unless deg i < deg j, so
// D_d is a polynomial of degree O-1-d and lives on the first nbasis(O-d) modes; only those
// modes of its adjoint G_d matter. With Z_c = G_{d+1} K_c the reverse time kernel is
// G_d = c_d mu + c'_d mu_half + sum_c S_c^T Z_c and the star correlation of level d is
// Z_c D_d^T; with V_c = lambda K_c^T the volume term is mu = -sum_c S_c^T V_c and its
// correlation -V_c T^T.
template <int O>
__global__ void __launch_bounds__(AdjPredCfg<O>::THREADS, 1) k_adj_pred(DevOps ops, AdjLtsArgs a, PhaseArgs ph) {
  using C = AdjPredCfg<O>;
  constexpr int B = C::B, F = C::F, NB9 = C::NB9, NT = C::NT, NSCR = C::NSCR;
  extern __shared__ __align__(16) float smem[];
  float* tKT = smem;
  float* tK = tKT + 3 * B * B;
  float* tFt = tK + 3 * B * B;
  float* tFhT = tFt + 4 * B * F;
  float* tFtT = tFhT + 4 * B * F;
  for (int i = threadIdx.x; i < 3 * B * B; i += C::THREADS) {
    tKT[i] = a.KT[i];
    tK[i] = ops.K[i];
  }
  for (int i = threadIdx.x; i < 4 * B * F; i += C::THREADS) {
    tFt[i] = ops.Ft[i];
    tFhT[i] = a.FhT[i];
    tFtT[i] = a.FtT[i];
  }
  __syncthreads();
  const int g = threadIdx.x / NT, t = threadIdx.x % NT;
  float* sM = smem + C::TAB + g * C::ELEM;
  float* sL = sM + AM_SIZE;
  float* sT = sL + NB9;
  float* sG0 = sT + NB9;          // G ping-pong [2][9B]
  float* sDb = sG0 + 2 * NB9;     // D_0 .. D_{O-1} [O][9B]
  float* sScr = sDb + O * NB9;    // V_c, then the face products, then Z_c
  (void)NSCR;
  for (int k = blockIdx.x * C::G + g; k < a.end; k += gridDim.x * C::G) {
    const int meta = a.meta[k];
    const int cl = meta & 0xff;
    const bool finer = meta & FLAG_FINER, coarser = meta & FLAG_COARSER;
    const bool even = ph.parity[cl] == 0;
    stage<AM_SIZE, NT>(sM, a.amat + (size_t)k * AM_SIZE, t);
    double* Wk = a.W + (size_t)k * AM_SIZE;
    // star correlations summed over the simulations, one 3 x 3 tile (c, row block, column
    // block) per thread t < 27
    const int tc = t / 9, trb = (t / 3) % 3, tsb = t % 3;
    float wst[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int q = 0; q < 3; ++q) wst[i][q] = 0.f;
    for (int sim = 0; sim < a.nsim; ++sim) {
      const size_t kf = (size_t)k * a.nsim + sim;
      stage<NB9, NT>(sL, a.lq + kf * NB9, t);
      stage_strided<NB9, NT>(sDb, a.Qs + (size_t)k * a.qs + (size_t)(sim / a.G) * (NB9 * a.G) + sim % a.G, a.G, t);
      {
        // the adjoints of the buffers this pass wrote: lambda_B1 (+ lambda_B3) into sG0[0],
        // lambda_B2 into sG0[1]; reset here (lambda_B3 survives an accumulation)
        constexpr int R = (NB9 + NT - 1) / NT;
        const size_t o = kf * NB9;
        float v1[R], v2[R], v3[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int q = t + j * NT;
          v1[j] = v2[j] = v3[j] = 0.f;
          if (q < NB9) {
            v1[j] = a.lb1[o + q];
            if (coarser) v3[j] = a.lb3[o + q];
            if (finer) v2[j] = a.lb2[o + q];
          }
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int q = t + j * NT;
          if (q < NB9) {
            sG0[q] = v1[j] + v3[j];
            sG0[NB9 + q] = v2[j];
            a.lb1[o + q] = 0.f;
            if (coarser && even) a.lb3[o + q] = 0.f;
            if (finer) a.lb2[o + q] = 0.f;
          }
        }
      }
      gsync<NT>(g);
      const float* S = sM + AM_STAR;
      // ---- forward time kernel: D_{d+1} = sum_c S_c D_d K_c^T on the support of D_{d+1}
#pragma unroll
      for (int d = 0; d < O - 1; ++d) {
        const int nin = nbasis(O - d), nout = nbasis(O - 1 - d);
        if (t < B) {
          float Y[3][9];
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int s = 0; s < 9; ++s) Y[c][s] = 0.f;
          if (t < nout)
#pragma unroll 4
            for (int kk = 0; kk < nin; ++kk)
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                const float kc = tKT[(c * B + kk) * B + t];
#pragma unroll
                for (int s = 0; s < 9; ++s) Y[c][s] = fmaf(sDb[(d) * NB9 + s * B + kk], kc, Y[c][s]);
              }
          float v[9];
#pragma unroll
          for (int r = 0; r < 9; ++r) v[r] = 0.f;
#pragma unroll
          for (int c = 0; c < 3; ++c) star_acc<false>(S + c * 81, Y[c], v);
#pragma unroll
          for (int r = 0; r < 9; ++r) sDb[(d + 1) * NB9 + r * B + t] = v[r];
        }
        gsync<NT>(g);
      }
      float mu[9], muh[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) mu[r] = muh[r] = 0.f;
      float* sV = sScr;
      if (t < B) {
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          float v = 0.f;
          for (int d = 0; d < O; ++d) v = fmaf(ph.coef[cl][d], sDb[(d) * NB9 + r * B + t], v);
          sT[r * B + t] = v;
        }
        // V_c = lambda K_c^T and the volume term
        float V[3][9];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int s = 0; s < 9; ++s) V[c][s] = 0.f;
#pragma unroll 4
        for (int b = 0; b < B; ++b)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float kc = tKT[(c * B + b) * B + t];
#pragma unroll
            for (int s = 0; s < 9; ++s) V[c][s] = fmaf(sL[s * B + b], kc, V[c][s]);
          }
        float w[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) w[r] = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          star_acc<true>(S + c * 81, V[c], w);
#pragma unroll
          for (int s = 0; s < 9; ++s) sV[c * NB9 + s * B + t] = V[c][s];
        }
#pragma unroll
        for (int r = 0; r < 9; ++r) mu[r] = -w[r];
      }
      gsync<NT>(g);
      if (t < 27) {
        float tv[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int q = 0; q < 3; ++q) tv[i][q] = 0.f;
        tile33<B>(sV + tc * NB9, sT, 3 * trb, 3 * tsb, B, tv);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int q = 0; q < 3; ++q) wst[i][q] -= tv[i][q];
      }
      gsync<NT>(g);
      // local surface: LF_i = lambda F^_i^T, TF_i = T F~_i, U_i = A-_i^T LF_i, per (face, f)
      float* sLF = sScr;
      float* sTF = sScr + 36 * F;
      float* sU = sScr + 72 * F;
      for (int p = t; p < 4 * F; p += NT) {
        const int i = p / F, f = p % F;
        float lf[9], tf[9], u[9];
        rows9s<B, B>(sL, tFhT + i * B * F, F, f, lf);
        rows9s<B, B>(sT, tFt + i * B * F, F, f, tf);
        const float* Am = sM + AM_LOC + i * 81;
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          float v = 0.f;
#pragma unroll
          for (int s = 0; s < 9; ++s) v = fmaf(Am[s * 9 + r], lf[s], v);
          u[r] = v;
        }
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          sLF[(i * 9 + r) * F + f] = lf[r];
          sTF[(i * 9 + r) * F + f] = tf[r];
          sU[(i * 9 + r) * F + f] = u[r];
        }
      }
      gsync<NT>(g);
      if (t < B)
        for (int i = 0; i < 4; ++i)
#pragma unroll 5
          for (int f = 0; f < F; ++f) {
            const float w = tFtT[(i * F + f) * B + t];
#pragma unroll
            for (int r = 0; r < 9; ++r) mu[r] = fmaf(sU[(i * 9 + r) * F + f], w, mu[r]);
          }
      for (int p = t; p < 36; p += NT) {
        const int i = p / 9, rb = (p / 3) % 3, sb = p % 3;
        float acc[3][3];
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
          for (int q = 0; q < 3; ++q) acc[ii][q] = 0.f;
        tile33<F>(sLF + i * 9 * F, sTF + i * 9 * F, 3 * rb, 3 * sb, F, acc);
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
          for (int q = 0; q < 3; ++q) atomicAdd(Wk + AM_LOC + i * 81 + (3 * rb + ii) * 9 + 3 * sb + q, (double)acc[ii][q]);
      }
      // the buffers this pass wrote
      if (t < B) {
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          mu[r] += sG0[r * B + t];
          muh[r] = sG0[NB9 + r * B + t];
        }
#pragma unroll
        for (int r = 0; r < 9; ++r)
          sG0[((O - 1) & 1) * NB9 + r * B + t] = ph.coef[cl][O - 1] * mu[r] + ph.hcoef[cl][O - 1] * muh[r];
      }
      gsync<NT>(g);
      // ---- reverse time kernel
      float* sZ = sScr;
#pragma unroll
      for (int d = O - 2; d >= 0; --d) {
        const int nk = nbasis(O - 1 - d), nout = nbasis(O - d);
        const float* Gn = (sG0 + ((d + 1) & 1) * NB9);
        if (t < B) {
          float Z[3][9];
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < 9; ++r) Z[c][r] = 0.f;
          if (t < nout)
#pragma unroll 4
            for (int kk = 0; kk < nk; ++kk)
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                const float kc = tK[(c * B + kk) * B + t];
#pragma unroll
                for (int r = 0; r < 9; ++r) Z[c][r] = fmaf(Gn[r * B + kk], kc, Z[c][r]);
              }
          float g[9];
#pragma unroll
          for (int r = 0; r < 9; ++r) g[r] = ph.coef[cl][d] * mu[r] + ph.hcoef[cl][d] * muh[r];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            star_acc<true>(S + c * 81, Z[c], g);
#pragma unroll
            for (int r = 0; r < 9; ++r) sZ[c * NB9 + r * B + t] = Z[c][r];
          }
#pragma unroll
          for (int r = 0; r < 9; ++r) sG0[(d & 1) * NB9 + r * B + t] = g[r];
        }
        gsync<NT>(g);
        if (t < 27) tile33<B>(sZ + tc * NB9, (sDb + (d) * NB9), 3 * trb, 3 * tsb, nout, wst);
        gsync<NT>(g);
      }
      if (t < B)
#pragma unroll
        for (int r = 0; r < 9; ++r) a.lq[kf * NB9 + r * B + t] = sL[r * B + t] + sG0[(0) * NB9 + r * B + t];
      gsync<NT>(g);   // the group's region is refilled for the next simulation or element
    }
    if (t < 27)
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int q = 0; q < 3; ++q) atomicAdd(Wk + AM_STAR + tc * 81 + (3 * trb + i) * 9 + 3 * tsb + q, (double)wst[i][q]);
  }
}

// Reverse of a neighbour pass, one CTA per buffer owner (every element): for each face
// whose neighbour (the receiver) was active, the receiver's transposed flux goes to the
// adjoint of the buffer it read, and the receiver's correlation with that buffer is
// accumulated. Every (receiver, face) pair is visited by exactly one owner. The four faces
// are handled together: with LF = lambda_k F^_ip^T and XF = X F-_jh (9 x F each), the
// transposed flux is (A+^T LF) F-_jh^T and the correlation LF XF^T.
template <int O>
__global__ void __launch_bounds__(AdjNT<O>::value) k_adj_nbr(DevOps ops, AdjLtsArgs a, PhaseArgs ph) {
  constexpr int B = nbasis(O), F = nface(O), NB9 = 9 * B;
  __shared__ float sA[4][81];
  __shared__ float sLk[4][NB9], sX[4][NB9];
  __shared__ float sLF[4][9 * F], sXF[4][9 * F], sU[4][9 * F];
  __shared__ int sF[8], sBk[8];
  const int kn = blockIdx.x, t = threadIdx.x, nt = blockDim.x;
  if (t < 8) {
    sF[t] = a.fwd[kn * 8 + t];
    sBk[t] = a.back[kn * 8 + t];
  }
  __syncthreads();
  // buffer each active receiver read: 0 B1 (same cluster), 1 B3 (receiver coarser),
  // 2 B2 / 3 B1 - B2 (receiver finer, first / second half); -1 receiver not active
  const int lo = a.meta[kn] & 0xff;
  // modes packed 3 bits per face as mode + 1, so that a runtime face index needs no stack
  int modes = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int k = sF[2 * i];
    if (k < 0 || k >= a.end) continue;
    const int lr = a.meta[k] & 0xff;
    const int m = (lo == lr - 1) ? 1 : (lo == lr + 1) ? ((ph.parity[lr] == 0) ? 2 : 3) : 0;
    modes |= (m + 1) << (3 * i);
  }
  if (modes == 0) return;   // the same for every thread of the CTA
  auto mode = [modes](int i) { return ((modes >> (3 * i)) & 7) - 1; };
  constexpr int NT = AdjNT<O>::value, R = (NB9 + NT - 1) / NT;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (mode(i) >= 0) stage<81, NT>(sA[i], a.amat + (size_t)sF[2 * i] * AM_SIZE + AM_NBR + sBk[2 * i] * 81, t);
  for (int sim = 0; sim < a.nsim; ++sim) {
    // this simulation's block of the owner's buffers (stride G between modes)
    const size_t xo = (size_t)kn * a.bufs + (size_t)(sim / a.G) * (NB9 * a.G) + sim % a.G;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = mode(i);
      if (m < 0) continue;
      const int k = sF[2 * i];
      stage<NB9, NT>(sLk[i], a.lq + ((size_t)k * a.nsim + sim) * NB9, t);
      const float* b0 = (m == 1) ? a.B3s : (m == 2) ? a.B2s : a.B1s;
      float x[R], x2[R];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int q = t + j * NT;
        x[j] = x2[j] = 0.f;
        if (q < NB9) {
          x[j] = __ldg(b0 + xo + (size_t)q * a.G);
          if (m == 3) x2[j] = __ldg(a.B2s + xo + (size_t)q * a.G);
        }
      }
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (t + j * NT < NB9) sX[i][t + j * NT] = x[j] - x2[j];
    }
    __syncthreads();
    for (int p = t; p < 4 * F; p += nt) {
      const int i = p / F, f = p % F;
      if (mode(i) < 0) continue;
      const int ip = sBk[2 * i], jh = sBk[2 * i + 1];
      float lf[9], xf[9];
      rows9<B, B>(sLk[i], a.FhT + ip * B * F, F, f, lf);
      rows9<B, B>(sX[i], ops.Fb + jh * B * F, F, f, xf);
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float u = 0.f;
#pragma unroll
        for (int s = 0; s < 9; ++s) u = fmaf(sA[i][s * 9 + r], lf[s], u);
        sLF[i][r * F + f] = lf[r];
        sXF[i][r * F + f] = xf[r];
        sU[i][r * F + f] = u;
      }
    }
    __syncthreads();
    if (t < B) {
      // the faces' contributions summed per buffer, then one update of each adjoint touched
      float y1[9], y2[9], y3[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) y1[r] = y2[r] = y3[r] = 0.f;
      bool u1 = false, u2 = false, u3 = false;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int m = mode(i);
        if (m < 0) continue;
        float y[9];
        rows9<F, F>(sU[i], a.FbT + sBk[2 * i + 1] * F * B, B, t, y);
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          if (m == 1) {
            y3[r] += y[r];
          } else if (m == 2) {
            y2[r] += y[r];
          } else if (m == 3) {
            y1[r] += y[r];
            y2[r] -= y[r];
          } else {
            y1[r] += y[r];
          }
        }
        u1 |= (m == 0 || m == 3);
        u2 |= (m == 2 || m == 3);
        u3 |= (m == 1);
      }
      const size_t o = ((size_t)kn * a.nsim + sim) * NB9 + t;
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        if (u1) atomicAdd(a.lb1 + o + r * B, y1[r]);
        if (u2) atomicAdd(a.lb2 + o + r * B, y2[r]);
        if (u3) atomicAdd(a.lb3 + o + r * B, y3[r]);
      }
    }
    for (int p = t; p < 36; p += nt) {
      const int i = p / 9, rb = (p / 3) % 3, sb = p % 3;
      if (mode(i) < 0) continue;
      float acc[3][3];
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
#pragma unroll
        for (int q = 0; q < 3; ++q) acc[ii][q] = 0.f;
      tile33<F>(sLF[i], sXF[i], 3 * rb, 3 * sb, F, acc);
      double* Wk = a.W + (size_t)sF[2 * i] * AM_SIZE + AM_NBR + sBk[2 * i] * 81;
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
#pragma unroll
        for (int q = 0; q < 3; ++q) atomicAdd(Wk + (3 * rb + ii) * 9 + 3 * sb + q, (double)acc[ii][q]);
    }
    __syncthreads();   // the staged blocks are refilled for the next simulation
  }
}

}  // namespace ltsdev
