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
  const int* owners;                  // neighbour reverse: the pass's buffer owners with an active
                                      // receiver (one CTA each), or null: owner = CTA index
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

// acc[i][q] += sum_{j < n} X[(r0 + i) * LD + j] * Y[(s0 + q) * LD + j] for a 3 x 3 tile, four
// j at a time (LD and n multiples of 4, X and Y 16-byte aligned; entries j >= the true length
// are zero on one side at least).
template <int LD>
__device__ __forceinline__ void tile33v(const float* X, const float* Y, int r0, int s0, int n, float acc[3][3]) {
#pragma unroll 1
  for (int j = 0; j < n; j += 4) {
    float4 x[3], y[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      x[i] = *reinterpret_cast<const float4*>(X + (r0 + i) * LD + j);
      y[i] = *reinterpret_cast<const float4*>(Y + (s0 + i) * LD + j);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        acc[i][q] = fmaf(x[i].x, y[q].x, acc[i][q]);
        acc[i][q] = fmaf(x[i].y, y[q].y, acc[i][q]);
        acc[i][q] = fmaf(x[i].z, y[q].z, acc[i][q]);
        acc[i][q] = fmaf(x[i].w, y[q].w, acc[i][q]);
      }
  }
}

// The nine rows of a [9][LD] block, entries j .. j + 3 (16-byte aligned; the same address in
// every lane, so each load is one broadcast).
template <int LD>
__device__ __forceinline__ void load_cols4(const float* src, int j, float4 x[9]) {
#pragma unroll
  for (int r = 0; r < 9; ++r) x[r] = *reinterpret_cast<const float4*>(src + r * LD + j);
}
__device__ __forceinline__ float lane4(const float4& v, int u) { return u == 0 ? v.x : u == 1 ? v.y : u == 2 ? v.z : v.w; }

// v[r] = sum_{j < N} src[r * LD + j] * tab[j * ts + t] for the 9 rows r, the broadcast
// operand four entries at a time (N, LD multiples of 4; pad entries zero on one side).
template <int N, int LD>
__device__ __forceinline__ void rows9v(const float* src, const float* tab, int ts, int t, float v[9]) {
#pragma unroll
  for (int r = 0; r < 9; ++r) v[r] = 0.f;
#pragma unroll 1
  for (int j = 0; j < N; j += 4) {
    float4 x[9];
    load_cols4<LD>(src, j, x);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float w = tab[(j + u) * ts + t];
#pragma unroll
      for (int r = 0; r < 9; ++r) v[r] = fmaf(lane4(x[r], u), w, v[r]);
    }
  }
}

// Elastic star matrix S_c (row-major [out][in]) in compact form: it couples the six stresses
// only to the three velocities and back, so only the 6 x 3 block S[r][6 + s] (row-major, 18
// entries) and the 3 x 6 block S[6 + r][s] (18 entries) are kept, 36 floats per c.
__device__ __forceinline__ int star_compact_index(int x) {
  return x < 18 ? (x / 3) * 9 + 6 + x % 3 : (6 + (x - 18) / 6) * 9 + (x - 18) % 6;
}
// y += S x (TR = false) or y += S^T x (TR = true), S in compact form (16-byte aligned).
template <bool TR>
__device__ __forceinline__ void star_acc(const float* Sc, const float x[9], float y[9]) {
  float e[36];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float4 v = reinterpret_cast<const float4*>(Sc)[i];
    e[4 * i] = v.x;
    e[4 * i + 1] = v.y;
    e[4 * i + 2] = v.z;
    e[4 * i + 3] = v.w;
  }
  if (!TR) {
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int s = 0; s < 3; ++s) y[r] = fmaf(e[r * 3 + s], x[6 + s], y[r]);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int s = 0; s < 6; ++s) y[6 + r] = fmaf(e[18 + r * 6 + s], x[s], y[6 + r]);
  } else {
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
      for (int r = 0; r < 6; ++r) y[6 + s] = fmaf(e[r * 3 + s], x[r], y[6 + s]);
#pragma unroll
    for (int s = 0; s < 6; ++s)
#pragma unroll
      for (int r = 0; r < 3; ++r) y[s] = fmaf(e[18 + r * 6 + s], x[6 + r], y[s]);
  }
}

// Polynomial degree of volume mode j (modes are ordered by degree).
__device__ __forceinline__ int mode_degree(int j) {
  int p = 0;
  while (nbasis(p + 1) <= j) ++p;
  return p;
}

// Shared-memory plan of k_adj_pred, a persistent kernel: the operator tables (K_c^T, K_c,
// F~_i, F^_i^T, F~_i^T) once per CTA, then one region per element group. A group is one warp
// (orders 3-4) or two (order 5) and takes the CTA's elements in turn; G groups fill the
// shared memory (at most 128 registers a thread, 15 named barriers for two-warp groups).
// Mode rows are padded to BP = rup(B, 4) and face-mode rows to FP = rup(F, 4), the pad entries
// zero (table rows past B or F zero as well), so that every contraction reads its broadcast
// operand four entries at a time.
template <int O>
struct AdjPredCfg {
  static constexpr int B = nbasis(O), F = nface(O), NT = AdjNT<O>::value;
  static constexpr int BP = rup(B, 4), FP = rup(F, 4), NB9 = 9 * BP;
  static constexpr int NSTAR = 3 * 36, NALOC = 4 * 9 * 12;       // compact S_c; A-_i rows padded to 12
  static constexpr int NSCR = (3 * NB9 > 27 * 4 * FP) ? 3 * NB9 : 27 * 4 * FP;
  static constexpr int ELEM = NSTAR + NALOC + (4 + O) * NB9 + NSCR;   // sS, sA, sL, sT, sG[2], sD[O], scratch
  static constexpr int TAB = 6 * BP * B + 8 * BP * F + 4 * FP * B;
  static constexpr int G_SMEM = (227 * 1024 / 4 - TAB) / ELEM;
  static constexpr int G_REG = 65536 / (128 * NT);
  static constexpr int G_BAR = (NT == 32) ? 32 : 15;
  static constexpr int G0 = G_SMEM < G_REG ? G_SMEM : G_REG;
  static constexpr int G = G0 < G_BAR ? G0 : G_BAR;
  static constexpr int THREADS = G * NT;
  static constexpr int SMEM_BYTES = 4 * (TAB + G * ELEM);
  static_assert(G >= 1 && SMEM_BYTES <= 227 * 1024, "k_adj_pred shared-memory plan");
  static_assert(TAB % 4 == 0 && ELEM % 4 == 0 && NB9 % 4 == 0, "16-byte aligned regions");
};

// Barrier of one element group: the warp itself, or a named barrier over its two warps.
template <int NT>
__device__ __forceinline__ void gsync(int g) {
  if constexpr (NT == 32)
    __syncwarp();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "n"(NT) : "memory");
}

// dst[(q / B) BP + q % B] = src[q G] for q < 9 B: a [9][B] block (stride G between entries)
// into the padded [9][BP] layout, every load issued before the first store.
template <int B, int BP, int NT>
__device__ __forceinline__ void stage_pad(float* dst, const float* __restrict__ src, int G, int t) {
  constexpr int N = 9 * B, R = (N + NT - 1) / NT;
  float v[R];
#pragma unroll
  for (int j = 0; j < R; ++j)
    if (t + j * NT < N) v[j] = __ldg(src + (size_t)(t + j * NT) * G);
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int q = t + j * NT;
    if (q < N) dst[(q / B) * BP + q % B] = v[j];
  }
}

// Reverse of a predict pass over the active elements [0, end).
//
// Degree structure used throughout (exact): K_c[i][j] vanishes unless deg i < deg j, so
// D_d is a polynomial of degree O-1-d and lives on the first nbasis(O-d) modes; only those
// modes of its adjoint G_d matter. With Z_c = G_{d+1} K_c the reverse time kernel is
// G_d = c_d mu + c'_d mu_half + sum_c S_c^T Z_c and the star correlation of level d is
// Z_c D_d^T; with V_c = lambda K_c^T the volume term is mu = -sum_c S_c^T V_c and its
// correlation -V_c T^T. The contractions run over a multiple of four entries; the extra
// entries multiply structural zeros of K_c or zero pads, so the sums are those of the
// unpadded loops, term for term.
template <int O>
__global__ void __launch_bounds__(AdjPredCfg<O>::THREADS, 1) k_adj_pred(DevOps ops, AdjLtsArgs a, PhaseArgs ph) {
  using C = AdjPredCfg<O>;
  constexpr int B = C::B, F = C::F, BP = C::BP, FP = C::FP, NB9 = C::NB9, NT = C::NT;
  extern __shared__ __align__(16) float smem[];
  float* tKT = smem;                  // [3][BP][B]   K_c^T[j][i] at (c BP + j) B + i
  float* tK = tKT + 3 * BP * B;       // [3][BP][B]   K_c[j][i]
  float* tFt = tK + 3 * BP * B;       // [4][BP][F]   F~_i[b][f] at (i BP + b) F + f
  float* tFhT = tFt + 4 * BP * F;     // [4][BP][F]   F^_i[f][b] at (i BP + b) F + f
  float* tFtT = tFhT + 4 * BP * F;    // [4][FP][B]   F~_i[b][f] at (i FP + f) B + b
  // K_c[i][j] vanishes unless deg i < deg j (phi_i is orthogonal to the derivative of phi_j
  // otherwise); those entries are set to exact zeros, so that the padded loops below add
  // exact zeros only
  for (int i = threadIdx.x; i < 3 * BP * B; i += C::THREADS) {
    const int c = i / (BP * B), j = (i / B) % BP, x = i % B;
    const bool in = j < B;
    tKT[i] = (in && mode_degree(x) < mode_degree(j)) ? a.KT[(c * B + j) * B + x] : 0.f;
    tK[i] = (in && mode_degree(j) < mode_degree(x)) ? ops.K[(c * B + j) * B + x] : 0.f;
  }
  for (int i = threadIdx.x; i < 4 * BP * F; i += C::THREADS) {
    const int fi = i / (BP * F), j = (i / F) % BP, f = i % F;
    tFt[i] = (j < B) ? ops.Ft[(fi * B + j) * F + f] : 0.f;
    tFhT[i] = (j < B) ? a.FhT[(fi * B + j) * F + f] : 0.f;
  }
  for (int i = threadIdx.x; i < 4 * FP * B; i += C::THREADS) {
    const int fi = i / (FP * B), f = (i / B) % FP, x = i % B;
    tFtT[i] = (f < F) ? a.FtT[(fi * F + f) * B + x] : 0.f;
  }
  // every group region starts zero: the pad entries are never written afterwards
  for (int i = threadIdx.x; i < C::G * C::ELEM; i += C::THREADS) smem[C::TAB + i] = 0.f;
  __syncthreads();
  const int g = threadIdx.x / NT, t = threadIdx.x % NT;
  float* sS = smem + C::TAB + g * C::ELEM;   // compact S_c [3][36]
  float* sA = sS + C::NSTAR;      // A-_i [4][9][12]: row s of face i at (i 9 + s) 12
  float* sL = sA + C::NALOC;      // [9][BP] lambda
  float* sT = sL + NB9;
  float* sG0 = sT + NB9;          // G ping-pong [2][9][BP]
  float* sDb = sG0 + 2 * NB9;     // D_0 .. D_{O-1} [O][9][BP]
  float* sScr = sDb + O * NB9;    // V_c, then the face products, then Z_c
  for (int k = blockIdx.x * C::G + g; k < a.end; k += gridDim.x * C::G) {
    const int meta = a.meta[k];
    const int cl = meta & 0xff;
    const bool finer = meta & FLAG_FINER, coarser = meta & FLAG_COARSER;
    const bool even = ph.parity[cl] == 0;
    {
      const float* am = a.amat + (size_t)k * AM_SIZE;
      for (int q = t; q < C::NSTAR; q += NT) sS[q] = __ldg(am + AM_STAR + (q / 36) * 81 + star_compact_index(q % 36));
      for (int q = t; q < 4 * 81; q += NT) sA[(q / 9) * 12 + q % 9] = __ldg(am + AM_LOC + q);
    }
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
      stage_pad<B, BP, NT>(sL, a.lq + kf * (9 * B), 1, t);
      stage_pad<B, BP, NT>(sDb, a.Qs + (size_t)k * a.qs + (size_t)(sim / a.G) * (9 * B * a.G) + sim % a.G, a.G, t);
      {
        // the adjoints of the buffers this pass wrote: lambda_B1 (+ lambda_B3) into sG0[0],
        // lambda_B2 into sG0[1]; reset here (lambda_B3 survives an accumulation)
        constexpr int N = 9 * B, R = (N + NT - 1) / NT;
        const size_t o = kf * N;
        float v1[R], v2[R], v3[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int q = t + j * NT;
          v1[j] = v2[j] = v3[j] = 0.f;
          if (q < N) {
            v1[j] = a.lb1[o + q];
            if (coarser) v3[j] = a.lb3[o + q];
            if (finer) v2[j] = a.lb2[o + q];
          }
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int q = t + j * NT;
          if (q < N) {
            const int qp = (q / B) * BP + q % B;
            sG0[qp] = v1[j] + v3[j];
            sG0[NB9 + qp] = v2[j];
            a.lb1[o + q] = 0.f;
            if (coarser && even) a.lb3[o + q] = 0.f;
            if (finer) a.lb2[o + q] = 0.f;
          }
        }
      }
      gsync<NT>(g);
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
#pragma unroll 1
            for (int kk = 0; kk < nin; kk += 4) {
              float4 x[9];
              load_cols4<BP>(sDb + d * NB9, kk, x);
#pragma unroll
              for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  const float kc = tKT[(c * BP + kk + u) * B + t];
#pragma unroll
                  for (int s = 0; s < 9; ++s) Y[c][s] = fmaf(lane4(x[s], u), kc, Y[c][s]);
                }
            }
          float v[9];
#pragma unroll
          for (int r = 0; r < 9; ++r) v[r] = 0.f;
#pragma unroll
          for (int c = 0; c < 3; ++c) star_acc<false>(sS + c * 36, Y[c], v);
#pragma unroll
          for (int r = 0; r < 9; ++r) sDb[(d + 1) * NB9 + r * BP + t] = v[r];
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
          for (int d = 0; d < O; ++d) v = fmaf(ph.coef[cl][d], sDb[d * NB9 + r * BP + t], v);
          sT[r * BP + t] = v;
        }
        // V_c = lambda K_c^T and the volume term
        float V[3][9];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int s = 0; s < 9; ++s) V[c][s] = 0.f;
#pragma unroll 1
        for (int b = 0; b < BP; b += 4) {
          float4 x[9];
          load_cols4<BP>(sL, b, x);
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float kc = tKT[(c * BP + b + u) * B + t];
#pragma unroll
              for (int s = 0; s < 9; ++s) V[c][s] = fmaf(lane4(x[s], u), kc, V[c][s]);
            }
        }
        float w[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) w[r] = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          star_acc<true>(sS + c * 36, V[c], w);
#pragma unroll
          for (int s = 0; s < 9; ++s) sV[c * NB9 + s * BP + t] = V[c][s];
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
        tile33v<BP>(sV + tc * NB9, sT, 3 * trb, 3 * tsb, BP, tv);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int q = 0; q < 3; ++q) wst[i][q] -= tv[i][q];
      }
      gsync<NT>(g);
      // local surface: LF_i = lambda F^_i^T, TF_i = T F~_i, U_i = A-_i^T LF_i, per (face, f);
      // the pad columns f >= F are written zero
      float* sLF = sScr;              // [4][9][FP]
      float* sTF = sScr + 36 * FP;
      float* sU = sScr + 72 * FP;
      for (int p = t; p < 4 * FP; p += NT) {
        const int i = p / FP, f = p % FP;
        float lf[9], tf[9], u[9];
        if (f < F) {
          rows9v<BP, BP>(sL, tFhT + i * BP * F, F, f, lf);
          rows9v<BP, BP>(sT, tFt + i * BP * F, F, f, tf);
#pragma unroll
          for (int r = 0; r < 9; ++r) u[r] = 0.f;
          const float* Am = sA + i * 108;
#pragma unroll
          for (int s = 0; s < 9; ++s) {
            const float4 a0 = *reinterpret_cast<const float4*>(Am + s * 12);
            const float4 a1 = *reinterpret_cast<const float4*>(Am + s * 12 + 4);
            const float a8 = Am[s * 12 + 8];
            u[0] = fmaf(a0.x, lf[s], u[0]);
            u[1] = fmaf(a0.y, lf[s], u[1]);
            u[2] = fmaf(a0.z, lf[s], u[2]);
            u[3] = fmaf(a0.w, lf[s], u[3]);
            u[4] = fmaf(a1.x, lf[s], u[4]);
            u[5] = fmaf(a1.y, lf[s], u[5]);
            u[6] = fmaf(a1.z, lf[s], u[6]);
            u[7] = fmaf(a1.w, lf[s], u[7]);
            u[8] = fmaf(a8, lf[s], u[8]);
          }
        } else {
#pragma unroll
          for (int r = 0; r < 9; ++r) lf[r] = tf[r] = u[r] = 0.f;
        }
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          sLF[(i * 9 + r) * FP + f] = lf[r];
          sTF[(i * 9 + r) * FP + f] = tf[r];
          sU[(i * 9 + r) * FP + f] = u[r];
        }
      }
      gsync<NT>(g);
      if (t < B)
#pragma unroll 1
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int f = 0; f < FP; f += 4) {
            float4 x[9];
            load_cols4<FP>(sU + i * 9 * FP, f, x);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float w = tFtT[(i * FP + f + u) * B + t];
#pragma unroll
              for (int r = 0; r < 9; ++r) mu[r] = fmaf(lane4(x[r], u), w, mu[r]);
            }
          }
      for (int p = t; p < 36; p += NT) {
        const int i = p / 9, rb = (p / 3) % 3, sb = p % 3;
        float acc[3][3];
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
          for (int q = 0; q < 3; ++q) acc[ii][q] = 0.f;
        tile33v<FP>(sLF + i * 9 * FP, sTF + i * 9 * FP, 3 * rb, 3 * sb, FP, acc);
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
          for (int q = 0; q < 3; ++q) atomicAdd(Wk + AM_LOC + i * 81 + (3 * rb + ii) * 9 + 3 * sb + q, (double)acc[ii][q]);
      }
      // the buffers this pass wrote
      if (t < B) {
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          mu[r] += sG0[r * BP + t];
          muh[r] = sG0[NB9 + r * BP + t];
        }
#pragma unroll
        for (int r = 0; r < 9; ++r)
          sG0[((O - 1) & 1) * NB9 + r * BP + t] = ph.coef[cl][O - 1] * mu[r] + ph.hcoef[cl][O - 1] * muh[r];
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
          // entries kk >= nk of G_{d+1} meet K_c[kk][t] = 0 for t < nout (degree structure)
          if (t < nout)
#pragma unroll 1
            for (int kk = 0; kk < nk; kk += 4) {
              float4 x[9];
              load_cols4<BP>(Gn, kk, x);
#pragma unroll
              for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                  const float kc = tK[(c * BP + kk + u) * B + t];
#pragma unroll
                  for (int r = 0; r < 9; ++r) Z[c][r] = fmaf(lane4(x[r], u), kc, Z[c][r]);
                }
            }
          float gv[9];
#pragma unroll
          for (int r = 0; r < 9; ++r) gv[r] = ph.coef[cl][d] * mu[r] + ph.hcoef[cl][d] * muh[r];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            star_acc<true>(sS + c * 36, Z[c], gv);
#pragma unroll
            for (int r = 0; r < 9; ++r) sZ[c * NB9 + r * BP + t] = Z[c][r];
          }
#pragma unroll
          for (int r = 0; r < 9; ++r) sG0[(d & 1) * NB9 + r * BP + t] = gv[r];
        }
        gsync<NT>(g);
        if (t < 27) tile33v<BP>(sZ + tc * NB9, sDb + d * NB9, 3 * trb, 3 * tsb, rup(nout, 4), wst);
        gsync<NT>(g);
      }
      if (t < B)
#pragma unroll
        for (int r = 0; r < 9; ++r) a.lq[kf * (9 * B) + r * B + t] = sL[r * BP + t] + sG0[r * BP + t];
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
  const int kn = a.owners ? a.owners[blockIdx.x] : (int)blockIdx.x, t = threadIdx.x, nt = blockDim.x;
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
