// sm_103a kernels of the ADER-DG LTS update (FP32 CUDA cores).
//
// k_predict_local : time kernel (Cauchy-Kowalevski + Taylor integral, Sec. III-A
//                   "Time Kernel"), LTS buffers B1/B2/B3 (Eq. lts_buffers), volume kernel
//                   and local surface kernel, Q <- ((Q + V) + S^L)   (Eq. update, local part)
// k_neighbour     : neighbour surface kernel with the buffer chosen by the clusters'
//                   time-stepping relation (Sec. V-B), Q <- Q + S^N (Eq. update, neighbouring)
// k_receivers     : Taylor evaluation of d^dQ at receiver points
// k_sources       : moment-tensor point sources
// k_energy        : discrete elastic energy, FP64 reduction
//
// Work decomposition: a CTA owns a batch of NE elements staged in shared memory; thread
// = (element, mode column b). Tasks are ordered by the degree of b (highest first) so a
// warp mostly holds columns of one degree and can skip the zero blocks that the
// hierarchical orthonormal basis puts into K_c (int phi_i d phi_j != 0 only for
// deg i < deg j) and into the face matrices (int psi_f phi_b != 0 only for deg f <= deg b).
// The elastic rows of the operand are staged k-major ([element][mode][row], rows padded to
// 12 floats) so each thread reads 9 rows with two 16-byte and one 4-byte broadcast loads.
// Flux solvers are applied in closed form (normal / tangential impedance split) from 11
// floats per face instead of stored 9x9 and 6x9 matrices.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ltsdev {

__host__ __device__ constexpr int nbasis(int o) { return o * (o + 1) * (o + 2) / 6; }
__host__ __device__ constexpr int nface(int o) { return o * (o + 1) / 2; }
__host__ __device__ constexpr int rup(int x, int m) { return (x + m - 1) / m * m; }

constexpr int ED = 64;   // floats of per-element data for k_predict_local
constexpr int ND = 48;   // floats of per-element data for k_neighbour
constexpr int MAXC = 8;  // max clusters
constexpr int FUSED_GROUP = 4;   // simulations per CTA in fused mode
constexpr int FLAG_FINER = 1 << 8;     // element has a finer neighbour: writes B2
constexpr int FLAG_COARSER = 1 << 9;   // element has a coarser neighbour: writes B3
// ncode bit of a face whose neighbour lies in another partition: nbr then holds the slot of
// the face-local message H = X F-_{j,h} the neighbour's side computed (Sec. V-C)
constexpr int FACE_REMOTE = 1 << 16;

// FG = 1: a CTA slot is an element (single simulation). FG > 1: fused simulations, a CTA
// owns one element and FG of its simulations, one slot per simulation.
template <int O, int M, int FG = 1>
struct Cfg {
  static constexpr int B = nbasis(O), F = nface(O), NQ = 9 + 6 * M, NA = 6 * M;
  static constexpr int BS = (B % 2) ? B : B + 1;     // odd row stride: conflict-free rows and columns
  // staged K_c: three planes [c][row][col], odd row stride KS, read as 4-byte loads (a thread
  // reads its own column: three distinct-bank loads per k instead of one padded 16-byte load
  // that shared memory serves in four quarter-warp phases)
  static constexpr int KS = BS + 2;
  static constexpr int QS = rup(NQ * B, 4);          // element stride of Q
  static constexpr int BUFS = rup(9 * B, 4);         // element stride of B1/B2/B3
  // elements per CTA: 7 x 35 columns = 8 warps at order 5, so two CTAs fit with up to
  // 128 registers per thread (registers are allocated per SM sub-partition)
  static constexpr int NE = (FG > 1) ? FG : ((O == 3) ? 24 : (O == 4 ? 12 : 7));   // slots per CTA
  static constexpr int NEL = (FG > 1) ? 1 : NE;                                       // elements per CTA
  static constexpr int NT = rup(NE * B, 32);
  // resident CTAs per SM the register budget is sized for (registers are allocated per
  // SM sub-partition: 16K per quarter, whole warps)
  static constexpr int PMIN = (FG > 1) ? 3 : 2;
  static constexpr int NMIN = (FG > 1) ? 4 : 2;
  static constexpr int AR = 12;                      // staged elastic rows (padded, 16-byte stores)
  // staged Riemann states (v*, t*: 6 values) per face mode: a stride of 12 floats keeps the
  // 16-byte stores of 8 consecutive tasks on 8 distinct 4-bank groups
  static constexpr int FR = 12;
  // gathered neighbour rows: a stride of 10 floats gives 8-byte row loads and keeps the
  // 8-byte stores of 16 consecutive modes on distinct bank pairs
  static constexpr int XR = 10;
  // k_neighbour's staged Riemann states: 8 floats per face mode, and a slot stride of 4 banks
  // mod 32 so that the 16-byte reads of neighbouring slots do not collide
  static constexpr int FRN = 8;
  static constexpr int FLSN = 4 * F * FRN + 4;
  static constexpr int NPAIR = (F + 1) / 2;           // face-mode pairs of the neighbour product
  // time kernel load balance: columns of degree <= O-3 split their k-range with a
  // helper thread that owns a degree O-1 column (which has no time-kernel product)
  static constexpr int NSPLIT = nbasis(O - 2);
  static constexpr int SPR = 28;                     // floats per staged partial (27 + pad)
  // shared memory (floats) of k_predict_local
  static constexpr int P_K = 0;                      // K_c[row][col] at ((row * BS + col) * 4 + c)
  static constexpr int P_FT = rup(P_K + 3 * B * KS, 4);
  static constexpr int P_FH = rup(P_FT + 4 * B * F, 4);
  static constexpr int P_A = rup(P_FH + 4 * F * B, 4);
  static constexpr int P_FL = rup(P_A + 2 * NE * B * AR, 4);
  // slot stride of the staged Riemann states; odd in 16-byte units when slots vary fastest
  static constexpr int FLS = 4 * F * FR + ((FG > 1) ? 4 : 0);
  static constexpr int P_E = rup(P_FL + NE * FLS, 4);
  static constexpr int P_SP = rup(P_E + NEL * ED, 4);
  static constexpr int P_META = rup(P_SP + NE * NSPLIT * SPR, 4);
  static constexpr int P_TOTAL = rup(P_META + NEL, 4);
  // k_neighbour: its own batch size (kept equal to NE: a third CTA per SM leaves too
  // little L1 for the neighbour-buffer gathers)
  static constexpr int NEN = (FG > 1) ? FG : ((O == 5) ? 8 : NE);
  static constexpr int NELN = (FG > 1) ? 1 : NEN;
  static constexpr int NTN = rup(NEN * B, 32);
  static constexpr int N_FB = 0;
  static constexpr int N_FH = rup(N_FB + 12 * B * F, 4);
  static constexpr int N_X = rup(N_FH + 4 * F * B, 4);
  static constexpr int N_FL = rup(N_X + NEN * 4 * B * XR, 4);
  static constexpr int N_D = rup(N_FL + NEN * FLSN, 4);
  static constexpr int N_I = rup(N_D + NELN * ND, 4);      // ints: nbr[4], code[4], meta per element
  static constexpr int N_TOTAL = rup(N_I + NELN * 9, 4);
};

struct DevOps {
  const float* K;    // [3][B][B]   K_c[i][j] = int phi_i d phi_j / d xi_c
  const float* Ft;   // [4][B][F]   F~_i
  const float* Fh;   // [4F][B]     F^ stacked: row i*F+f = F^_i[f][:]
  const float* Fb;   // [12][B][F]  F-_{j,h}, index j*3+h
  const float* Rh;   // [3][F][F]   face-basis map of orientation h: F-_{j,h} = F~_j R_h
};

struct DevState {
  // Simulations are blocked in groups of G (G = FUSED_GROUP in fused mode, else 1): element k,
  // quantity r, mode b, simulation f = G g + j sits at Q[k * qs + g * NQ B G + (r B + b) G + j],
  // qs = NQ B nsim (one simulation: QS, rows padded); the LTS buffers likewise with 9 rows
  // and element stride bs.
  long long qs, bs;
  int nsim;
  float* Q;
  float* B1;
  float* B2;
  float* B3;
  const float* edata;    // [K][ED]
  const float* ndata;    // [K][ND]
  const int* nbr;        // [K][4] neighbour (internal index) or -1
  const int* ncode;      // [K][4] (j*3+h) | (relation << 8): 0 same, 1 neighbour finer, 2 neighbour coarser
  const int* meta;       // [K] cluster | FLAG_*
  const float* msg;      // [cut faces][nsim][9][F] face-local messages of a partitioned run (else unused)
};

struct PhaseArgs {
  int begin, end;              // element range (internal order)
  float coef[MAXC][6];         // dt_l^(d+1)/(d+1)!
  float hcoef[MAXC][6];        // (dt_l/2)^(d+1)/(d+1)!
  int parity[MAXC];            // step index parity of each cluster in this phase
  float omega[3];
  // bounded waits of the asynchronous copies (k_predict_sp): the device error word a kernel
  // sets when a wait gives up, the bound in SM cycles, and the failure-path test switch
  // (nothing is copied, so the waits run out)
  int* err;
  long long wait;
  int suppress;
};

// ------------------------------------------------------------------ helpers
// L2 prefetch of the DOFs a CTA's next batch reads: elements [e0, e0 + n) x qs floats
// (one simulation), or one simulation group's NQ x B x FG block of element e0 (fused);
// one 128-byte line per thread and step, every address inside the block.
template <int NQ, int B, int FG, int NT>
__device__ __forceinline__ void prefetch_batch_q(const float* Q, long long qs, int e0, int grp, int n, int tid) {
  const float* p = Q + (size_t)e0 * qs + ((FG > 1) ? (size_t)grp * (NQ * B * FG) : 0);
  const long long len = (FG > 1) ? (long long)NQ * B * FG : (long long)n * qs;
  for (long long off = 32LL * tid; off < len; off += 32LL * NT) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + off));
}

// Tasks ordered by the degree of the mode column, highest first; within a degree the mode
// varies fastest (SF = false) or the slot does (SF = true: fused simulations, so that
// neighbouring threads touch neighbouring simulations of one DOF).
template <int O, int NE, bool SF = false>
__device__ __forceinline__ void task_of(int t, int& e, int& b, int& p) {
  int off = 0;
#pragma unroll
  for (int q = O - 1; q >= 0; --q) {
    const int np = (q + 1) * (q + 2) / 2;
    if (t >= off && t < off + NE * np) {
      const int idx = t - off;
      e = SF ? idx % NE : idx / np;
      b = nbasis(q) + (SF ? idx / NE : idx % np);
      p = q;
    }
    off += NE * np;
  }
}

// Face tasks (element, face, face mode f), ordered by the degree of f (highest first): the
// product with F~ / F- only involves modes of degree >= deg f.
template <int O, int NE, bool SF = false>
__device__ __forceinline__ void face_task_of(int t, int& ee, int& i, int& f, int& pf) {
  int off = 0;
  ee = -1;
  i = f = pf = 0;
#pragma unroll
  for (int q = O - 1; q >= 0; --q) {
    const int n = NE * 4 * (q + 1);
    if (t >= off && t < off + n) {
      const int idx = t - off, r = SF ? idx / NE : idx % (4 * (q + 1));
      ee = SF ? idx % NE : idx / (4 * (q + 1));
      i = r / (q + 1);
      f = nface(q) + r % (q + 1);
      pf = q;
    }
    off += n;
  }
}

// Polynomial degree of face mode f (modes are ordered by degree).
__device__ __forceinline__ int face_degree(int f) {
  int q = 0;
  while (nface(q + 1) <= f) ++q;
  return q;
}

// Face-mode pair tasks of the face products: pair a holds modes F-1-2a and F-2-2a (the
// second absent when F is odd and a is the last pair), i.e. modes of equal or neighbouring
// degree, so that the pair's k-range (that of its lower-degree mode) adds few zero terms.
// The pair index varies slowest: the threads of a warp then walk the same k together, and
// a staged row read is one broadcast per slot instead of one address per pair (shared
// memory serves a 16-byte load in quarter-warp phases, a 4-byte broadcast in one). Within
// a pair the slot varies fastest for fused simulations (SF), else the face.
template <int NE, bool SF = false>
__device__ __forceinline__ void face_pair_of(int t, int& ee, int& i, int& a) {
  a = t / (4 * NE);
  const int r = t % (4 * NE);
  ee = SF ? r % NE : r / 4;
  i = SF ? r / NE : r % 4;
}

__device__ __forceinline__ void st2(float* p, float a, float b) {
  *reinterpret_cast<float2*>(p) = make_float2(a, b);
}

__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

// Physical combination of reference-derivative projections Y[c][q] (Sec. III-A star
// matrices): with W_d = sum_c dxi_c/dx_d Y_c, out = -sum_d A_d W_d (elastic Jacobians) and
// eps = sym grad v (the strain-rate projection). Jinv[c*3+d] = dxi_c/dx_d.
__device__ __forceinline__ void star_apply(const float (&Y)[3][9], const float* ed, float (&out)[9], float (&eps)[6]) {
  float g[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int j = 0; j < 3; ++j) g[d][j] = ed[d] * Y[0][6 + j] + ed[3 + d] * Y[1][6 + j] + ed[6 + d] * Y[2][6 + j];
  // stress divergence: sum_d d sigma_{i d} / d x_d
  const int SIG[3][3] = {{0, 3, 5}, {3, 1, 4}, {5, 4, 2}};
  float dv[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float s = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) s += ed[d] * Y[0][SIG[i][d]] + ed[3 + d] * Y[1][SIG[i][d]] + ed[6 + d] * Y[2][SIG[i][d]];
    dv[i] = s;
  }
  const float lam = ed[9], mu = ed[10], rinv = ed[11];
  const float tr = g[0][0] + g[1][1] + g[2][2];
  out[0] = lam * tr + 2.f * mu * g[0][0];
  out[1] = lam * tr + 2.f * mu * g[1][1];
  out[2] = lam * tr + 2.f * mu * g[2][2];
  out[3] = mu * (g[0][1] + g[1][0]);
  out[4] = mu * (g[1][2] + g[2][1]);
  out[5] = mu * (g[0][2] + g[2][0]);
  out[6] = rinv * dv[0];
  out[7] = rinv * dv[1];
  out[8] = rinv * dv[2];
  eps[0] = g[0][0];
  eps[1] = g[1][1];
  eps[2] = g[2][2];
  eps[3] = 0.5f * (g[0][1] + g[1][0]);
  eps[4] = 0.5f * (g[1][2] + g[2][1]);
  eps[5] = 0.5f * (g[0][2] + g[2][0]);
}

// E^l theta: stress rows -(lam Y^lam_l tr(theta) I + 2 mu Y^mu_l theta); ylam = lam Y^lam_l, ymu2 = 2 mu Y^mu_l
__device__ __forceinline__ void coupling_add(float (&s)[9], const float* th, float ylam, float ymu2) {
  const float tr = th[0] + th[1] + th[2];
  s[0] -= ylam * tr + ymu2 * th[0];
  s[1] -= ylam * tr + ymu2 * th[1];
  s[2] -= ylam * tr + ymu2 * th[2];
  s[3] -= ymu2 * th[3];
  s[4] -= ymu2 * th[4];
  s[5] -= ymu2 * th[5];
}

// Upwind (Godunov) interface state of a face state g (9 quantities, xyz components) in
// closed form. fd = n[3], a[4], b[4]: v*_n = a0 v_n + a1 t_n, t*_n = a2 t_n + a3 v_n (P pair)
// and the same with b for the tangential (S) parts, t = sigma n; the coefficients carry the
// -2|S_i|/|det J| scaling. w = (v*, t*).
__device__ __forceinline__ void riemann_state(const float (&g)[9], const float* fd, float (&w)[6]) {
  const float nx = fd[0], ny = fd[1], nz = fd[2];
  const float tx = g[0] * nx + g[3] * ny + g[5] * nz;
  const float ty = g[3] * nx + g[1] * ny + g[4] * nz;
  const float tz = g[5] * nx + g[4] * ny + g[2] * nz;
  const float tn = tx * nx + ty * ny + tz * nz;
  const float vn = g[6] * nx + g[7] * ny + g[8] * nz;
  const float tTx = tx - tn * nx, tTy = ty - tn * ny, tTz = tz - tn * nz;
  const float vTx = g[6] - vn * nx, vTy = g[7] - vn * ny, vTz = g[8] - vn * nz;
  const float vsn = fd[3] * vn + fd[4] * tn;
  const float tsn = fd[5] * tn + fd[6] * vn;
  w[0] = vsn * nx + fd[7] * vTx + fd[8] * tTx;
  w[1] = vsn * ny + fd[7] * vTy + fd[8] * tTy;
  w[2] = vsn * nz + fd[7] * vTz + fd[8] * tTz;
  w[3] = tsn * nx + fd[9] * tTx + fd[10] * vTx;
  w[4] = tsn * ny + fd[9] * tTy + fd[10] * vTy;
  w[5] = tsn * nz + fd[9] * tTz + fd[10] * vTz;
}

__device__ __forceinline__ void store_state(float* dst, const float (&w)[6]) {
  st4(dst, w[0], w[1], w[2], w[3]);
  *reinterpret_cast<float2*>(dst + 4) = make_float2(w[4], w[5]);
}

// Flux rows of a projected interface state W = (v*, t*) on a face with normal n, added to S:
// stresses -(lam (n.v*) I + mu (n v*^T + v* n^T)), velocities -t*/rho and, for M > 0, the
// memory-variable rows -sym(n v*^T) (omega_l factored out) in S[9..14]. The flux is linear
// in (v*, t*), so projecting these 6 rows through F^ and forming the flux afterwards equals
// projecting the 15 flux rows.
template <int NS>
__device__ __forceinline__ void flux_rows_add(const float (&W)[6], const float* n, float lam, float mu, float rinv,
                                              float (&S)[NS]) {
  const float nx = n[0], ny = n[1], nz = n[2];
  const float nv = nx * W[0] + ny * W[1] + nz * W[2];
  const float exx = nx * W[0], eyy = ny * W[1], ezz = nz * W[2];
  const float exy = nx * W[1] + ny * W[0], eyz = ny * W[2] + nz * W[1], exz = nx * W[2] + nz * W[0];
  const float ln = lam * nv, m2 = 2.f * mu;
  S[0] -= ln + m2 * exx;
  S[1] -= ln + m2 * eyy;
  S[2] -= ln + m2 * ezz;
  S[3] -= mu * exy;
  S[4] -= mu * eyz;
  S[5] -= mu * exz;
  S[6] -= rinv * W[3];
  S[7] -= rinv * W[4];
  S[8] -= rinv * W[5];
  if constexpr (NS > 9) {
    S[9] -= exx;
    S[10] -= eyy;
    S[11] -= ezz;
    S[12] -= 0.5f * exy;
    S[13] -= 0.5f * eyz;
    S[14] -= 0.5f * exz;
  }
}

// S[r][b] += sum over faces i and face modes f (deg f <= deg b) of the flux of the staged
// interface states projected by F^_i[f][b].
template <int NS, int F, int B, int FR>
__device__ __forceinline__ void project_faces(const float* Fl, const float* sFh, const float* nrm, int nstride,
                                              float lam, float mu, float rinv, int fmax, int b, float (&S)[NS]) {
#pragma unroll 1
  for (int i = 0; i < 4; ++i) {
    float W[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int f = 0; f < fmax; ++f) {
      const float* fl = Fl + (i * F + f) * FR;
      const float w = sFh[(i * F + f) * B + b];
      const float4 y0 = *reinterpret_cast<const float4*>(fl);
      const float2 y1 = *reinterpret_cast<const float2*>(fl + 4);
      W[0] = fmaf(y0.x, w, W[0]);
      W[1] = fmaf(y0.y, w, W[1]);
      W[2] = fmaf(y0.z, w, W[2]);
      W[3] = fmaf(y0.w, w, W[3]);
      W[4] = fmaf(y1.x, w, W[4]);
      W[5] = fmaf(y1.y, w, W[5]);
    }
    flux_rows_add<NS>(W, nrm + nstride * i, lam, mu, rinv, S);
  }
}

// ------------------------------------------------------------------ predict + local
template <int O, int M, int FG>
__global__ void __launch_bounds__(Cfg<O, M, FG>::NT, Cfg<O, M, FG>::PMIN) k_predict_local(DevOps ops, DevState st, PhaseArgs ph) {
  using C = Cfg<O, M, FG>;
  constexpr int B = C::B, F = C::F, NE = C::NE, NEL = C::NEL, NT = C::NT, KS = C::KS, AR = C::AR, FR = C::FR;
  constexpr int NQ = C::NQ, NA = C::NA, NSPLIT = C::NSPLIT, SPR = C::SPR;
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  float* sK = smem + C::P_K;
  float* sFt = smem + C::P_FT;
  float* sFh = smem + C::P_FH;
  float* sA = smem + C::P_A;
  float* sFl = smem + C::P_FL;
  float* sE = smem + C::P_E;
  float* sSP = smem + C::P_SP;
  int* sMeta = reinterpret_cast<int*>(smem + C::P_META);
  const int tid = threadIdx.x;

  for (int i = tid; i < 3 * B * KS; i += NT) {
    const int c = i / (B * KS), r = (i / KS) % B, col = i % KS;
    sK[i] = (col < B) ? ops.K[(c * B + r) * B + col] : 0.f;
  }
  // F~_i[k][f] vanishes for deg k < deg f; staged as exact zeros (see the neighbour kernel)
  for (int i = tid; i < 4 * B * F; i += NT) {
    const int f = i % F, k = (i / F) % B;
    sFt[i] = (k < nbasis(face_degree(f))) ? 0.f : ops.Ft[i];
  }
  for (int i = tid; i < 4 * F * B; i += NT) sFh[i] = ops.Fh[i];

  int e = -1, b = 0, p = 0;
  task_of<O, NE, (FG > 1)>(tid, e, b, p);
  const bool act = e >= 0;
  const int es = act ? e : 0;
  // time-kernel product of this thread: column ck_col over a k-range set per derivative
  const int hj = b - nbasis(O - 1);                    // index among the degree O-1 columns
  const bool helper = act && p == O - 1 && hj < NSPLIT;
  const bool split_owner = act && b < NSPLIT;
  // (k-range of the first derivative; a split owner takes the first half of its column's
  // range, the helper the second)
  auto kmid = [](int col, int pd) { return (nbasis(pd + 1) + B + 1) / 2; };
  int ck_col = b, ck_p = p, ck_k0 = nbasis(p + 1), ck_k1 = B;
  if (helper) {
    int ph_ = 0;
    while (nbasis(ph_ + 1) <= hj) ++ph_;
    ck_col = hj;
    ck_p = ph_;
    ck_k0 = kmid(hj, ph_);
    ck_k1 = B;
  } else if (split_owner) {
    ck_k1 = kmid(b, p);
  }
  if (!act) ck_k0 = ck_k1 = 0;
  const int ke_vol = nbasis(p);         // K_c[k][b] != 0 needs deg k < deg b
  const int fmax = nface(p + 1);        // face modes of degree <= deg b
  const int nelem = ph.end - ph.begin;
  // element strides and simulation count: compile-time constants for one simulation
  const long long qs = (FG > 1) ? st.qs : C::QS, bs = (FG > 1) ? st.bs : C::BUFS;
  const int nsim = (FG > 1) ? st.nsim : 1;
  const int nsg = nsim / FG;                             // simulation groups per element
  const int nbatch = (FG > 1) ? nelem * nsg : (nelem + NE - 1) / NE;
  constexpr int rs = B * FG;                             // row stride of Q and the buffers

  for (int batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int e0 = (FG > 1) ? ph.begin + batch / nsg : ph.begin + batch * NE;
    const int grp = (FG > 1) ? batch % nsg : 0;          // simulation group
    __syncthreads();
    const int g = e0 + ((FG > 1) ? 0 : e);
    const int eb = (FG > 1) ? 0 : es;                    // element slot in the staged tables
    const int j = (FG > 1) ? es : 0;                     // simulation within the group
    const bool valid = act && g < ph.end;
    const size_t qoff = (size_t)g * qs + (size_t)grp * (C::NQ * B * FG) + b * FG + j;
    const size_t boff = (size_t)g * bs + (size_t)grp * (9 * B * FG) + b * FG + j;
    // DOF loads are issued together with the element tables, before the barrier
    float T[NQ], Th[9], Da[NA > 0 ? NA : 1];
    float v[12];
#pragma unroll
    for (int r = 0; r < 12; ++r) v[r] = 0.f;
    if (valid) {
      const float* q = st.Q + qoff;
#pragma unroll
      for (int r = 0; r < 9; ++r) v[r] = q[r * rs];
#pragma unroll
      for (int r = 0; r < NA; ++r) Da[r] = q[(9 + r) * rs];
    } else {
#pragma unroll
      for (int r = 0; r < NA; ++r) Da[r] = 0.f;
    }
    for (int i = tid; i < NEL * ED; i += NT) {
      const int ee = i / ED, gg = e0 + ee;
      sE[i] = (gg < ph.end) ? st.edata[(size_t)gg * ED + (i % ED)] : 0.f;
    }
    if (tid < NEL) sMeta[tid] = (e0 + tid < ph.end) ? st.meta[e0 + tid] : 0;
    __syncthreads();
    const float* ed = sE + eb * ED;
    const int meta = act ? sMeta[eb] : 0;
    const int cl = meta & 0xff;
    {
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        T[r] = ph.coef[cl][0] * v[r];
        Th[r] = ph.hcoef[cl][0] * v[r];
      }
#pragma unroll
      for (int r = 0; r < NA; ++r) T[9 + r] = ph.coef[cl][0] * Da[r];
      if (act) {
        float* a0 = sA + ((0 * NE + es) * B + b) * AR;
        st4(a0, v[0], v[1], v[2], v[3]);
        st4(a0 + 4, v[4], v[5], v[6], v[7]);
        st4(a0 + 8, v[8], 0.f, 0.f, 0.f);
      }
    }
    // ---- time kernel: d^{d+1} Q from d^d Q (Cauchy-Kowalevski), Taylor sums
    int buf = 0;
#pragma unroll 1
    for (int d = 0; d < O - 1; ++d) {
      __syncthreads();
      float Y[3][9];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 9; ++r) Y[c][r] = 0.f;
      {
        // X = d^d Q: column ck_col needs the modes k of degree > deg ck_col. Elastic: d^d Q
        // has degree <= O-1-d (each derivative is one spatial derivative), so only the first
        // nbasis(O-d) modes are nonzero; the anelastic coupling keeps every degree
        int k0 = ck_k0, k1 = ck_k1;
        if constexpr (M == 0) {
          const int kend = nbasis(O - d);
          const int kb = nbasis(ck_p + 1), km = max(kb, (kb + kend + 1) / 2);
          k0 = act ? (helper ? km : kb) : 0;
          k1 = act ? (split_owner ? km : kend) : 0;
        }
        const float* Ab = sA + ((buf * NE + es) * B) * AR;
        const float* K0 = sK + ck_col * KS;
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
          const float4 x0 = *reinterpret_cast<const float4*>(Ab + k * AR);
          const float4 x1 = *reinterpret_cast<const float4*>(Ab + k * AR + 4);
          const float x8 = Ab[k * AR + 8];
          const float xs[9] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w, x8};
          const float kc[3] = {K0[k], K0[B * KS + k], K0[2 * B * KS + k]};
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < 9; ++r) Y[c][r] = fmaf(xs[r], kc[c], Y[c][r]);
        }
      }
      if (helper) {
        // hand the second half of column hj's product to its owner
        float* sp = sSP + (es * NSPLIT + hj) * SPR;
        st4(sp, Y[0][0], Y[0][1], Y[0][2], Y[0][3]);
        st4(sp + 4, Y[0][4], Y[0][5], Y[0][6], Y[0][7]);
        st4(sp + 8, Y[0][8], Y[1][0], Y[1][1], Y[1][2]);
        st4(sp + 12, Y[1][3], Y[1][4], Y[1][5], Y[1][6]);
        st4(sp + 16, Y[1][7], Y[1][8], Y[2][0], Y[2][1]);
        st4(sp + 20, Y[2][2], Y[2][3], Y[2][4], Y[2][5]);
        st4(sp + 24, Y[2][6], Y[2][7], Y[2][8], 0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int r = 0; r < 9; ++r) Y[c][r] = 0.f;    // own column has degree O-1: no product
      }
      __syncthreads();
      if (split_owner) {
        const float* sp = sSP + (es * NSPLIT + b) * SPR;
        float w[28];
#pragma unroll
        for (int q4 = 0; q4 < 7; ++q4) {
          const float4 t4 = *reinterpret_cast<const float4*>(sp + 4 * q4);
          w[4 * q4] = t4.x;
          w[4 * q4 + 1] = t4.y;
          w[4 * q4 + 2] = t4.z;
          w[4 * q4 + 3] = t4.w;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int r = 0; r < 9; ++r) Y[c][r] += w[c * 9 + r];
      }
      if (act) {
        float out[9], eps[6];
        star_apply(Y, ed, out, eps);
#pragma unroll
        for (int l = 0; l < M; ++l) coupling_add(out, Da + 6 * l, ed[12 + 2 * l], ed[13 + 2 * l]);
        const float c1 = ph.coef[cl][d + 1], h1 = ph.hcoef[cl][d + 1];
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          T[r] = fmaf(c1, out[r], T[r]);
          Th[r] = fmaf(h1, out[r], Th[r]);
        }
#pragma unroll
        for (int l = 0; l < M; ++l)
#pragma unroll
          for (int r = 0; r < 6; ++r) {
            const float v = ph.omega[l] * (eps[r] - Da[6 * l + r]);
            Da[6 * l + r] = v;
            T[9 + 6 * l + r] = fmaf(c1, v, T[9 + 6 * l + r]);
          }
        float* an = sA + (((buf ^ 1) * NE + es) * B + b) * AR;
        st4(an, out[0], out[1], out[2], out[3]);
        st4(an + 4, out[4], out[5], out[6], out[7]);
        st4(an + 8, out[8], 0.f, 0.f, 0.f);
      }
      buf ^= 1;
    }
    // ---- LTS buffers (Eq. lts_buffers)
    if (valid) {
      float* b1 = st.B1 + boff;
#pragma unroll
      for (int r = 0; r < 9; ++r) b1[r * rs] = T[r];
      if (meta & FLAG_FINER) {
        float* b2 = st.B2 + boff;
#pragma unroll
        for (int r = 0; r < 9; ++r) b2[r * rs] = Th[r];
      }
      if (meta & FLAG_COARSER) {
        float* b3 = st.B3 + boff;
        if (ph.parity[cl] == 0) {
#pragma unroll
          for (int r = 0; r < 9; ++r) b3[r * rs] = T[r];
        } else {
#pragma unroll
          for (int r = 0; r < 9; ++r) b3[r * rs] += T[r];
        }
      }
    }
    // ---- volume kernel
    if (act) {
      float* a = sA + ((buf * NE + es) * B + b) * AR;
      st4(a, T[0], T[1], T[2], T[3]);
      st4(a + 4, T[4], T[5], T[6], T[7]);
      st4(a + 8, T[8], 0.f, 0.f, 0.f);
    }
    __syncthreads();
    float acc[NQ];
    {
      float Z[3][9];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 9; ++r) Z[c][r] = 0.f;
      if (act) {
        const float* Ab = sA + ((buf * NE + e) * B) * AR;
#pragma unroll 4
        for (int k = 0; k < ke_vol; ++k) {
          const float4 x0 = *reinterpret_cast<const float4*>(Ab + k * AR);
          const float4 x1 = *reinterpret_cast<const float4*>(Ab + k * AR + 4);
          const float x8 = Ab[k * AR + 8];
          const float* Kk = sK + k * KS + b;
          const float xs[9] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w, x8};
          const float kc[3] = {Kk[0], Kk[B * KS], Kk[2 * B * KS]};
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < 9; ++r) Z[c][r] = fmaf(xs[r], kc[c], Z[c][r]);
        }
      }
      if (valid) {
        float out[9], eps[6];
        star_apply(Z, ed, out, eps);
        float V[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) V[r] = -out[r];
#pragma unroll
        for (int l = 0; l < M; ++l) coupling_add(V, T + 9 + 6 * l, ed[12 + 2 * l], ed[13 + 2 * l]);
        const float* q = st.Q + qoff;
#pragma unroll
        for (int r = 0; r < 9; ++r) acc[r] = q[r * rs] + V[r];
#pragma unroll
        for (int l = 0; l < M; ++l)
#pragma unroll
          for (int r = 0; r < 6; ++r)
            acc[9 + 6 * l + r] = q[(9 + 6 * l + r) * rs] + ph.omega[l] * (-eps[r] - T[9 + 6 * l + r]);
      }
    }
    // ---- local surface kernel: G_i = T^e F~_i for two face modes per task (as in the
    // neighbour kernel), flux, staged for F^
#pragma unroll 1
    for (int t = tid; t < NE * 4 * C::NPAIR; t += NT) {
      int fe, fi, a;
      face_pair_of<NE, (FG > 1)>(t, fe, fi, a);
      const int f1 = F - 1 - 2 * a, f2 = f1 - 1;     // f2 < 0: f1 alone
      const int f2r = (f2 >= 0) ? f2 : f1;
      float g1[9], g2[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) g1[r] = g2[r] = 0.f;
      const float* Ab = sA + ((buf * NE + fe) * B) * AR;
      const float* Fi = sFt + fi * B * F;
#pragma unroll 4
      for (int k = nbasis(face_degree(f2r)); k < B; ++k) {
        const float4 x0 = *reinterpret_cast<const float4*>(Ab + k * AR);
        const float4 x1 = *reinterpret_cast<const float4*>(Ab + k * AR + 4);
        const float xs[9] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w, Ab[k * AR + 8]};
        const float w1 = Fi[k * F + f1], w2 = Fi[k * F + f2r];
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          g1[r] = fmaf(xs[r], w1, g1[r]);
          g2[r] = fmaf(xs[r], w2, g2[r]);
        }
      }
      const float* fd = sE + ((FG > 1) ? 0 : fe) * ED + 20 + 11 * fi;
      float* fl = sFl + fe * C::FLS + fi * F * FR;
      float w6[6];
      riemann_state(g1, fd, w6);
      store_state(fl + f1 * FR, w6);
      if (f2 >= 0) {
        riemann_state(g2, fd, w6);
        store_state(fl + f2 * FR, w6);
      }
    }
    __syncthreads();
    if (valid) {
      constexpr int NS = (M > 0) ? 15 : 9;
      float S[NS];
#pragma unroll
      for (int r = 0; r < NS; ++r) S[r] = 0.f;
      project_faces<NS, F, B, FR>(sFl + e * C::FLS, sFh, ed + 20, 11, ed[9], ed[10], ed[11], fmax, b, S);
      float* q = st.Q + qoff;
#pragma unroll
      for (int r = 0; r < 9; ++r) q[r * rs] = acc[r] + S[r];
      if constexpr (M > 0) {
#pragma unroll
        for (int l = 0; l < M; ++l)
#pragma unroll
          for (int r = 0; r < 6; ++r) q[(9 + 6 * l + r) * rs] = acc[9 + 6 * l + r] + ph.omega[l] * S[NS - 6 + r];
      }
    }
    {
      const int bn = batch + gridDim.x;                    // this CTA's next batch
      if (bn < nbatch) {
        const int en = (FG > 1) ? ph.begin + bn / nsg : ph.begin + bn * NE;
        prefetch_batch_q<NQ, B, FG, NT>(st.Q, qs, en, (FG > 1) ? bn % nsg : 0, min(NE, ph.end - en), tid);
      }
    }
  }
}

// ------------------------------------------------------------------ neighbour
template <int O, int M, int FG>
__global__ void __launch_bounds__(Cfg<O, M, FG>::NTN, Cfg<O, M, FG>::NMIN) k_neighbour(DevOps ops, DevState st, PhaseArgs ph) {
  using C = Cfg<O, M, FG>;
  constexpr int B = C::B, F = C::F, NE = C::NEN, NEL = C::NELN, NT = C::NTN, FR = C::FRN, XR = C::XR;
  constexpr int NPAIR = C::NPAIR;
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  float* sFb = smem + C::N_FB;
  float* sFh = smem + C::N_FH;
  float* sX = smem + C::N_X;
  float* sFl = smem + C::N_FL;
  float* sD = smem + C::N_D;
  int* sI = reinterpret_cast<int*>(smem + C::N_I);   // per element: nbr[4], code[4], meta
  const int tid = threadIdx.x;
  // F-_{j,h}[k][f] vanishes for deg k < deg f (the trace of a lower-degree polynomial is
  // orthogonal to face mode f); those entries are staged as exact zeros, so that a face-mode
  // pair may run over the k-range of its lower-degree mode and the other mode's extra terms
  // add nothing
  for (int i = tid; i < 12 * B * F; i += NT) {
    const int f = i % F, k = (i / F) % B;
    sFb[i] = (k < nbasis(face_degree(f))) ? 0.f : ops.Fb[i];
  }
  for (int i = tid; i < 4 * F * B; i += NT) sFh[i] = ops.Fh[i];

  int e = -1, b = 0, p = 0;
  task_of<O, NE, (FG > 1)>(tid, e, b, p);
  const bool act = e >= 0;
  const int fmax = nface(p + 1);
  const int nelem = ph.end - ph.begin;
  const long long qs = (FG > 1) ? st.qs : C::QS, bs = (FG > 1) ? st.bs : C::BUFS;
  const int nsim = (FG > 1) ? st.nsim : 1;
  const int nsg = nsim / FG;
  const int nbatch = (FG > 1) ? nelem * nsg : (nelem + NE - 1) / NE;
  constexpr int rs = B * FG;

  // per-element tables (face data; neighbours, codes, meta) of a batch, fetched into
  // registers one batch ahead so that the gathers need not wait for them
  constexpr int RD = (NEL * ND + NT - 1) / NT, RI = (NEL * 9 + NT - 1) / NT;
  float pd[RD];
  int pi[RI];
  auto fetch = [&](int bt) {
    const int f0 = (FG > 1) ? ph.begin + bt / nsg : ph.begin + bt * NE;
#pragma unroll
    for (int u = 0; u < RD; ++u) {
      const int i = tid + u * NT, gg = f0 + i / ND;
      pd[u] = (i < NEL * ND && bt < nbatch && gg < ph.end) ? __ldg(st.ndata + (size_t)gg * ND + (i % ND)) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < RI; ++u) {
      const int i = tid + u * NT, c = i % 9, gg = f0 + i / 9;
      int v = -1;
      if (i < NEL * 9 && bt < nbatch && gg < ph.end)
        v = (c < 4) ? __ldg(st.nbr + (size_t)gg * 4 + c) : (c < 8 ? __ldg(st.ncode + (size_t)gg * 4 + c - 4) : __ldg(st.meta + gg));
      pi[u] = v;
    }
  };
  fetch(blockIdx.x);
  for (int batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int e0 = (FG > 1) ? ph.begin + batch / nsg : ph.begin + batch * NE;
    const int grp = (FG > 1) ? batch % nsg : 0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < RD; ++u)
      if (tid + u * NT < NEL * ND) sD[tid + u * NT] = pd[u];
#pragma unroll
    for (int u = 0; u < RI; ++u)
      if (tid + u * NT < NEL * 9) sI[tid + u * NT] = pi[u];
    fetch(batch + gridDim.x);
    {
      const int bn = batch + gridDim.x;
      if (bn < nbatch) {
        const int en = (FG > 1) ? ph.begin + bn / nsg : ph.begin + bn * NE;
        prefetch_batch_q<C::NQ, B, FG, NT>(st.Q, qs, en, (FG > 1) ? bn % nsg : 0, min(NE, ph.end - en), tid);
      }
    }
    __syncthreads();
    const int g = e0 + ((FG > 1) ? 0 : e);
    const int eb = (FG > 1) ? 0 : e;                     // element slot in the staged tables
    const int j = (FG > 1) ? e : 0;
    const bool valid = act && g < ph.end;
    // ---- gather the neighbours' time-integrated DOFs by cluster relation (Sec. V-B):
    // all 4 x 9 loads are issued before the shared-memory stores
    if (act) {
      const int* ie = sI + eb * 9;
      const int cl = ie[8] & 0xff;
      const int par = valid ? ph.parity[cl] : 0;
      float xv[4][9];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int nb = (valid && !(ie[4 + i] & FACE_REMOTE)) ? ie[i] : -1;
        const int rel = (ie[4 + i] >> 8) & 0xff;
        const float* src1 = (rel == 1) ? st.B3 : ((rel == 2 && par == 0) ? st.B2 : st.B1);
        const bool sub = (rel == 2 && par == 1);
        const size_t off = (size_t)(nb < 0 ? 0 : nb) * bs + (size_t)grp * (9 * B * FG) + b * FG + j;
#pragma unroll
        for (int r = 0; r < 9; ++r) xv[i][r] = (nb < 0) ? 0.f : __ldg(src1 + off + r * rs);
        if (sub) {
#pragma unroll
          for (int r = 0; r < 9; ++r) xv[i][r] -= __ldg(st.B2 + off + r * rs);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float* x = sX + ((e * 4 + i) * B + b) * XR;
        st2(x, xv[i][0], xv[i][1]);
        st2(x + 2, xv[i][2], xv[i][3]);
        st2(x + 4, xv[i][4], xv[i][5]);
        st2(x + 6, xv[i][6], xv[i][7]);
        x[8] = xv[i][8];
      }
    }
    __syncthreads();
    // ---- H_i = X F-_{j,h} for two face modes per task (they share the staged rows),
    // closed-form interface states with the neighbour's coefficients
#pragma unroll 1
    for (int t = tid; t < NE * 4 * NPAIR; t += NT) {
      int ee, i, a;
      face_pair_of<NE, (FG > 1)>(t, ee, i, a);
      const int eel = (FG > 1) ? 0 : ee;
      if (sI[eel * 9 + 8] < 0) continue;   // slot past the end of the phase: no face data
      const int f1 = F - 1 - 2 * a, f2 = f1 - 1;     // f2 < 0: f1 alone
      const int f2r = (f2 >= 0) ? f2 : f1;
      const int code = sI[eel * 9 + 4 + i];
      const int jh = code & 0xff;
      float g1[9], g2[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) g1[r] = g2[r] = 0.f;
      if (code & FACE_REMOTE) {
        // computed by the neighbour's partition (k_pack_faces), one message per simulation
        const int sim = (FG > 1) ? grp * FG + ee : 0;
        const float* h = st.msg + ((size_t)sI[eel * 9 + i] * nsim + sim) * 9 * F;
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          g1[r] = h[r * F + f1];
          g2[r] = h[r * F + f2r];
        }
      } else {
        const float* X = sX + (ee * 4 + i) * B * XR;
        const float* Fm = sFb + jh * B * F;
#pragma unroll 4
        for (int k = nbasis(face_degree(f2r)); k < B; ++k) {
          const float2 x01 = *reinterpret_cast<const float2*>(X + k * XR);
          const float2 x23 = *reinterpret_cast<const float2*>(X + k * XR + 2);
          const float2 x45 = *reinterpret_cast<const float2*>(X + k * XR + 4);
          const float2 x67 = *reinterpret_cast<const float2*>(X + k * XR + 6);
          const float xs[9] = {x01.x, x01.y, x23.x, x23.y, x45.x, x45.y, x67.x, x67.y, X[k * XR + 8]};
          const float w1 = Fm[k * F + f1], w2 = Fm[k * F + f2r];
#pragma unroll
          for (int r = 0; r < 9; ++r) {
            g1[r] = fmaf(xs[r], w1, g1[r]);
            g2[r] = fmaf(xs[r], w2, g2[r]);
          }
        }
      }
      const float* fd = sD + eel * ND + 4 + 11 * i;
      float* fl = sFl + ee * C::FLSN + i * F * FR;
      float w6[6];
      riemann_state(g1, fd, w6);
      store_state(fl + f1 * FR, w6);
      if (f2 >= 0) {
        riemann_state(g2, fd, w6);
        store_state(fl + f2 * FR, w6);
      }
    }
    __syncthreads();
    if (valid) {
      constexpr int NS = (M > 0) ? 15 : 9;
      constexpr int NQ = C::NQ;
      // the DOF loads are issued first so their latency overlaps the F^ product
      float* q = st.Q + (size_t)g * qs + (size_t)grp * (C::NQ * B * FG) + b * FG + j;
      float qv[NQ];
#pragma unroll
      for (int r = 0; r < NQ; ++r) qv[r] = q[r * rs];
      float S[NS];
#pragma unroll
      for (int r = 0; r < NS; ++r) S[r] = 0.f;
      const float* nd = sD + eb * ND;
      project_faces<NS, F, B, FR>(sFl + e * C::FLSN, sFh, nd + 4, 11, nd[0], nd[1], nd[2], fmax, b, S);
#pragma unroll
      for (int r = 0; r < 9; ++r) q[r * rs] = qv[r] + S[r];
      if constexpr (M > 0) {
#pragma unroll
        for (int l = 0; l < M; ++l)
#pragma unroll
          for (int r = 0; r < 6; ++r) q[(9 + 6 * l + r) * rs] = qv[9 + 6 * l + r] + ph.omega[l] * S[NS - 6 + r];
      }
    }
  }
}

// ------------------------------------------------------------------ face-local messages
// Sender side of a partitioned run (Sec. V-C): for every cut face whose receiving element is
// active in this phase, H = X F-_{j,h} (9 x F values) from the sending element's buffer X,
// chosen by the cluster relation exactly as k_neighbour chooses it (B1, B3, B2 or B1 - B2 by
// the receiver's step parity), with the same product order, so the receiver's flux sees the
// values it would have computed itself. One thread per (cut face, face mode).
template <int O, int M>
__global__ void k_pack_faces(DevOps ops, DevState st, PhaseArgs ph, const int* send_elem, const int* send_code,
                             const int* recv_cluster, int n, int fg, float* msg) {
  using C = Cfg<O, M>;
  constexpr int B = C::B, F = C::F;
  const int nsim = st.nsim;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nsim * F) return;
  const int c = t / (nsim * F), sim = (t / F) % nsim, f = t % F;
  int pf = 0;
  while (nface(pf + 1) <= f) ++pf;
  const int code = send_code[c];
  const int jh = code & 0xff, rel = (code >> 8) & 0xff;
  const int par = ph.parity[recv_cluster[c]];
  const float* src1 = (rel == 1) ? st.B3 : ((rel == 2 && par == 0) ? st.B2 : st.B1);
  const bool sub = (rel == 2 && par == 1);
  // simulation sim's rows in the sender's buffer (groups of fg simulations, innermost)
  const size_t off = (size_t)send_elem[c] * st.bs + (size_t)(sim / fg) * (9 * B * fg) + sim % fg;
  const float* Fm = ops.Fb + jh * B * F + f;
  float gq[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) gq[r] = 0.f;
#pragma unroll 4
  for (int k = nbasis(pf); k < B; ++k) {
    const float w = Fm[k * F];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
      float x = __ldg(src1 + off + (size_t)(r * B + k) * fg);
      if (sub) x -= __ldg(st.B2 + off + (size_t)(r * B + k) * fg);
      gq[r] = fmaf(x, w, gq[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < 9; ++r) msg[(((size_t)c * nsim + sim) * 9 + r) * F + f] = gq[r];
}

// ------------------------------------------------------------------ receivers
struct RecvItem {
  int elem;        // internal element index
  int sim;         // simulation (fused mode), else 0
  int phi_off;     // offset of phi values (B floats) in recv_phi
  int out_off;     // first output sample slot
  int n;           // samples in this step (<= 8)
  float tau[8];    // t_j - t_n
};

// One CTA per receiver item, one thread per mode column; recomputes the element's time
// derivatives from Q (full state at the start of its step) and evaluates
// sum_d tau^d/d! (d^dQ) phi(xi_r) for the 9 elastic quantities.
template <int O, int M>
__global__ void k_receivers(DevOps ops, const float* Q, long long qs, int nsim, int fg, const float* edata,
                            const float* recv_phi, const RecvItem* items, float* out, float om0, float om1,
                            float om2) {
  using C = Cfg<O, M>;
  constexpr int B = C::B, NQ = C::NQ;
  __shared__ float sA[B * 9];
  __shared__ float sRed[8][9][2];
  const RecvItem it = items[blockIdx.x];
  const int b = threadIdx.x;
  const float om[3] = {om0, om1, om2};
  const float* ed = edata + (size_t)it.elem * ED;
  float D[NQ];
  float acc[8][9];
  const float phi = (b < B) ? recv_phi[it.phi_off + b] : 0.f;
#pragma unroll
  for (int r = 0; r < NQ; ++r)
    D[r] = (b < B) ? Q[(size_t)it.elem * qs + (size_t)(it.sim / fg) * NQ * B * fg + (r * B + b) * fg + it.sim % fg]
                   : 0.f;
#pragma unroll
  for (int s = 0; s < 8; ++s)
#pragma unroll
    for (int r = 0; r < 9; ++r) acc[s][r] = 0.f;
  float w[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) w[s] = 1.f;   // tau^d / d!
#pragma unroll 1
  for (int d = 0; d < O; ++d) {
#pragma unroll
    for (int s = 0; s < 8; ++s)
#pragma unroll
      for (int r = 0; r < 9; ++r) acc[s][r] = fmaf(w[s], D[r] * phi, acc[s][r]);
#pragma unroll
    for (int s = 0; s < 8; ++s) w[s] *= it.tau[s] / (float)(d + 1);
    if (d == O - 1) break;
    __syncthreads();
    if (b < B) {
#pragma unroll
      for (int r = 0; r < 9; ++r) sA[b * 9 + r] = D[r];
    }
    __syncthreads();
    if (b < B) {
      float Y[3][9];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 9; ++r) Y[c][r] = 0.f;
      for (int k = 0; k < B; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float kc = ops.K[(c * B + b) * B + k];
#pragma unroll
          for (int r = 0; r < 9; ++r) Y[c][r] = fmaf(sA[k * 9 + r], kc, Y[c][r]);
        }
      float outv[9], eps[6];
      star_apply(Y, ed, outv, eps);
      if constexpr (M > 0) {
#pragma unroll
        for (int l = 0; l < M; ++l) coupling_add(outv, D + 9 + 6 * l, ed[12 + 2 * l], ed[13 + 2 * l]);
#pragma unroll
        for (int l = 0; l < M; ++l)
#pragma unroll
          for (int r = 0; r < 6; ++r) D[9 + 6 * l + r] = om[l] * (eps[r] - D[9 + 6 * l + r]);
      }
#pragma unroll
      for (int r = 0; r < 9; ++r) D[r] = outv[r];
    }
  }
  // reduce over the mode columns (blockDim.x <= 64)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < 8; ++s)
#pragma unroll
    for (int r = 0; r < 9; ++r) {
      float v = acc[s][r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) sRed[s][r][warp] = v;
    }
  __syncthreads();
  // 9 n values (up to 72) written by a block of 32 or 64 threads
  for (int i = threadIdx.x; i < 9 * it.n; i += blockDim.x) {
    const int s = i / 9, r = i % 9;
    float v = sRed[s][r][0];
    if (blockDim.x > 32) v += sRed[s][r][1];
    out[((size_t)(it.out_off + s) * nsim + it.sim) * 9 + r] = v;
  }
}

// ------------------------------------------------------------------ sources
struct SrcItem {
  int elem;
  int sim;         // simulation (fused mode), else 0
  int phi_off;
  float amp[6];    // -m0 m6 (int s dt) / |det J|
};

template <int O, int M>
__global__ void k_sources(float* Q, long long qs, int fg, const float* src_phi, const SrcItem* items, int n) {
  using C = Cfg<O, M>;
  constexpr int B = C::B, NQ = C::NQ;
  for (int s = 0; s < n; ++s) {
    const SrcItem it = items[s];
    for (int i = threadIdx.x; i < 6 * B; i += blockDim.x) {
      const int r = i / B, b = i % B;
      Q[(size_t)it.elem * qs + (size_t)(it.sim / fg) * NQ * B * fg + (r * B + b) * fg + it.sim % fg] +=
          it.amp[r] * src_phi[it.phi_off + b];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ energy
// sum_k |det J_k| sum_b (rho |v_b|^2 / 2 + sigma_b : C^-1 sigma_b / 2), FP64, summed over
// all simulations; one partial sum per block (blockDim.x = 256).
template <int O, int M>
__global__ void k_energy(const float* Q, long long qs, int nsim, int fg, const double* emat, int K,
                         double* partial) {
  using C = Cfg<O, M>;
  constexpr int B = C::B, NQ = C::NQ;
  double local = 0.0;
  const size_t per = (size_t)B * nsim;
  const size_t rs = (size_t)B * fg;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)K * per; i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i / per);
    const int bf = (int)(i % per);               // (group, mode, simulation in group)
    const int grp = bf / (B * fg), rem = bf % (B * fg);
    const float* q = Q + (size_t)k * qs + (size_t)grp * NQ * B * fg + rem;
    const double* em = emat + (size_t)k * 4;     // lam, mu, rho, |det J|
    const double lam = em[0], mu = em[1], rho = em[2];
    double s[6], v[3];
    for (int r = 0; r < 6; ++r) s[r] = q[r * rs];
    for (int r = 0; r < 3; ++r) v[r] = q[(6 + r) * rs];
    const double tr = s[0] + s[1] + s[2];
    const double ss = s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + 2.0 * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
    const double pot = 0.5 * (ss / (2.0 * mu) - lam / (2.0 * mu * (3.0 * lam + 2.0 * mu)) * tr * tr);
    const double kin = 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    local += em[3] * (kin + pot);
  }
  __shared__ double red[256];
  red[threadIdx.x] = local;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

}  // namespace ltsdev
