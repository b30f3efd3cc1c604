// Discrete adjoint of the global-time-stepping loop, elastic equations (one simulation).
//
// One forward step maps Q to Q' = Q + V(T) + S_L(T) + S_N(T of the face neighbours), with
// D_0 = Q, D_{d+1} = sum_c S_c D_d K_c^T (S_c the star matrices of the time kernel),
// T = sum_d c_d D_d, V = -sum_c S_c T K_c, S_L = sum_i A-_i (T F~_i) F^_i and
// S_N = sum_i A+_i (T_{k_i} F-_{j,h}) F^_i (A-_i, A+_i the 9 x 9 flux solvers of face i).
// For the adjoint lambda = dJ/dQ' of one step this file's kernels compute, per element,
//   mu = dJ/dT = -sum_c S_c^T lambda K_c^T + sum_i ((A-_i^T lambda) F^_i^T) F~_i^T
//        + sum over the neighbours k' of ((A+_{k',i'}^T lambda_k') F^_{i'}^T) F-_{i,h'}^T,
//   G_{O-1} = c_{O-1} mu, G_d = c_d mu + sum_c S_c^T G_{d+1} K_c,   dJ/dQ = lambda + G_0,
// and the per-element correlations that the material derivatives of S_c, A-_i, A+_i
// are contracted with once the loop is done:
//   W_c  += sum_{d<O-1} G_{d+1} (D_d K_c^T)^T - lambda (T K_c)^T,
//   W-_i += lambda (T F~_i F^_i)^T,   W+_i += lambda (T_{k_i} F-_{j,h} F^_i)^T.
// The matrices are explicit (FP32, built on the host from the same closed forms as the
// forward kernels' star and flux code); one CTA per element, plain CUDA cores.
#pragma once
#include "kernels.cuh"

namespace ltsdev {

constexpr int AM_STAR = 0;       // S_c, c = 0..2: [out][in]
constexpr int AM_LOC = 243;      // A-_i, i = 0..3
constexpr int AM_NBR = 567;      // A+_i, i = 0..3
constexpr int AM_SIZE = 891;     // floats per element (also the size of the correlations W)

struct AdjArgs {
  const float* Q;        // Q^n, element stride qs, rows of B
  const float* tbuf;     // [K][9B] T of step n
  const float* lam_in;   // [K][9B] lambda^{n+1}
  float* lam_out;        // [K][9B] lambda^n without the misfit's source
  const float* amat;     // [K][AM_SIZE]
  const int* fwd;        // [K][4][2]: neighbour (internal index, -1 none), j*3+h of F- for this face
  const int* back;       // [K][4][2]: the neighbour's face i' pointing here, i*3+h' of its F-
  double* W;             // [K][AM_SIZE]
  long long qs;
  float cd[6];           // dt^(d+1)/(d+1)!
};

// T of every element from Q^n (the time kernel with the explicit star matrices).
template <int O>
__global__ void __launch_bounds__(64) k_adj_T(DevOps ops, AdjArgs a, float* tbuf) {
  constexpr int B = nbasis(O), NB9 = 9 * B;
  __shared__ float sS[243];
  __shared__ float sX[2][NB9];
  const int k = blockIdx.x, t = threadIdx.x;
  for (int i = t; i < 243; i += blockDim.x) sS[i] = a.amat[(size_t)k * AM_SIZE + AM_STAR + i];
  for (int i = t; i < NB9; i += blockDim.x) sX[0][i] = a.Q[(size_t)k * a.qs + i];
  __syncthreads();
  float T[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) T[r] = (t < B) ? a.cd[0] * sX[0][r * B + t] : 0.f;
  int cur = 0;
  for (int d = 0; d < O - 1; ++d) {
    float nxt[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) nxt[r] = 0.f;
    if (t < B) {
      float Y[3][9];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int s = 0; s < 9; ++s) Y[c][s] = 0.f;
      for (int kk = 0; kk < B; ++kk) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float kc = ops.K[(c * B + t) * B + kk];
#pragma unroll
          for (int s = 0; s < 9; ++s) Y[c][s] = fmaf(sX[cur][s * B + kk], kc, Y[c][s]);
        }
      }
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float v = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int s = 0; s < 9; ++s) v = fmaf(sS[c * 81 + r * 9 + s], Y[c][s], v);
        nxt[r] = v;
        T[r] = fmaf(a.cd[d + 1], v, T[r]);
      }
    }
    if (t < B)
#pragma unroll
      for (int r = 0; r < 9; ++r) sX[cur ^ 1][r * B + t] = nxt[r];
    __syncthreads();
    cur ^= 1;
  }
  if (t < B)
#pragma unroll
    for (int r = 0; r < 9; ++r) tbuf[(size_t)k * NB9 + r * B + t] = T[r];
}

// One reverse step for every element (one CTA each): lambda^n and the correlations.
template <int O>
__global__ void __launch_bounds__(128) k_adj_step(DevOps ops, AdjArgs a) {
  constexpr int B = nbasis(O), F = nface(O), NB9 = 9 * B;
  __shared__ float sM[AM_SIZE];
  __shared__ float sAb[4][81];
  __shared__ float sL[NB9], sT[NB9];
  __shared__ float sD[O][NB9], sG[O][NB9];
  __shared__ float sP[3][NB9];
  __shared__ float sU[9 * F];
  __shared__ int sF[8], sBk[8];
  const int k = blockIdx.x, t = threadIdx.x, nt = blockDim.x;
  for (int i = t; i < AM_SIZE; i += nt) sM[i] = a.amat[(size_t)k * AM_SIZE + i];
  if (t < 8) {
    sF[t] = a.fwd[k * 8 + t];
    sBk[t] = a.back[k * 8 + t];
  }
  for (int i = t; i < NB9; i += nt) {
    sL[i] = a.lam_in[(size_t)k * NB9 + i];
    sT[i] = a.tbuf[(size_t)k * NB9 + i];
    sD[0][i] = a.Q[(size_t)k * a.qs + i];
  }
  __syncthreads();
  for (int i = t; i < 4 * 81; i += nt) {
    const int f = i / 81, kn = sF[2 * f];
    sAb[f][i % 81] = (kn >= 0) ? a.amat[(size_t)kn * AM_SIZE + AM_NBR + sBk[2 * f] * 81 + i % 81] : 0.f;
  }
  const float* S = sM + AM_STAR;
  // ---- forward derivatives D_1 .. D_{O-1}
  for (int d = 0; d < O - 1; ++d) {
    if (t < B) {
      float Y[3][9];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int s = 0; s < 9; ++s) Y[c][s] = 0.f;
      for (int kk = 0; kk < B; ++kk)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float kc = ops.K[(c * B + t) * B + kk];
#pragma unroll
          for (int s = 0; s < 9; ++s) Y[c][s] = fmaf(sD[d][s * B + kk], kc, Y[c][s]);
        }
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float v = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int s = 0; s < 9; ++s) v = fmaf(S[c * 81 + r * 9 + s], Y[c][s], v);
        sD[d + 1][r * B + t] = v;
      }
    }
    __syncthreads();
  }
  // ---- mu = dJ/dT: volume term
  float mu[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) mu[r] = 0.f;
  if (t < B)
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float v = 0.f;
#pragma unroll
        for (int s = 0; s < 9; ++s) v = fmaf(S[c * 81 + s * 9 + r], sL[s * B + t], v);
        sP[c][r * B + t] = v;
      }
  __syncthreads();
  if (t < B)
    for (int kk = 0; kk < B; ++kk)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float kc = ops.K[(c * B + t) * B + kk];
#pragma unroll
        for (int r = 0; r < 9; ++r) mu[r] = fmaf(-sP[c][r * B + kk], kc, mu[r]);
      }
  __syncthreads();
  // local surface term, face by face
  for (int i = 0; i < 4; ++i) {
    const float* Am = sM + AM_LOC + i * 81;
    if (t < B)
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float v = 0.f;
#pragma unroll
        for (int s = 0; s < 9; ++s) v = fmaf(Am[s * 9 + r], sL[s * B + t], v);
        sP[0][r * B + t] = v;
      }
    __syncthreads();
    if (t < F)
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float v = 0.f;
        for (int kk = 0; kk < B; ++kk) v = fmaf(sP[0][r * B + kk], ops.Fh[(i * F + t) * B + kk], v);
        sU[r * F + t] = v;
      }
    __syncthreads();
    if (t < B)
      for (int f = 0; f < F; ++f) {
        const float w = ops.Ft[(i * B + t) * F + f];
#pragma unroll
        for (int r = 0; r < 9; ++r) mu[r] = fmaf(sU[r * F + f], w, mu[r]);
      }
    __syncthreads();
  }
  // neighbour surface term: the faces of the neighbours that read this element's T
  for (int i = 0; i < 4; ++i) {
    const int kn = sF[2 * i];
    if (kn < 0) continue;
    for (int q = t; q < NB9; q += nt) sP[1][q] = a.lam_in[(size_t)kn * NB9 + q];
    __syncthreads();
    if (t < B)
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float v = 0.f;
#pragma unroll
        for (int s = 0; s < 9; ++s) v = fmaf(sAb[i][s * 9 + r], sP[1][s * B + t], v);
        sP[0][r * B + t] = v;
      }
    __syncthreads();
    const int ip = sBk[2 * i], jh = sBk[2 * i + 1];
    if (t < F)
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float v = 0.f;
        for (int kk = 0; kk < B; ++kk) v = fmaf(sP[0][r * B + kk], ops.Fh[(ip * F + t) * B + kk], v);
        sU[r * F + t] = v;
      }
    __syncthreads();
    if (t < B)
      for (int f = 0; f < F; ++f) {
        const float w = ops.Fb[(jh * B + t) * F + f];
#pragma unroll
        for (int r = 0; r < 9; ++r) mu[r] = fmaf(sU[r * F + f], w, mu[r]);
      }
    __syncthreads();
  }
  // ---- reverse time kernel: G_{O-1} = c mu, G_d = c_d mu + sum_c S_c^T G_{d+1} K_c
  if (t < B)
#pragma unroll
    for (int r = 0; r < 9; ++r) sG[O - 1][r * B + t] = a.cd[O - 1] * mu[r];
  __syncthreads();
  for (int d = O - 2; d >= 0; --d) {
    if (t < B)
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          float v = 0.f;
#pragma unroll
          for (int s = 0; s < 9; ++s) v = fmaf(S[c * 81 + s * 9 + r], sG[d + 1][s * B + t], v);
          sP[c][r * B + t] = v;
        }
    __syncthreads();
    if (t < B) {
      float g[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) g[r] = a.cd[d] * mu[r];
      for (int kk = 0; kk < B; ++kk)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float kc = ops.K[(c * B + kk) * B + t];
#pragma unroll
          for (int r = 0; r < 9; ++r) g[r] = fmaf(sP[c][r * B + kk], kc, g[r]);
        }
#pragma unroll
      for (int r = 0; r < 9; ++r) sG[d][r * B + t] = g[r];
    }
    __syncthreads();
  }
  if (t < B)
#pragma unroll
    for (int r = 0; r < 9; ++r) a.lam_out[(size_t)k * NB9 + r * B + t] = sL[r * B + t] + sG[0][r * B + t];
  // ---- correlations (thread t < 81 owns entry (rr, ss))
  const int rr = t / 9, ss = t % 9;
  double* Wk = a.W + (size_t)k * AM_SIZE;
  for (int c = 0; c < 3; ++c) {
    double acc = 0.0;
    if (t < B)
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        float v = 0.f;
        for (int kk = 0; kk < B; ++kk) v = fmaf(sT[s * B + kk], ops.K[(c * B + kk) * B + t], v);
        sP[0][s * B + t] = v;
      }
    __syncthreads();
    if (t < 81)
      for (int b = 0; b < B; ++b) acc -= (double)sL[rr * B + b] * (double)sP[0][ss * B + b];
    __syncthreads();
    for (int d = 0; d < O - 1; ++d) {
      if (t < B)
#pragma unroll
        for (int s = 0; s < 9; ++s) {
          float v = 0.f;
          for (int kk = 0; kk < B; ++kk) v = fmaf(sD[d][s * B + kk], ops.K[(c * B + t) * B + kk], v);
          sP[0][s * B + t] = v;
        }
      __syncthreads();
      if (t < 81)
        for (int b = 0; b < B; ++b) acc += (double)sG[d + 1][rr * B + b] * (double)sP[0][ss * B + b];
      __syncthreads();
    }
    if (t < 81) Wk[AM_STAR + c * 81 + t] += acc;
  }
  for (int i = 0; i < 4; ++i) {
    if (t < F)
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        float v = 0.f;
        for (int kk = 0; kk < B; ++kk) v = fmaf(sT[s * B + kk], ops.Ft[(i * B + kk) * F + t], v);
        sU[s * F + t] = v;
      }
    __syncthreads();
    if (t < B)
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        float v = 0.f;
        for (int f = 0; f < F; ++f) v = fmaf(sU[s * F + f], ops.Fh[(i * F + f) * B + t], v);
        sP[0][s * B + t] = v;
      }
    __syncthreads();
    if (t < 81) {
      double acc = 0.0;
      for (int b = 0; b < B; ++b) acc += (double)sL[rr * B + b] * (double)sP[0][ss * B + b];
      Wk[AM_LOC + i * 81 + t] += acc;
    }
    __syncthreads();
  }
  for (int i = 0; i < 4; ++i) {
    const int kn = sF[2 * i];
    if (kn < 0) continue;
    const int jh = sF[2 * i + 1];
    for (int q = t; q < NB9; q += nt) sP[1][q] = a.tbuf[(size_t)kn * NB9 + q];
    __syncthreads();
    if (t < F)
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        float v = 0.f;
        for (int kk = 0; kk < B; ++kk) v = fmaf(sP[1][s * B + kk], ops.Fb[(jh * B + kk) * F + t], v);
        sU[s * F + t] = v;
      }
    __syncthreads();
    if (t < B)
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        float v = 0.f;
        for (int f = 0; f < F; ++f) v = fmaf(sU[s * F + f], ops.Fh[(i * F + f) * B + t], v);
        sP[0][s * B + t] = v;
      }
    __syncthreads();
    if (t < 81) {
      double acc = 0.0;
      for (int b = 0; b < B; ++b) acc += (double)sL[rr * B + b] * (double)sP[0][ss * B + b];
      Wk[AM_NBR + i * 81 + t] += acc;
    }
    __syncthreads();
  }
}

// Velocity at the receivers from Q^n: out[r][q] = sum_b Q[elem_r][6+q][b] phi_r[b].
template <int O>
__global__ void k_adj_sample(const float* Q, long long qs, const int* elem, const float* phi, int nrec, float* out) {
  constexpr int B = nbasis(O);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * nrec) return;
  const int r = t / 3, q = t % 3;
  const float* row = Q + (size_t)elem[r] * qs + (6 + q) * B;
  float v = 0.f;
  for (int b = 0; b < B; ++b) v = fmaf(row[b], phi[r * B + b], v);
  out[t] = v;
}

// The misfit's source: lambda[elem_r][6+q][b] += res[r][q] phi_r[b] (receivers in order, so
// receivers that share an element add in a fixed order).
template <int O>
__global__ void k_adj_source(float* lam, const int* elem, const float* phi, const float* res, int nrec) {
  constexpr int B = nbasis(O);
  const int b = threadIdx.x;
  if (b >= B) return;
  for (int r = 0; r < nrec; ++r)
    for (int q = 0; q < 3; ++q) lam[(size_t)elem[r] * 9 * B + (6 + q) * B + b] += res[r * 3 + q] * phi[r * B + b];
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
  double* W;
  long long qs, bufs;
  int end;                            // active elements [0, end)
};

// Reverse of a predict pass, one CTA per active element.
template <int O>
__global__ void __launch_bounds__(128) k_adj_pred(DevOps ops, AdjLtsArgs a, PhaseArgs ph) {
  constexpr int B = nbasis(O), F = nface(O), NB9 = 9 * B;
  __shared__ float sM[AM_SIZE];
  __shared__ float sL[NB9], sT[NB9];
  __shared__ float sD[O][NB9], sG[O][NB9];
  __shared__ float sP[3][NB9];
  __shared__ float sU[9 * F];
  const int k = blockIdx.x, t = threadIdx.x, nt = blockDim.x;
  const int meta = a.meta[k];
  const int cl = meta & 0xff;
  const bool finer = meta & FLAG_FINER, coarser = meta & FLAG_COARSER;
  const bool even = ph.parity[cl] == 0;
  for (int i = t; i < AM_SIZE; i += nt) sM[i] = a.amat[(size_t)k * AM_SIZE + i];
  for (int i = t; i < NB9; i += nt) {
    sL[i] = a.lq[(size_t)k * NB9 + i];
    sD[0][i] = a.Qs[(size_t)k * a.qs + i];
  }
  __syncthreads();
  const float* S = sM + AM_STAR;
  for (int d = 0; d < O - 1; ++d) {
    if (t < B) {
      float Y[3][9];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int s = 0; s < 9; ++s) Y[c][s] = 0.f;
      for (int kk = 0; kk < B; ++kk)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float kc = ops.K[(c * B + t) * B + kk];
#pragma unroll
          for (int s = 0; s < 9; ++s) Y[c][s] = fmaf(sD[d][s * B + kk], kc, Y[c][s]);
        }
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float v = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int s = 0; s < 9; ++s) v = fmaf(S[c * 81 + r * 9 + s], Y[c][s], v);
        sD[d + 1][r * B + t] = v;
      }
    }
    __syncthreads();
  }
  if (t < B)
#pragma unroll
    for (int r = 0; r < 9; ++r) {
      float v = 0.f;
      for (int d = 0; d < O; ++d) v = fmaf(ph.coef[cl][d], sD[d][r * B + t], v);
      sT[r * B + t] = v;
    }
  // mu: volume and local surface terms of this pass, then the buffers it wrote
  float mu[9], muh[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) mu[r] = muh[r] = 0.f;
  if (t < B)
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float v = 0.f;
#pragma unroll
        for (int s = 0; s < 9; ++s) v = fmaf(S[c * 81 + s * 9 + r], sL[s * B + t], v);
        sP[c][r * B + t] = v;
      }
  __syncthreads();
  if (t < B)
    for (int kk = 0; kk < B; ++kk)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float kc = ops.K[(c * B + t) * B + kk];
#pragma unroll
        for (int r = 0; r < 9; ++r) mu[r] = fmaf(-sP[c][r * B + kk], kc, mu[r]);
      }
  __syncthreads();
  for (int i = 0; i < 4; ++i) {
    const float* Am = sM + AM_LOC + i * 81;
    if (t < B)
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float v = 0.f;
#pragma unroll
        for (int s = 0; s < 9; ++s) v = fmaf(Am[s * 9 + r], sL[s * B + t], v);
        sP[0][r * B + t] = v;
      }
    __syncthreads();
    if (t < F)
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float v = 0.f;
        for (int kk = 0; kk < B; ++kk) v = fmaf(sP[0][r * B + kk], ops.Fh[(i * F + t) * B + kk], v);
        sU[r * F + t] = v;
      }
    __syncthreads();
    if (t < B)
      for (int f = 0; f < F; ++f) {
        const float w = ops.Ft[(i * B + t) * F + f];
#pragma unroll
        for (int r = 0; r < 9; ++r) mu[r] = fmaf(sU[r * F + f], w, mu[r]);
      }
    __syncthreads();
  }
  if (t < B) {
    const size_t o = (size_t)k * NB9 + t;
#pragma unroll
    for (int r = 0; r < 9; ++r) {
      mu[r] += a.lb1[o + r * B];
      a.lb1[o + r * B] = 0.f;
      if (coarser) {
        mu[r] += a.lb3[o + r * B];
        if (even) a.lb3[o + r * B] = 0.f;
      }
      if (finer) {
        muh[r] = a.lb2[o + r * B];
        a.lb2[o + r * B] = 0.f;
      }
    }
#pragma unroll
    for (int r = 0; r < 9; ++r) sG[O - 1][r * B + t] = ph.coef[cl][O - 1] * mu[r] + ph.hcoef[cl][O - 1] * muh[r];
  }
  __syncthreads();
  for (int d = O - 2; d >= 0; --d) {
    if (t < B)
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          float v = 0.f;
#pragma unroll
          for (int s = 0; s < 9; ++s) v = fmaf(S[c * 81 + s * 9 + r], sG[d + 1][s * B + t], v);
          sP[c][r * B + t] = v;
        }
    __syncthreads();
    if (t < B) {
      float g[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) g[r] = ph.coef[cl][d] * mu[r] + ph.hcoef[cl][d] * muh[r];
      for (int kk = 0; kk < B; ++kk)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float kc = ops.K[(c * B + kk) * B + t];
#pragma unroll
          for (int r = 0; r < 9; ++r) g[r] = fmaf(sP[c][r * B + kk], kc, g[r]);
        }
#pragma unroll
      for (int r = 0; r < 9; ++r) sG[d][r * B + t] = g[r];
    }
    __syncthreads();
  }
  if (t < B)
#pragma unroll
    for (int r = 0; r < 9; ++r) a.lq[(size_t)k * NB9 + r * B + t] = sL[r * B + t] + sG[0][r * B + t];
  // correlations of the star matrices and of the local flux solvers
  const int rr = t / 9, ss = t % 9;
  double* Wk = a.W + (size_t)k * AM_SIZE;
  for (int c = 0; c < 3; ++c) {
    double acc = 0.0;
    if (t < B)
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        float v = 0.f;
        for (int kk = 0; kk < B; ++kk) v = fmaf(sT[s * B + kk], ops.K[(c * B + kk) * B + t], v);
        sP[0][s * B + t] = v;
      }
    __syncthreads();
    if (t < 81)
      for (int b = 0; b < B; ++b) acc -= (double)sL[rr * B + b] * (double)sP[0][ss * B + b];
    __syncthreads();
    for (int d = 0; d < O - 1; ++d) {
      if (t < B)
#pragma unroll
        for (int s = 0; s < 9; ++s) {
          float v = 0.f;
          for (int kk = 0; kk < B; ++kk) v = fmaf(sD[d][s * B + kk], ops.K[(c * B + t) * B + kk], v);
          sP[0][s * B + t] = v;
        }
      __syncthreads();
      if (t < 81)
        for (int b = 0; b < B; ++b) acc += (double)sG[d + 1][rr * B + b] * (double)sP[0][ss * B + b];
      __syncthreads();
    }
    if (t < 81) Wk[AM_STAR + c * 81 + t] += acc;
  }
  for (int i = 0; i < 4; ++i) {
    if (t < F)
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        float v = 0.f;
        for (int kk = 0; kk < B; ++kk) v = fmaf(sT[s * B + kk], ops.Ft[(i * B + kk) * F + t], v);
        sU[s * F + t] = v;
      }
    __syncthreads();
    if (t < B)
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        float v = 0.f;
        for (int f = 0; f < F; ++f) v = fmaf(sU[s * F + f], ops.Fh[(i * F + f) * B + t], v);
        sP[0][s * B + t] = v;
      }
    __syncthreads();
    if (t < 81) {
      double acc = 0.0;
      for (int b = 0; b < B; ++b) acc += (double)sL[rr * B + b] * (double)sP[0][ss * B + b];
      Wk[AM_LOC + i * 81 + t] += acc;
    }
    __syncthreads();
  }
}

// Reverse of a neighbour pass, one CTA per buffer owner (every element): for each face
// whose neighbour (the receiver) was active, the receiver's transposed flux goes to the
// adjoint of the buffer it read, and the receiver's correlation with that buffer is
// accumulated. Every (receiver, face) pair is visited by exactly one owner.
template <int O>
__global__ void __launch_bounds__(128) k_adj_nbr(DevOps ops, AdjLtsArgs a, PhaseArgs ph) {
  constexpr int B = nbasis(O), F = nface(O), NB9 = 9 * B;
  __shared__ float sA[81];
  __shared__ float sLk[NB9], sX[NB9], sR[NB9];
  __shared__ float sU[9 * F];
  __shared__ int sF[8], sBk[8];
  const int kn = blockIdx.x, t = threadIdx.x, nt = blockDim.x;
  if (t < 8) {
    sF[t] = a.fwd[kn * 8 + t];
    sBk[t] = a.back[kn * 8 + t];
  }
  __syncthreads();
  const int lo = a.meta[kn] & 0xff;
  for (int i = 0; i < 4; ++i) {
    const int k = sF[2 * i];
    if (k < 0 || k >= a.end) continue;
    const int lr = a.meta[k] & 0xff;
    const int par = ph.parity[lr];
    const int ip = sBk[2 * i], jh = sBk[2 * i + 1];
    for (int q = t; q < 81; q += nt) sA[q] = a.amat[(size_t)k * AM_SIZE + AM_NBR + ip * 81 + q];
    for (int q = t; q < NB9; q += nt) {
      sLk[q] = a.lq[(size_t)k * NB9 + q];
      const size_t o = (size_t)kn * a.bufs + q;
      float x;
      if (lo == lr - 1) x = a.B3s[o];
      else if (lo == lr + 1) x = (par == 0) ? a.B2s[o] : a.B1s[o] - a.B2s[o];
      else x = a.B1s[o];
      sX[q] = x;
    }
    __syncthreads();
    if (t < B)
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float v = 0.f;
#pragma unroll
        for (int s = 0; s < 9; ++s) v = fmaf(sA[s * 9 + r], sLk[s * B + t], v);
        sR[r * B + t] = v;
      }
    __syncthreads();
    if (t < F)
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float v = 0.f;
        for (int kk = 0; kk < B; ++kk) v = fmaf(sR[r * B + kk], ops.Fh[(ip * F + t) * B + kk], v);
        sU[r * F + t] = v;
      }
    __syncthreads();
    if (t < B) {
      const size_t o = (size_t)kn * NB9 + t;
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        float y = 0.f;
        for (int f = 0; f < F; ++f) y = fmaf(sU[r * F + f], ops.Fb[(jh * B + t) * F + f], y);
        if (lo == lr - 1) {
          a.lb3[o + r * B] += y;
        } else if (lo == lr + 1) {
          if (par == 0) {
            a.lb2[o + r * B] += y;
          } else {
            a.lb1[o + r * B] += y;
            a.lb2[o + r * B] -= y;
          }
        } else {
          a.lb1[o + r * B] += y;
        }
      }
    }
    __syncthreads();
    // correlation of the receiver's neighbour flux solver: lambda_Q_k (X F-_{jh} F^_ip)^T
    if (t < F)
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        float v = 0.f;
        for (int kk = 0; kk < B; ++kk) v = fmaf(sX[s * B + kk], ops.Fb[(jh * B + kk) * F + t], v);
        sU[s * F + t] = v;
      }
    __syncthreads();
    if (t < B)
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        float v = 0.f;
        for (int f = 0; f < F; ++f) v = fmaf(sU[s * F + f], ops.Fh[(ip * F + f) * B + t], v);
        sR[s * B + t] = v;
      }
    __syncthreads();
    if (t < 81) {
      const int rr = t / 9, ss = t % 9;
      double acc = 0.0;
      for (int b = 0; b < B; ++b) acc += (double)sLk[rr * B + b] * (double)sR[ss * B + b];
      a.W[(size_t)k * AM_SIZE + AM_NBR + ip * 81 + t] += acc;
    }
    __syncthreads();
  }
}

}  // namespace ltsdev
