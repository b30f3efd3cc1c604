// k_adj_pred_sp: the reverse of a predict pass of the clustered-LTS adjoint (elastic, one or
// fused simulations) with the operator products in generated sparse form, the counterpart of
// k_predict_sp for the transposed scheme. The arithmetic is that of k_adj_pred (see there
// and kernels_adj.cuh for the derivation); only the organisation differs:
//   row phase:    thread = (part, pair), pair = (element e, quantity row r); the thread keeps
//                 one row of its operand in registers and forms one part of the generated
//                 products with the nonzero entries of K_c and F~_i as immediate operands
//                 (sparse_ops.cuh): the time kernel D_d K_c^T (forward recomputation, and
//                 V_c = lambda K_c^T), the face traces lambda F~_i and T F~_i (F^_i = F~_i^T in
//                 the orthonormal face basis), the summed transposed traces sum_i U_i F~_i^T
//                 and the reverse time kernel Z_c = G_{d+1} K_c on the support of level d;
//   column phase: thread = (element e, mode b): star matrices (S_c, S_c^T, compact), Taylor
//                 weights, the buffer adjoints, and the next row operand;
//   face phase:   thread = (element, face, face mode): U_i = A-_i^T (lambda F~_i);
//   correlations: thread = (element, 3 x 3 tile): W_c and W-_i over the modes (face modes),
//                 the batch's W_c summed in shared memory and added to the FP64 totals once.
// Staging arrays are [mode or output][pair] with an odd pair stride XP, as in k_predict_sp.
#pragma once
#include "kernels_adj.cuh"
#include "sparse_ops.cuh"

namespace ltsdev {

// elements per CTA and parts of the row phase (NT = rup(9 NE, 32) NPART threads, NE B <= NT)
template <int O>
struct AdjSpShape;
template <>
struct AdjSpShape<5> {
  static constexpr int NE = 7, NPART = 4;
};
template <>
struct AdjSpShape<4> {
  static constexpr int NE = 12, NPART = 2;
};
template <>
struct AdjSpShape<3> {
  static constexpr int NE = 12, NPART = 1;
};

// rows of D_0 .. D_{d-1}, D_j kept on its nbasis(O - j) modes
__host__ __device__ constexpr int adj_drow(int O, int d) {
  int r = 0;
  for (int j = 0; j < d; ++j) r += nbasis(O - j);
  return r;
}

template <int O>
struct AdjSpCfg {
  static constexpr int B = nbasis(O), F = nface(O);
  static constexpr int NE = AdjSpShape<O>::NE, NPART = AdjSpShape<O>::NPART;
  static constexpr int NPAIR = 9 * NE;
  static constexpr int RT = rup(NPAIR, 32);
  static constexpr int NT = RT * NPART;
  static_assert(NE * B <= NT, "column phase needs one thread per (element, mode)");
  static constexpr int XP = NPAIR | 1;                      // odd pair stride
  static constexpr int DROWS = adj_drow(O, O - 1);          // D_0 .. D_{O-2}
  static constexpr int WROWS = (3 * B > 8 * F) ? 3 * B : 8 * F;
  static constexpr int S_X = 0;                             // [B] row operand
  static constexpr int S_T = S_X + B * XP;                  // [B] T
  static constexpr int S_D = S_T + B * XP;                  // [DROWS] D_d
  static constexpr int S_W = S_D + DROWS * XP;              // [3B] Y_c, V_c, Z_c or [8F] LF_i (U_i), TF_i
  static constexpr int S_STAR = rup(S_W + WROWS * XP, 4);   // [NE][3][36] compact S_c
  static constexpr int S_AL = S_STAR + NE * 108;            // [NE][4][9][12] A-_i, rows padded to 12
  static constexpr int S_WC = S_AL + NE * 432;              // [NE][243] W_c of the batch
  static constexpr int S_META = S_WC + NE * 243;            // [NE] ints
  static constexpr int TOTAL = rup(S_META + NE, 4);
};

template <int O, int XP>
__device__ __forceinline__ void sp_trace(int part, const float* x, float* g) {
  if constexpr (O == 5) ltssp::sp_trace_o5<XP>(part, x, g);
  if constexpr (O == 4) ltssp::sp_trace_o4<XP>(part, x, g);
  if constexpr (O == 3) ltssp::sp_trace_o3<XP>(part, x, g);
}
template <int O, int XP>
__device__ __forceinline__ void sp_tproj(int part, const float* x, float* y) {
  if constexpr (O == 5) ltssp::sp_tproj_o5<XP>(part, x, y);
  if constexpr (O == 4) ltssp::sp_tproj_o4<XP>(part, x, y);
  if constexpr (O == 3) ltssp::sp_tproj_o3<XP>(part, x, y);
}
template <int O, int XP>
__device__ __forceinline__ void sp_kvol(int part, int variant, const float* x, float* y) {
  if constexpr (O == 5) ltssp::sp_kvol_o5<XP>(part, variant, x, y);
  if constexpr (O == 4) ltssp::sp_kvol_o4<XP>(part, variant, x, y);
  if constexpr (O == 3) ltssp::sp_kvol_o3<XP>(part, variant, x, y);
}
template <int O, int XP>
__device__ __forceinline__ void sp_time_adj(int part, int variant, const float* x, float* y) {
  if constexpr (O == 5) ltssp::sp_time_o5<XP>(part, variant, x, y);
  if constexpr (O == 4) ltssp::sp_time_o4<XP>(part, variant, x, y);
  if constexpr (O == 3) ltssp::sp_time_o3<XP>(part, variant, x, y);
}

// Star correlations of a batch: W_c[r][s] (+/-)= sum_{b0 <= b < n} X[(c B + b) XP + 9 e + r]
// Y[(y0 + b) XP + 9 e + s], one 3 x 3 tile (element, c, row block, column block) per task,
// accumulated into the batch's W_c in shared memory (one writer per entry).
template <int B, int XP, int NE, int NT>
__device__ __forceinline__ void star_corr(const float* X, const float* Y, int y0, int b0, int n, bool sub, float* sWc,
                                          int tid) {
  for (int j = tid; j < 27 * NE; j += NT) {
    const int e = j / 27, c = (j / 9) % 3, rb = (j / 3) % 3, sb = j % 3;
    float acc[3][3];
    float* w = sWc + e * 243 + c * 81 + (3 * rb) * 9 + 3 * sb;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int q = 0; q < 3; ++q) acc[i][q] = sub ? 0.f : w[i * 9 + q];
    const float* x = X + c * B * XP + 9 * e + 3 * rb;
    const float* y = Y + y0 * XP + 9 * e + 3 * sb;
    for (int b = b0; b < n; ++b) {
      float xv[3], yv[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        xv[i] = x[b * XP + i];
        yv[i] = y[b * XP + i];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int q = 0; q < 3; ++q) acc[i][q] = fmaf(xv[i], yv[q], acc[i][q]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int q = 0; q < 3; ++q) w[i * 9 + q] = sub ? w[i * 9 + q] - acc[i][q] : acc[i][q];
  }
}

template <int O>
__global__ void __launch_bounds__(AdjSpCfg<O>::NT, 2) k_adj_pred_sp(AdjLtsArgs a, PhaseArgs ph) {
  using S = AdjSpCfg<O>;
  constexpr int B = S::B, F = S::F, NE = S::NE, NT = S::NT, XP = S::XP;
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  float* sX = smem + S::S_X;
  float* sT = smem + S::S_T;
  float* sD = smem + S::S_D;
  float* sW = smem + S::S_W;
  float* sStar = smem + S::S_STAR;
  float* sAl = smem + S::S_AL;
  float* sWc = smem + S::S_WC;
  int* sMeta = reinterpret_cast<int*>(smem + S::S_META);
  const int tid = threadIdx.x;
  // column task (element, mode), modes fastest
  const bool act = tid < NE * B;
  const int es = act ? tid / B : 0, b = act ? tid % B : 0;
  const int col = 9 * es;
  // row task (part, pair): warp w takes part w mod NPART, as in k_predict_sp
  const int part = (tid >> 5) % S::NPART, pair = ((tid >> 5) / S::NPART) * 32 + (tid & 31);
  const bool ract = pair < S::NPAIR;
  const int nbatch = (a.end + NE - 1) / NE;

  for (int batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int k0 = batch * NE;
    __syncthreads();   // the previous batch is done with shared memory
    const int k = k0 + es;
    const bool valid = act && k < a.end;
    // the batch's star matrices (compact), A-_i (rows padded), and zero star correlations
    if (tid < NE) sMeta[tid] = (k0 + tid < a.end) ? a.meta[k0 + tid] : 0;
    for (int q = tid; q < NE * 108; q += NT) {
      const int e = q / 108, x = q % 108;
      sStar[q] = (k0 + e < a.end)
                     ? __ldg(a.amat + (size_t)(k0 + e) * AM_SIZE + AM_STAR + (x / 36) * 81 + star_compact_index(x % 36))
                     : 0.f;
    }
    for (int q = tid; q < NE * 324; q += NT) {
      const int e = q / 324, x = q % 324;
      sAl[e * 432 + (x / 9) * 12 + x % 9] = (k0 + e < a.end) ? __ldg(a.amat + (size_t)(k0 + e) * AM_SIZE + AM_LOC + x) : 0.f;
    }
    for (int q = tid; q < NE * 243; q += NT) sWc[q] = 0.f;
    const int meta = valid ? a.meta[k] : 0;
    const int cl = meta & 0xff;
    // fused runs take the simulations of the batch in turn: the operator matrices are staged
    // once, W_c sums over the simulations (in order) and W-_i receives one addition per
    // simulation, in order
    for (int sim = 0; sim < a.nsim; ++sim) {
      // this simulation's adjoints [element][simulation][9][B]
      const size_t ao = ((size_t)k * a.nsim + sim) * (9 * B) + b;
      // D_0 = Q before the pass (this column; simulation-blocked state, groups of G)
      float T[9];
      {
        float v[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) v[r] = 0.f;
        if (valid) {
          const float* q = a.Qs + (size_t)k * a.qs + (size_t)(sim / a.G) * (9 * B * a.G) + sim % a.G + (size_t)b * a.G;
#pragma unroll
          for (int r = 0; r < 9; ++r) v[r] = __ldg(q + (size_t)r * B * a.G);
        }
        if (act) {
#pragma unroll
          for (int r = 0; r < 9; ++r) {
            sX[b * XP + col + r] = v[r];
            sD[b * XP + col + r] = v[r];
            T[r] = ph.coef[cl][0] * v[r];
          }
        }
      }
      __syncthreads();
      if (sim == 0) {
        // the next batch's inputs into L2 while this batch computes: operator matrices, Q,
        // lambda and lambda_B1 of every simulation (128-byte lines)
        const int kn = k0 + gridDim.x * NE;
        if (kn < a.end) {
          const int nn = min(NE, a.end - kn);
          const long long la = (long long)nn * AM_SIZE, lqn = (long long)nn * a.nsim * 9 * B, lQ = (long long)nn * a.qs;
          const float* pa = a.amat + (size_t)kn * AM_SIZE;
          const float* pq = a.Qs + (size_t)kn * a.qs;
          const float* pl = a.lq + (size_t)kn * a.nsim * 9 * B;
          const float* pb = a.lb1 + (size_t)kn * a.nsim * 9 * B;
          for (long long off = 32LL * tid; off < la; off += 32LL * NT) asm volatile("prefetch.global.L2 [%0];" ::"l"(pa + off));
          for (long long off = 32LL * tid; off < lQ; off += 32LL * NT) asm volatile("prefetch.global.L2 [%0];" ::"l"(pq + off));
          for (long long off = 32LL * tid; off < lqn; off += 32LL * NT) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(pl + off));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(pb + off));
          }
        }
      }
      const float* Sk = sStar + es * 108;
      // ---- forward time kernel: D_{d+1} = sum_c S_c D_d K_c^T (variant d: D_d on nbasis(O - d)
      // modes, D_{d+1} on nbasis(O - 1 - d))
#pragma unroll 1
      for (int d = 0; d < O - 1; ++d) {
        if (ract) sp_time_adj<O, XP>(part, d, sX + pair, sW + pair);
        __syncthreads();
        const int nout = nbasis(O - 1 - d);
        if (act) {
          float v[9];
#pragma unroll
          for (int r = 0; r < 9; ++r) v[r] = 0.f;
          if (b < nout) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              float y[9];
#pragma unroll
              for (int s = 0; s < 9; ++s) y[s] = sW[(c * B + b) * XP + col + s];
              star_acc<false>(Sk + c * 36, y, v);
            }
          }
          const float c1 = ph.coef[cl][d + 1];
#pragma unroll
          for (int r = 0; r < 9; ++r) {
            T[r] = fmaf(c1, v[r], T[r]);
            sX[b * XP + col + r] = v[r];
          }
          if (d + 1 <= O - 2 && b < nout) {
            float* dp = sD + (adj_drow(O, d + 1) + b) * XP + col;
#pragma unroll
            for (int r = 0; r < 9; ++r) dp[r] = v[r];
          }
        }
        __syncthreads();
      }
      // ---- volume: V_c = lambda K_c^T (on nbasis(O - 1) modes), mu = -sum_c S_c^T V_c,
      // W_c -= V_c T^T
      float lam[9], mu[9], muh[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) lam[r] = 0.f;
      if (valid) {
        const float* lp = a.lq + ao;
#pragma unroll
        for (int r = 0; r < 9; ++r) lam[r] = lp[r * B];
      }
      if (act) {
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          sX[b * XP + col + r] = lam[r];
          sT[b * XP + col + r] = T[r];
        }
      }
      __syncthreads();
      if (ract) sp_time_adj<O, XP>(part, 0, sX + pair, sW + pair);
      __syncthreads();
      constexpr int NV = nbasis(O - 1);
      {
        float w[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) w[r] = 0.f;
        if (act && b < NV) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float v[9];
#pragma unroll
            for (int s = 0; s < 9; ++s) v[s] = sW[(c * B + b) * XP + col + s];
            star_acc<true>(Sk + c * 36, v, w);
          }
        }
#pragma unroll
        for (int r = 0; r < 9; ++r) mu[r] = -w[r];
      }
      star_corr<B, XP, NE, NT>(sW, sT, 0, 0, NV, true, sWc, tid);
      __syncthreads();
      // ---- local surface: LF_i = lambda F~_i and TF_i = T F~_i (row phase)
      if (ract) {
        sp_trace<O, XP>(part, sX + pair, sW + pair);
        sp_trace<O, XP>(part, sT + pair, sW + 4 * F * XP + pair);
      }
      __syncthreads();
      // W-_i += LF_i TF_i^T: one writer per entry (the simulations in turn)
      for (int j = tid; j < 36 * NE; j += NT) {
        const int e = j / 36, i = (j / 9) % 4, rb = (j / 3) % 3, sb = j % 3;
        float acc[3][3];
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
#pragma unroll
          for (int q = 0; q < 3; ++q) acc[ii][q] = 0.f;
        const float* x = sW + i * F * XP + 9 * e + 3 * rb;
        const float* y = sW + (4 + i) * F * XP + 9 * e + 3 * sb;
        for (int f = 0; f < F; ++f) {
          float xv[3], yv[3];
#pragma unroll
          for (int ii = 0; ii < 3; ++ii) {
            xv[ii] = x[f * XP + ii];
            yv[ii] = y[f * XP + ii];
          }
#pragma unroll
          for (int ii = 0; ii < 3; ++ii)
#pragma unroll
            for (int q = 0; q < 3; ++q) acc[ii][q] = fmaf(xv[ii], yv[q], acc[ii][q]);
        }
        if (k0 + e < a.end) {
          double* Wk = a.W + (size_t)(k0 + e) * AM_SIZE + AM_LOC + i * 81 + (3 * rb) * 9 + 3 * sb;
#pragma unroll
          for (int ii = 0; ii < 3; ++ii)
#pragma unroll
            for (int q = 0; q < 3; ++q) atomicAdd(Wk + ii * 9 + q, (double)acc[ii][q]);
        }
      }
      __syncthreads();
      // U_i = A-_i^T LF_i per (element, face, face mode), over LF_i
      for (int j = tid; j < NE * 4 * F; j += NT) {
        const int e = j / (4 * F), i = (j / F) % 4, f = j % F;
        float* lp = sW + (i * F + f) * XP + 9 * e;
        float lf[9], u[9];
#pragma unroll
        for (int s = 0; s < 9; ++s) {
          lf[s] = lp[s];
          u[s] = 0.f;
        }
        const float* Am = sAl + e * 432 + i * 108;
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
#pragma unroll
        for (int r = 0; r < 9; ++r) lp[r] = u[r];
      }
      // the adjoints of the buffers this pass wrote: lambda_B1 (+ lambda_B3) join mu,
      // lambda_B2 is mu_half; reset here (lambda_B3 survives an accumulation)
      float l13[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) l13[r] = muh[r] = 0.f;
      if (valid) {
        const bool finer = meta & FLAG_FINER, coarser = meta & FLAG_COARSER;
        const bool even = ph.parity[cl] == 0;
        const size_t o = ao;
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          l13[r] = a.lb1[o + r * B] + (coarser ? a.lb3[o + r * B] : 0.f);
          if (finer) muh[r] = a.lb2[o + r * B];
        }
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          a.lb1[o + r * B] = 0.f;
          if (coarser && even) a.lb3[o + r * B] = 0.f;
          if (finer) a.lb2[o + r * B] = 0.f;
        }
      }
      __syncthreads();
      // mu += sum_i U_i F~_i^T (row phase, into the row operand's place)
      if (ract) sp_tproj<O, XP>(part, sW + pair, sX + pair);
      __syncthreads();
      // ---- reverse time kernel: G_{O-1} = c_{O-1} mu + c'_{O-1} mu_half (over this column's
      // face sum: read and written by the same thread), then G_d = c_d mu + c'_d mu_half +
      // sum_c S_c^T Z_c with Z_c = G_{d+1} K_c, and W_c += Z_c D_d^T
      if (act) {
#pragma unroll
        for (int r = 0; r < 9; ++r) {
          mu[r] += sX[b * XP + col + r];
          mu[r] += l13[r];
          sX[b * XP + col + r] = ph.coef[cl][O - 1] * mu[r] + ph.hcoef[cl][O - 1] * muh[r];
        }
      }
      __syncthreads();
      float g0[9];
#pragma unroll 1
      for (int d = O - 2; d >= 0; --d) {
        if (ract) sp_kvol<O, XP>(part, d, sX + pair, sW + pair);
        __syncthreads();
        const int nout = nbasis(O - d);
        if (act) {
          float gv[9];
#pragma unroll
          for (int r = 0; r < 9; ++r) gv[r] = ph.coef[cl][d] * mu[r] + ph.hcoef[cl][d] * muh[r];
          // Z_c[0] = 0 (not written)
          if (b >= 1 && b < nout) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              float z[9];
#pragma unroll
              for (int r = 0; r < 9; ++r) z[r] = sW[(c * B + b) * XP + col + r];
              star_acc<true>(Sk + c * 36, z, gv);
            }
          }
#pragma unroll
          for (int r = 0; r < 9; ++r) {
            sX[b * XP + col + r] = gv[r];
            g0[r] = gv[r];
          }
        }
        star_corr<B, XP, NE, NT>(sW, sD, adj_drow(O, d), 1, nout, false, sWc, tid);
        __syncthreads();
      }
      if (valid) {
        float* lp = a.lq + ao;
#pragma unroll
        for (int r = 0; r < 9; ++r) lp[r * B] = lam[r] + g0[r];
      }
    }  // simulations
    // the batch's star correlations into the FP64 totals (one addition per entry and pass)
    for (int q = tid; q < NE * 243; q += NT) {
      const int e = q / 243;
      if (k0 + e < a.end) atomicAdd(a.W + (size_t)(k0 + e) * AM_SIZE + AM_STAR + q % 243, (double)sWc[q]);
    }
  }
}

}  // namespace ltsdev
