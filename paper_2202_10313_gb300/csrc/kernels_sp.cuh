// k_predict_sp: the predict + local kernel (time kernel, LTS buffers, volume kernel, local
// surface kernel; Sec. III-A and Eq. lts_buffers) with the operator products in generated
// sparse form (one simulation).
//
// Each time derivative (and the volume / face-trace step) is done in two phases separated
// by a barrier:
//   row phase:    thread = (part, pair), pair = (element e, quantity row r). The thread
//                 keeps its row X_e[r][0..B) in registers and forms the products of one part
//                 of the outputs with the nonzero operator entries as immediate operands
//                 (sparse_ops.cuh, generated from the reference operators): Y_c[r][b] =
//                 sum_k X[r][k] K_c[b][k] for the time kernel; Z_c[r][b] = sum_k T[r][k]
//                 K_c[k][b] and G_i[r][f] = sum_k T[r][k] F~_i[k][f] for the volume and local
//                 face kernels. No operator entry is read from memory and the structural zeros
//                 of K_c and F~_i (Sec. IV-A "all sparsity") are not multiplied.
//   column phase: thread = (element e, mode b) as in k_predict_local: it reads the 27
//                 products of its column, applies the star matrices (physical form), the
//                 anelastic coupling and relaxation, adds the Taylor terms and writes the
//                 next derivative's column back for the next row phase.
// Shared-memory arrays are [mode or output][pair] with a pair stride XP = 1 mod 32, so the
// row phase's loads and stores (consecutive pairs) and the column phase's accesses
// (consecutive modes) fall on distinct banks.
// The local surface kernel's Riemann states and F^ projection, the receivers, sources and
// neighbour kernel are those of kernels.cuh.
#pragma once
#include "kernels.cuh"
#include "sparse_ops.cuh"

namespace ltsdev {

template <int O>
struct SpShape;
// elements per CTA and parts of the row phase: NT = rup(9 NE, 32) x NPART threads, with
// NE B <= NT (column phase) and two CTAs per SM within 128 registers per thread
template <>
struct SpShape<5> {
  static constexpr int NE = 7, NPART = 4;
};
template <>
struct SpShape<4> {
  static constexpr int NE = 12, NPART = 2;
};
template <>
struct SpShape<3> {
  static constexpr int NE = 25, NPART = 1;
};

template <int O, int M>
struct SpCfg {
  using C = Cfg<O, M, 1>;
  static constexpr int B = C::B, F = C::F, NQ = C::NQ, NA = C::NA;
  static constexpr int NE = SpShape<O>::NE, NPART = SpShape<O>::NPART;
  static constexpr int NPAIR = 9 * NE;                 // (element, elastic row) pairs
  static constexpr int RT = rup(NPAIR, 32);            // threads per part
  static constexpr int NT = RT * NPART;
  static_assert(NE * B <= NT, "column phase needs one thread per (element, mode)");
  static constexpr int XP = RT + 1;                    // pair stride (1 mod 32)
  static constexpr int FR = C::FR;                     // floats per staged Riemann state
  static constexpr int FLS = 4 * F * FR;               // staged Riemann states per element
  static constexpr int S_X = 0;                        // [B][XP]        row operand
  static constexpr int S_Y = rup(S_X + B * XP, 4);     // [3 B][XP]      products Y_c / Z_c
  static constexpr int S_G = rup(S_Y + 3 * B * XP, 4); // [4 F][XP]      face traces G_i
  static constexpr int S_FH = rup(S_G + 4 * F * XP, 4);// [4 F][B]       F^
  static constexpr int S_FL = rup(S_FH + 4 * F * B, 4);
  static constexpr int S_E = rup(S_FL + NE * FLS, 4);
  static constexpr int S_META = rup(S_E + NE * ED, 4);
  static constexpr int TOTAL = rup(S_META + NE, 4);
};

// the generated products of order O
template <int O, int XP>
__device__ __forceinline__ void sp_time(int part, int variant, const float* x, float* y) {
  if constexpr (O == 5) ltssp::sp_time_o5<XP>(part, variant, x, y);
  if constexpr (O == 4) ltssp::sp_time_o4<XP>(part, variant, x, y);
  if constexpr (O == 3) ltssp::sp_time_o3<XP>(part, variant, x, y);
}
template <int O, int XP>
__device__ __forceinline__ void sp_vol(int part, const float* x, float* y, float* g) {
  if constexpr (O == 5) ltssp::sp_vol_o5<XP>(part, x, y, g);
  if constexpr (O == 4) ltssp::sp_vol_o4<XP>(part, x, y, g);
  if constexpr (O == 3) ltssp::sp_vol_o3<XP>(part, x, y, g);
}

template <int O, int M>
__global__ void __launch_bounds__(SpCfg<O, M>::NT, 2) k_predict_sp(DevOps ops, DevState st, PhaseArgs ph) {
  using S = SpCfg<O, M>;
  using C = typename S::C;
  constexpr int B = S::B, F = S::F, NE = S::NE, NT = S::NT, XP = S::XP, FR = S::FR, NQ = S::NQ, NA = S::NA;
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  float* sX = smem + S::S_X;
  float* sY = smem + S::S_Y;
  float* sG = smem + S::S_G;
  float* sFh = smem + S::S_FH;
  float* sFl = smem + S::S_FL;
  float* sE = smem + S::S_E;
  int* sMeta = reinterpret_cast<int*>(smem + S::S_META);
  const int tid = threadIdx.x;

  for (int i = tid; i < 4 * F * B; i += NT) sFh[i] = ops.Fh[i];

  // column task (element, mode), modes of the highest degree first
  int e = -1, b = 0, p = 0;
  task_of<O, NE>(tid, e, b, p);
  const bool act = e >= 0;
  const int es = act ? e : 0;
  const int fmax = nface(p + 1);                // face modes of degree <= deg b
  // row task (part, pair)
  const int part = tid / S::RT, pair = tid % S::RT;
  const bool ract = pair < S::NPAIR;
  const int nelem = ph.end - ph.begin;
  const int nbatch = (nelem + NE - 1) / NE;
  constexpr long long qs = C::QS, bs = C::BUFS;
  const int col = es * 9;                       // this column's pair offset

  for (int batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int e0 = ph.begin + batch * NE;
    __syncthreads();
    const int g = e0 + es;
    const bool valid = act && g < ph.end;
    const size_t qoff = (size_t)g * qs + b;
    const size_t boff = (size_t)g * bs + b;
    float T[NQ], Th[9], Da[NA > 0 ? NA : 1];
    float v[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) v[r] = 0.f;
    if (valid) {
      const float* q = st.Q + qoff;
#pragma unroll
      for (int r = 0; r < 9; ++r) v[r] = q[r * B];
#pragma unroll
      for (int r = 0; r < NA; ++r) Da[r] = q[(9 + r) * B];
    } else {
#pragma unroll
      for (int r = 0; r < NA; ++r) Da[r] = 0.f;
    }
    for (int i = tid; i < NE * ED; i += NT) {
      const int gg = e0 + i / ED;
      sE[i] = (gg < ph.end) ? st.edata[(size_t)gg * ED + (i % ED)] : 0.f;
    }
    if (tid < NE) sMeta[tid] = (e0 + tid < ph.end) ? st.meta[e0 + tid] : 0;
    if (act) {
#pragma unroll
      for (int r = 0; r < 9; ++r) sX[b * XP + col + r] = v[r];
    }
    __syncthreads();
    const float* ed = sE + es * ED;
    const int meta = act ? sMeta[es] : 0;
    const int cl = meta & 0xff;
#pragma unroll
    for (int r = 0; r < 9; ++r) {
      T[r] = ph.coef[cl][0] * v[r];
      Th[r] = ph.hcoef[cl][0] * v[r];
    }
#pragma unroll
    for (int r = 0; r < NA; ++r) T[9 + r] = ph.coef[cl][0] * Da[r];
    // ---- time kernel: d^{d+1} Q from d^d Q (Cauchy-Kowalevski), Taylor sums
#pragma unroll 1
    for (int d = 0; d < O - 1; ++d) {
      // elastic: d^d Q has degree <= O-1-d, so the product is truncated (variant d); the
      // anelastic coupling keeps every degree (variant 0)
      const int variant = (M == 0) ? d : 0;
      if (ract) sp_time<O, XP>(part, variant, sX + pair, sY + pair);
      __syncthreads();
      float Y[3][9];
      // outputs b >= nbasis(O-1-variant) are identically zero and not written
      const bool has = act && b < nbasis(O - 1 - variant);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 9; ++r) Y[c][r] = has ? sY[(c * B + b) * XP + col + r] : 0.f;
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
            const float w = ph.omega[l] * (eps[r] - Da[6 * l + r]);
            Da[6 * l + r] = w;
            T[9 + 6 * l + r] = fmaf(c1, w, T[9 + 6 * l + r]);
          }
        // next row operand: the next derivative, or after the last one the time integral
        float* xo = sX + b * XP + col;
        if (d < O - 2) {
#pragma unroll
          for (int r = 0; r < 9; ++r) xo[r] = out[r];
        } else {
#pragma unroll
          for (int r = 0; r < 9; ++r) xo[r] = T[r];
        }
      }
      __syncthreads();
    }
    // ---- LTS buffers (Eq. lts_buffers)
    if (valid) {
      float* b1 = st.B1 + boff;
#pragma unroll
      for (int r = 0; r < 9; ++r) b1[r * B] = T[r];
      if (meta & FLAG_FINER) {
        float* b2 = st.B2 + boff;
#pragma unroll
        for (int r = 0; r < 9; ++r) b2[r * B] = Th[r];
      }
      if (meta & FLAG_COARSER) {
        float* b3 = st.B3 + boff;
        if (ph.parity[cl] == 0) {
#pragma unroll
          for (int r = 0; r < 9; ++r) b3[r * B] = T[r];
        } else {
#pragma unroll
          for (int r = 0; r < 9; ++r) b3[r * B] += T[r];
        }
      }
    }
    // ---- volume products and local face traces of T (row phase)
    if (ract) sp_vol<O, XP>(part, sX + pair, sY + pair, sG + pair);
    __syncthreads();
    float acc[NQ];
    {
      float Z[3][9];
      // Z_c[0] = 0: K_c[k][0] vanishes for every k (the constant mode has no derivative)
      const bool has = act && b > 0;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 9; ++r) Z[c][r] = has ? sY[(c * B + b) * XP + col + r] : 0.f;
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
        for (int r = 0; r < 9; ++r) acc[r] = q[r * B] + V[r];
#pragma unroll
        for (int l = 0; l < M; ++l)
#pragma unroll
          for (int r = 0; r < 6; ++r)
            acc[9 + 6 * l + r] = q[(9 + 6 * l + r) * B] + ph.omega[l] * (-eps[r] - T[9 + 6 * l + r]);
      }
    }
    // ---- local surface kernel: interface states of the face traces G_i (one task per
    // element, face and face mode, face modes fastest), staged for the F^ projection
#pragma unroll 1
    for (int t = tid; t < NE * 4 * F; t += NT) {
      const int fe = t / (4 * F), fi = (t / F) % 4, f = t % F;
      const float* gp = sG + (fi * F + f) * XP + fe * 9;
      float gv[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) gv[r] = gp[r];
      float w6[6];
      riemann_state(gv, sE + fe * ED + 20 + 11 * fi, w6);
      store_state(sFl + fe * S::FLS + (fi * F + f) * FR, w6);
    }
    __syncthreads();
    if (valid) {
      constexpr int NS = (M > 0) ? 15 : 9;
      float Sv[NS];
#pragma unroll
      for (int r = 0; r < NS; ++r) Sv[r] = 0.f;
      project_faces<NS, F, B, FR>(sFl + es * S::FLS, sFh, ed + 20, 11, ed[9], ed[10], ed[11], fmax, b, Sv);
      float* q = st.Q + qoff;
#pragma unroll
      for (int r = 0; r < 9; ++r) q[r * B] = acc[r] + Sv[r];
      if constexpr (M > 0) {
#pragma unroll
        for (int l = 0; l < M; ++l)
#pragma unroll
          for (int r = 0; r < 6; ++r) q[(9 + 6 * l + r) * B] = acc[9 + 6 * l + r] + ph.omega[l] * Sv[NS - 6 + r];
      }
    }
    {
      const int bn = batch + gridDim.x;                    // this CTA's next batch
      if (bn < nbatch) {
        const int en = ph.begin + bn * NE;
        prefetch_batch_q<NQ, B, 1, NT>(st.Q, qs, en, 0, min(NE, ph.end - en), tid);
      }
    }
  }
}

}  // namespace ltsdev
