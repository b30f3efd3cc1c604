// k_predict_sp: the predict + local kernel (time kernel, LTS buffers, volume kernel, local
// surface kernel; Sec. III-A and Eq. lts_buffers) with the operator products in generated
// sparse form (one simulation, or (element, simulation) slots of fused simulations), and
// k_neighbour_sp, the neighbour surface kernel of the same engine (below).
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
//   column phase: thread = (element e, mode b), modes fastest (fused simulations: the
//                 simulations of an element fastest): it reads the 27 products of
//                 its column, applies the star matrices (physical form), the
//                 anelastic coupling and relaxation, adds the Taylor terms and writes the
//                 next derivative's column back for the next row phase.
// Shared-memory arrays are [mode or output][pair] with a pair stride XP = 1 mod 32, so the
// row phase's loads and stores (consecutive pairs) and the column phase's accesses
// (consecutive modes) fall on distinct banks.
// The local surface kernel's interface states (closed-form Riemann solver of kernels.cuh) are
// projected the same way (row phase with the generated F^_i products), and the column phase
// forms the flux rows per face. A batch's DOFs arrive in shared memory by one bulk
// asynchronous copy (TMA), issued a batch ahead. Receivers and sources are those of
// kernels.cuh.
#pragma once
#include "kernels.cuh"
#include "sparse_ops.cuh"
#include "tc.cuh"

namespace ltsdev {

template <int O>
struct SpShape;
// elements per CTA and parts of the row phase: NT = rup(9 NE, 32) x NPART threads, with
// NE B <= NT (column phase), within 128 registers per thread. Order 5: one CTA of 512 threads
// per SM (14 elements), so that the SM's warps run each phase's code together — the kernel
// is bound by instruction fetch, and two CTAs of 7 elements in different phases fetch two
// phases' code at once (measured: 88.5 against 72.2 M sim-element-updates/s with 4 fused
// simulations, 88.5 against 86.7 M element-updates/s for one); orders 3 and 4: two CTAs.
template <>
struct SpShape<5> {
  static constexpr int NE = 14, NPART = 4;
};
template <>
struct SpShape<4> {
  static constexpr int NE = 12, NPART = 2;
};
template <>
struct SpShape<3> {
  static constexpr int NE = 25, NPART = 1;
};

template <int O, int M, bool FU = false>
struct SpCfg {
  using C = Cfg<O, M, 1>;
  static constexpr int B = C::B, F = C::F, NQ = C::NQ, NA = C::NA;
  static constexpr int NE = SpShape<O>::NE, NPART = SpShape<O>::NPART;
  static constexpr int NPAIR = 9 * NE;                 // (element, elastic row) pairs
  static constexpr int RT = rup(NPAIR, 32);            // threads per part
  static constexpr int NT = RT * NPART;
  static_assert(NE * B <= NT, "column phase needs one thread per (element, mode)");
  static constexpr int XP = RT + 1;                    // pair stride (1 mod 32)
  static constexpr int EDP = ED + 1;                   // staged element data stride (odd: elements
                                                       // of one warp on distinct banks)
  static constexpr int S_X = 0;                        // [B][XP]          row operand
  static constexpr int S_Y = rup(S_X + B * XP, 4);     // [3 B][XP]        products Y_c / Z_c
  static constexpr int S_G = rup(S_Y + 3 * B * XP, 4); // [4 F][XP]        face traces G_i
  static constexpr int S_P = S_Y;                      // [4 B][XP]        projected states P_i
  static_assert(S_P + 4 * B * XP <= S_G + 4 * F * XP, "P_i overlays Y and G");
  static constexpr int S_W = rup(S_G + 4 * F * XP, 4); // [4 F][XP]        interface states, 6 rows
  static constexpr int S_E = rup(S_W + 4 * F * XP, 4);
  static constexpr int S_META = rup(S_E + NE * EDP, 4);  // [3][NE] ints: meta, element, simulation
  // the batch's DOFs: NE elements of QS floats (one simulation), or the simulation groups
  // that NE consecutive (element, simulation) slots touch, at most NE / G + 2 groups of
  // NQ x B x G floats (fused, G = FUSED_GROUP)
  static constexpr int GB = NQ * B * FUSED_GROUP;
  static constexpr int QBUF = FU ? (NE / FUSED_GROUP + 2) * GB : NE * C::QS;
  static constexpr int S_Q = rup(S_META + 3 * NE, 4);      // [QBUF] the batch's DOFs
  static constexpr int S_BAR = rup(S_Q + QBUF, 4);         // mbarrier of the DOF copy (8 bytes)
  static constexpr int TOTAL = S_BAR + 4;
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
template <int O, int XP>
__device__ __forceinline__ void sp_proj(int part, const float* x, float* y) {
  if constexpr (O == 5) ltssp::sp_proj_o5<XP>(part, x, y);
  if constexpr (O == 4) ltssp::sp_proj_o4<XP>(part, x, y);
  if constexpr (O == 3) ltssp::sp_proj_o3<XP>(part, x, y);
}

// Slots of a phase: one simulation (FUSED false): slot = element; fused simulations: slot =
// (element, simulation), the simulations of an element consecutive, simulation f of element
// k at k * (element stride) + (f / G) * (rows x B x G) + (row x B + mode) x G + f mod G in the
// simulation-blocked layout (G = FUSED_GROUP). The per-slot arithmetic is the same either way.
// Slot counts fit 32 bits (checked when the mesh is set). Fused kernels decode a batch's
// slots once (one division each, by the first NE threads) into shared memory.
template <bool FUSED>
struct Slots {
  int nsim;
  int n;                                        // slots in the phase
  __device__ Slots(const DevState& st, const PhaseArgs& ph)
      : nsim(FUSED ? st.nsim : 1), n((ph.end - ph.begin) * (FUSED ? st.nsim : 1)) {}
  // element (offset from the phase's first) and simulation of slot t < n
  __device__ void decode(int t, int& e, int& f) const {
    if (!FUSED) {
      e = t;
      f = 0;
    } else {
      e = (int)((unsigned)t / (unsigned)nsim);
      f = t - e * nsim;
    }
  }
  // offset of (simulation f, row 0, mode 0) from its element's start in an array of `rows` rows
  __device__ static int sub(int f, int rows, int B) {
    if (!FUSED) return 0;
    return (int)((unsigned)f / FUSED_GROUP) * rows * B * FUSED_GROUP + (int)((unsigned)f % FUSED_GROUP);
  }
};

template <int O, int M, bool FUSED>
__global__ void __launch_bounds__(SpCfg<O, M, FUSED>::NT, (SpCfg<O, M, FUSED>::NT >= 512 ? 1 : 2))
    k_predict_sp(DevOps ops, DevState st, PhaseArgs ph) {
  using S = SpCfg<O, M, FUSED>;
  using C = typename S::C;
  constexpr int B = S::B, F = S::F, NE = S::NE, NT = S::NT, XP = S::XP, NQ = S::NQ, NA = S::NA, EDP = S::EDP;
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  float* sX = smem + S::S_X;
  float* sY = smem + S::S_Y;
  float* sG = smem + S::S_G;
  float* sP = smem + S::S_P;
  float* sW = smem + S::S_W;
  float* sE = smem + S::S_E;
  int* sMeta = reinterpret_cast<int*>(smem + S::S_META);
  int* sSlot = sMeta + NE;                    // fused: [2][NE] element, simulation of the batch's slots
  float* sQ = smem + S::S_Q;
  uint64_t* sBar = reinterpret_cast<uint64_t*>(smem + S::S_BAR);
  const int tid = threadIdx.x;

  // column task (slot, mode). One simulation: modes fastest (a warp spans at most two
  // elements, and reads a row's consecutive modes). Fused simulations: set per batch below.
  const bool act = tid < NE * B;
  int es = act ? tid / B : 0;
  int b = act ? tid % B : 0;
  // row task (part, pair): warp w takes part w mod NPART, so that the warps an SM
  // sub-partition runs (w mod 4) all execute the same part's straight-line code and its
  // instruction cache holds one part only
  const int part = (tid >> 5) % S::NPART, pair = ((tid >> 5) / S::NPART) * 32 + (tid & 31);
  const bool ract = pair < S::NPAIR;          // (element, quantity) rows of the 9 elastic rows
  const bool pact = pair < 6 * NE;            // (element, interface-state) rows of the projection
  const Slots<FUSED> sl(st, ph);
  const int nbatch = (sl.n + NE - 1) / NE;
  const long long qs = FUSED ? st.qs : C::QS, bs = FUSED ? st.bs : C::BUFS;
  constexpr int RS = FUSED ? B * FUSED_GROUP : B;   // row stride of Q and the buffers
  constexpr int CS = FUSED ? FUSED_GROUP : 1;       // mode stride
  int col = es * 9;                           // this column's pair offset
  // A batch's DOFs arrive in shared memory by one bulk asynchronous copy (TMA) that thread 0
  // issues for the next batch as soon as the current one has read its copy, completing on an
  // mbarrier (one phase per batch): one simulation, the batch's contiguous elements (n x QS
  // floats); fused simulations, the contiguous simulation groups from the batch's first slot
  // to its last. Every wait is bounded; one that gives up sets the error word and the CTA
  // returns.
  constexpr int GB = S::GB;
  auto issue_q = [&](int bt) {
    const float* src;
    uint32_t bytes;
    if constexpr (!FUSED) {
      const int e0 = ph.begin + bt * NE;
      src = st.Q + (size_t)e0 * C::QS;
      bytes = (uint32_t)min(NE, ph.end - e0) * C::QS * 4;
    } else {
      int e0, f0, e1, f1;
      sl.decode(bt * NE, e0, f0);
      sl.decode(min(sl.n, bt * NE + NE) - 1, e1, f1);
      const int ngr = sl.nsim / FUSED_GROUP;
      src = st.Q + (size_t)(ph.begin + e0) * qs + (size_t)(f0 / FUSED_GROUP) * GB;
      bytes = (uint32_t)((e1 - e0) * ngr + f1 / FUSED_GROUP - f0 / FUSED_GROUP + 1) * GB * 4;
    }
    tc::bulk_load(sQ, src, bytes, sBar);
  };
  uint32_t qpar = 0;
  if (tid == 0) tc::mbar_init(sBar, 1);
  __syncthreads();
  if (tid == 0 && blockIdx.x < nbatch && !ph.suppress) issue_q(blockIdx.x);

  for (int batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int t0 = batch * NE;
    // element of the batch's slot k (fused: decoded below; every read of sSlot comes before
    // the batch's second barrier, every write before its first)
    auto elem_of = [&](int k) { return FUSED ? sSlot[k] : ph.begin + t0 + k; };
    if (FUSED && tid < NE) {
      int e = 0, f = 0;
      if (t0 + tid < sl.n) sl.decode(t0 + tid, e, f);
      sSlot[tid] = ph.begin + e;
      sSlot[NE + tid] = f;
    }
    // one simulation: the barrier of the DOF wait below follows the previous batch's update
    if constexpr (FUSED) __syncthreads();
    if (FUSED && act) {
      // fused column tasks ordered by (element, mode, simulation): the slots of the batch that
      // share an element form a segment [s0, s1), and its B (s1 - s0) tasks take the modes in
      // turn with the segment's simulations fastest, so that a warp's lanes read consecutive
      // floats of the simulation-blocked layout (tasks of slot m lie in segment of slot m)
      const int m = tid / B;
      const int nval = min(NE, sl.n - t0);
      if (m < nval) {
        const int fm = sSlot[NE + m];
        const int s0 = max(0, m - fm), s1 = min(nval, m - fm + sl.nsim);
        const int local = tid - B * s0, nf = s1 - s0;
        b = local / nf;
        es = s0 + local % nf;
      } else {
        es = m;
        b = tid % B;
      }
      col = es * 9;
    }
    const int ts = t0 + es;
    const bool valid = act && ts < sl.n;
    const int g = valid ? elem_of(es) : ph.begin;
    const int fs = (FUSED && valid) ? sSlot[NE + es] : 0;
    const size_t qoff = (size_t)g * qs + Slots<FUSED>::sub(fs, NQ, B) + (size_t)b * CS;
    const size_t boff = (size_t)g * bs + Slots<FUSED>::sub(fs, 9, B) + (size_t)b * CS;
    {
      // the batch's DOFs have arrived (or the wait gave up: every thread leaves)
      const bool ok = tc::mbar_wait(sBar, qpar, ph.wait);
      qpar ^= 1;
      if (!__syncthreads_and(ok)) {
        if (tid == 0) {
          atomicOr(ph.err, 1);
          tc::mbar_wait(sBar, qpar ^ 1, ph.wait);   // the copy in flight, if any, lands first
        }
        return;
      }
    }
    // this column's DOFs in the staged copy (row stride RS, as in Q)
    size_t soff = (size_t)es * C::QS + b;
    if constexpr (FUSED) {
      const int ngr = sl.nsim / FUSED_GROUP;
      const int gi = (g - sSlot[0]) * ngr + fs / FUSED_GROUP - sSlot[NE] / FUSED_GROUP;
      soff = (size_t)gi * GB + (size_t)b * CS + fs % FUSED_GROUP;
    }
    float T[NQ], Th[9], Da[NA > 0 ? NA : 1];
    float v[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) v[r] = 0.f;
    if (valid) {
      const float* q = sQ + soff;
#pragma unroll
      for (int r = 0; r < 9; ++r) v[r] = q[r * RS];
#pragma unroll
      for (int r = 0; r < NA; ++r) Da[r] = q[(9 + r) * RS];
    } else {
#pragma unroll
      for (int r = 0; r < NA; ++r) Da[r] = 0.f;
    }
    for (int i = tid; i < NE * ED; i += NT) {
      const int ee = i / ED;
      const bool in = t0 + ee < sl.n;
      sE[ee * EDP + i % ED] = in ? st.edata[(size_t)elem_of(ee) * ED + (i % ED)] : 0.f;
    }
    if (tid < NE) sMeta[tid] = (t0 + tid < sl.n) ? st.meta[elem_of(tid)] : 0;
    if (act) {
#pragma unroll
      for (int r = 0; r < 9; ++r) sX[b * XP + col + r] = v[r];
    }
    __syncthreads();
    const float* ed = sE + es * EDP;
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
      for (int r = 0; r < 9; ++r) b1[r * RS] = T[r];
      if (meta & FLAG_FINER) {
        float* b2 = st.B2 + boff;
#pragma unroll
        for (int r = 0; r < 9; ++r) b2[r * RS] = Th[r];
      }
      if (meta & FLAG_COARSER) {
        float* b3 = st.B3 + boff;
        if (ph.parity[cl] == 0) {
#pragma unroll
          for (int r = 0; r < 9; ++r) b3[r * RS] = T[r];
        } else {
#pragma unroll
          for (int r = 0; r < 9; ++r) b3[r * RS] += T[r];
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
        const float* q = sQ + soff;
#pragma unroll
        for (int r = 0; r < 9; ++r) acc[r] = q[r * RS] + V[r];
#pragma unroll
        for (int l = 0; l < M; ++l)
#pragma unroll
          for (int r = 0; r < 6; ++r)
            acc[9 + 6 * l + r] = q[(9 + 6 * l + r) * RS] + ph.omega[l] * (-eps[r] - T[9 + 6 * l + r]);
      }
    }
    // ---- local surface kernel: interface states (v*, t*) of the face traces G_i, one task
    // per element, face and face mode (face modes fastest), as rows of the projection
#pragma unroll 1
    for (int t = tid; t < NE * 4 * F; t += NT) {
      const int fe = t / (4 * F), fi = (t / F) % 4, f = t % F;
      const float* gp = sG + (fi * F + f) * XP + fe * 9;
      float gv[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) gv[r] = gp[r];
      float w6[6];
      riemann_state(gv, sE + fe * EDP + 20 + 11 * fi, w6);
      float* wp = sW + (fi * F + f) * XP + fe * 6;
#pragma unroll
      for (int r = 0; r < 6; ++r) wp[r] = w6[r];
    }
    __syncthreads();
    // the batch's DOF copy has been read: the next batch's copy goes out now
    if (tid == 0 && batch + (int)gridDim.x < nbatch && !ph.suppress) issue_q(batch + gridDim.x);
    // ---- projection P_i[r'][b] = sum_f W_i[r'][f] F^_i[f][b] (row phase, over Y and G)
    if (pact) sp_proj<O, XP>(part, sW + pair, sP + pair);
    __syncthreads();
    if (valid) {
      constexpr int NS = (M > 0) ? 15 : 9;
      float Sv[NS];
#pragma unroll
      for (int r = 0; r < NS; ++r) Sv[r] = 0.f;
      // one copy of the face code (the kernel is bound by instruction fetch)
#pragma unroll 1
      for (int i = 0; i < 4; ++i) {
        const float* pp = sP + (i * B + b) * XP + es * 6;
        float W[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) W[r] = pp[r];
        flux_rows_add<NS>(W, ed + 20 + 11 * i, ed[9], ed[10], ed[11], Sv);
      }
      float* q = st.Q + qoff;
#pragma unroll
      for (int r = 0; r < 9; ++r) q[r * RS] = acc[r] + Sv[r];
      if constexpr (M > 0) {
#pragma unroll
        for (int l = 0; l < M; ++l)
#pragma unroll
          for (int r = 0; r < 6; ++r) q[(9 + 6 * l + r) * RS] = acc[9 + 6 * l + r] + ph.omega[l] * Sv[NS - 6 + r];
      }
    }
  }
}

// ------------------------------------------------------------------ neighbour kernel
// k_neighbour_sp: the neighbour surface kernel (Sec. III-A, with the buffer chosen by the
// clusters' time-stepping relation, Sec. V-B), one simulation, no partition. The neighbour
// matrices factor as F-_{j,h} = F~_j R_h (trace on the neighbour's face j, then the face-basis
// map R_h of the orientation, block diagonal by degree), so H = X F-_{j,h} is formed as
// (X F~_j) R_h:
//   gather:      thread = (element, mode): the four neighbours' buffer columns (B1, B2, B3 or
//                B1 - B2) into shared memory, rows (element, face, quantity) as pairs;
//   trace phase: thread = (element, face, quantity): the generated sparse product X F~_j for
//                the face j its neighbour touches (a warp computes the faces its lanes need);
//   states:      thread = (element, face, face mode): H = G R_h (degree block), closed-form
//                interface state with the neighbour coefficients;
//   projection:  row phase with the generated F^_i products, as in k_predict_sp;
//   update:      thread = (element, mode): flux rows per face, Q <- Q + S^N.
template <int O, int M, int NE_>
struct SpnCfg {
  using C = Cfg<O, M, 1>;
  static constexpr int B = C::B, F = C::F, NQ = C::NQ;
  static constexpr int NE = NE_;                        // elements per CTA (tile variant: 8 or 4)
  static constexpr int NROW = NE * 4 * 9;               // (element, face, quantity) rows
  static constexpr int NT = rup(NROW > NE * B ? NROW : NE * B, 32);
  static constexpr int XN = NROW + 1;                   // row stride of gathered columns and traces
  static constexpr int NPART = SpShape<O>::NPART;       // parts of the projection
  static constexpr int RT6 = rup(6 * NE, 32);
  static_assert(NPART * RT6 <= NT, "projection rows");
  static constexpr int XP6 = RT6 + 1;                   // stride of interface states / projections
  static constexpr int NDP = ND + 1;
  static constexpr int S_X = 0;                                                      // [B][XN]
  static constexpr int S_P = 0;                                                      // [4B][XP6] over X
  static constexpr int S_G = rup((B * XN > 4 * B * XP6) ? B * XN : 4 * B * XP6, 4);  // [F][XN]
  static constexpr int S_W = rup(S_G + F * XN, 4);                                   // [4F][XP6]
  static constexpr int S_R = rup(S_W + 4 * F * XP6, 4);                              // [3][F][F]
  static constexpr int S_D = rup(S_R + 3 * F * F, 4);                                // [NE][NDP]
  static constexpr int S_I = rup(S_D + NE * NDP, 4);                                 // [NE][9] ints
  static constexpr int S_PERM = rup(S_I + NE * 9, 4);                                // [4 NE] ints
  static constexpr int S_SLOT = rup(S_PERM + 4 * NE, 4);                             // [2][NE] ints
  static constexpr int S_Q = rup(S_SLOT + 2 * NE, 4);                                // [NE][QS] one simulation: DOFs
  static constexpr int S_BAR = rup(S_Q + NE * C::QS, 4);                             // mbarrier (8 bytes)
  static constexpr int TOTAL = S_BAR + 4;
  static_assert(4 * NE <= 32, "one warp sorts the face slots of a batch");
};

template <int O, int XP>
__device__ __forceinline__ void sp_ntrace(int j, const float* x, float* y) {
  if constexpr (O == 5) ltssp::sp_ntrace_o5<XP>(j, x, y);
  if constexpr (O == 4) ltssp::sp_ntrace_o4<XP>(j, x, y);
  if constexpr (O == 3) ltssp::sp_ntrace_o3<XP>(j, x, y);
}

template <int O, int M, int NE_, bool FUSED>
__global__ void __launch_bounds__(SpnCfg<O, M, NE_>::NT, (NE_ == 8 ? 2 : 4))
    k_neighbour_sp(DevOps ops, DevState st, PhaseArgs ph) {
  using S = SpnCfg<O, M, NE_>;
  using C = typename S::C;
  constexpr int B = S::B, F = S::F, NE = S::NE, NT = S::NT, XN = S::XN, XP6 = S::XP6, NQ = S::NQ, NDP = S::NDP;
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  float* sX = smem + S::S_X;
  float* sP = smem + S::S_P;
  float* sG = smem + S::S_G;
  float* sW = smem + S::S_W;
  float* sR = smem + S::S_R;
  float* sD = smem + S::S_D;
  int* sI = reinterpret_cast<int*>(smem + S::S_I);      // per element: nbr[4], code[4], meta
  int* sPerm = reinterpret_cast<int*>(smem + S::S_PERM); // face slots ordered by the neighbour's face j
  int* sSlot = reinterpret_cast<int*>(smem + S::S_SLOT); // fused: element, simulation of the batch's slots
  float* sQ = smem + S::S_Q;
  uint64_t* sBar = reinterpret_cast<uint64_t*>(smem + S::S_BAR);
  const int tid = threadIdx.x;
  for (int i = tid; i < 3 * F * F; i += NT) sR[i] = ops.Rh[i];

  const bool act = tid < NE * B;                         // column task (slot, mode), as in k_predict_sp
  const int es = act ? (FUSED ? tid % NE : tid / B) : 0;
  const int b = act ? (FUSED ? tid / NE : tid % B) : 0;

  const int part = (tid >> 5) % S::NPART;                // projection row: as in k_predict_sp
  const int pair6 = ((tid >> 5) / S::NPART) * 32 + (tid & 31);
  const bool pact = pair6 < 6 * NE;
  const Slots<FUSED> sl(st, ph);
  const int nbatch = (sl.n + NE - 1) / NE;
  const long long qs = FUSED ? st.qs : C::QS, bs = FUSED ? st.bs : C::BUFS;
  constexpr int RS = FUSED ? B * FUSED_GROUP : B;   // row stride of Q and the buffers
  constexpr int CS = FUSED ? FUSED_GROUP : 1;       // mode stride
  // One simulation: the batch's DOFs (read by the update, the last phase) arrive by one bulk
  // asynchronous copy that thread 0 issues at the batch's start, completing on an mbarrier;
  // the wait before the update is bounded, as in k_predict_sp.
  uint32_t qpar = 0;
  if constexpr (!FUSED) {
    if (tid == 0) tc::mbar_init(sBar, 1);
  }

  for (int batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int t0 = batch * NE;
    // element of the batch's slot k, as in k_predict_sp
    auto elem_of = [&](int k) { return FUSED ? sSlot[k] : ph.begin + t0 + k; };
    if (FUSED && tid < NE) {
      int e = 0, f = 0;
      if (t0 + tid < sl.n) sl.decode(t0 + tid, e, f);
      sSlot[tid] = ph.begin + e;
      sSlot[NE + tid] = f;
    }
    // one simulation: no barrier here. The previous batch's update (its last reads of sD, sP
    // and sQ) ends before the barrier below, and its last read of sI came before its states
    // phase's barrier, so the sI writes that follow overwrite nothing still in use
    if constexpr (FUSED) __syncthreads();
    for (int i = tid; i < NE * 9; i += NT) {
      const int c = i % 9;
      int v = -1;
      if (t0 + i / 9 < sl.n) {
        const int gg = elem_of(i / 9);
        v = (c < 4) ? __ldg(st.nbr + (size_t)gg * 4 + c) : (c < 8 ? __ldg(st.ncode + (size_t)gg * 4 + c - 4) : __ldg(st.meta + gg));
      }
      sI[i] = v;
    }
    __syncthreads();
    if constexpr (!FUSED) {
      // the previous batch's update has read its copy (barrier above)
      if (tid == 0 && !ph.suppress) {
        const int e0 = ph.begin + t0;
        tc::bulk_load(sQ, st.Q + (size_t)e0 * C::QS, (uint32_t)min(NE, ph.end - e0) * C::QS * 4, sBar);
      }
    }
    // neighbour coefficients, first read by the states phase (two barriers on)
    for (int i = tid; i < NE * ND; i += NT) {
      const int ee = i / ND;
      sD[ee * NDP + i % ND] = (t0 + ee < sl.n) ? __ldg(st.ndata + (size_t)elem_of(ee) * ND + (i % ND)) : 0.f;
    }
    // face slots (element, face) sorted by the neighbour's face j (faces without one last), so
    // that the rows of a warp mostly ask for one face in the trace phase
    if (tid < 32) {
      const int fe = tid / 4, fi = tid % 4;
      int key = 5;                                      // lanes past the batch's face slots
      if (tid < 4 * NE) key = (t0 + fe < sl.n && sI[fe * 9 + fi] >= 0) ? (sI[fe * 9 + 4 + fi] & 0xff) / 3 : 4;
      const unsigned lt = (1u << tid) - 1u;
      int base = 0, rank = 0;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const unsigned m = __ballot_sync(0xffffffffu, key == k);
        if (key == k) rank = base + __popc(m & lt);
        base += __popc(m);
      }
      if (tid < 4 * NE) sPerm[rank] = tid;
    }
    const int ts = t0 + es;
    const bool valid = act && ts < sl.n;
    const int g = valid ? elem_of(es) : ph.begin;
    const int fs = (FUSED && valid) ? sSlot[NE + es] : 0;
    const size_t bsub = Slots<FUSED>::sub(fs, 9, B);    // this slot's simulation in the buffers
    // ---- gather the neighbours' time-integrated DOFs by cluster relation (Sec. V-B)
    if (act) {
      const int* ie = sI + es * 9;
      const int cl = ie[8] & 0xff;
      const int par = valid ? ph.parity[cl] : 0;
      float xv[4][9];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int nb = valid ? ie[i] : -1;
        const int rel = (ie[4 + i] >> 8) & 0xff;
        const float* src1 = (rel == 1) ? st.B3 : ((rel == 2 && par == 0) ? st.B2 : st.B1);
        const bool sub = (rel == 2 && par == 1);
        const size_t off = (size_t)(nb < 0 ? 0 : nb) * bs + bsub + (size_t)b * CS;
#pragma unroll
        for (int r = 0; r < 9; ++r) xv[i][r] = (nb < 0) ? 0.f : __ldg(src1 + off + r * RS);
        if (sub) {
#pragma unroll
          for (int r = 0; r < 9; ++r) xv[i][r] -= __ldg(st.B2 + off + r * RS);
        }
      }
      float* xo = sX + b * XN + es * 36;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int r = 0; r < 9; ++r) xo[i * 9 + r] = xv[i][r];
    }
    __syncthreads();
    // ---- traces on the neighbour's face j (every thread calls: warp-uniform face branches)
    {
      int j = -1, row = 0;
      if (tid < S::NROW) {
        const int slot = sPerm[tid / 9], fe = slot / 4, fi = slot % 4;
        row = slot * 9 + tid % 9;
        if (t0 + fe < sl.n && sI[fe * 9 + fi] >= 0) j = (sI[fe * 9 + 4 + fi] & 0xff) / 3;
      }
      sp_ntrace<O, XN>(j, sX + row, sG + row);
    }
    __syncthreads();
    // ---- H = G R_h per face mode (degree block), interface states with the neighbour
    // coefficients; faces without a neighbour contribute nothing
#pragma unroll 1
    for (int t = tid; t < NE * 4 * F; t += NT) {
      const int fe = t / (4 * F), fi = (t / F) % 4, f = t % F;
      float w6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (t0 + fe < sl.n && sI[fe * 9 + fi] >= 0) {
        const int h = (sI[fe * 9 + 4 + fi] & 0xff) % 3;
        const int pf = face_degree(f), f0 = nface(pf), f1 = nface(pf + 1);
        const float* gp = sG + (fe * 4 + fi) * 9;
        const float* R = sR + h * F * F + f;
        float hv[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) hv[r] = 0.f;
        for (int q = f0; q < f1; ++q) {
          const float w = R[q * F];
#pragma unroll
          for (int r = 0; r < 9; ++r) hv[r] = fmaf(gp[q * XN + r], w, hv[r]);
        }
        riemann_state(hv, sD + fe * NDP + 4 + 11 * fi, w6);
      }
      float* wp = sW + (fi * F + f) * XP6 + fe * 6;
#pragma unroll
      for (int r = 0; r < 6; ++r) wp[r] = w6[r];
    }
    __syncthreads();
    // ---- projection P_i[r'][b] = sum_f W_i[r'][f] F^_i[f][b] (row phase, over the gathers)
    if (pact) sp_proj<O, XP6>(part, sW + pair6, sP + pair6);
    // one simulation: the barrier of the DOF wait below orders the projections and the update
    if constexpr (FUSED) __syncthreads();
    if constexpr (!FUSED) {
      // the batch's DOFs have arrived (or the wait gave up: every thread leaves)
      const bool ok = tc::mbar_wait(sBar, qpar, ph.wait);
      qpar ^= 1;
      if (!__syncthreads_and(ok)) {
        if (tid == 0) {
          atomicOr(ph.err, 1);
          tc::mbar_wait(sBar, qpar ^ 1, ph.wait);   // the copy in flight, if any, lands first
        }
        return;
      }
    }
    if (valid) {
      constexpr int NS = (M > 0) ? 15 : 9;
      float* q = st.Q + (size_t)g * qs + Slots<FUSED>::sub(fs, NQ, B) + (size_t)b * CS;
      const float* qr = FUSED ? q : sQ + es * C::QS + b;
      float qv[NQ];
#pragma unroll
      for (int r = 0; r < NQ; ++r) qv[r] = qr[r * RS];
      float Sv[NS];
#pragma unroll
      for (int r = 0; r < NS; ++r) Sv[r] = 0.f;
      const float* nd = sD + es * NDP;
      // one copy of the face code (the kernel is bound by instruction fetch)
#pragma unroll 1
      for (int i = 0; i < 4; ++i) {
        const float* pp = sP + (i * B + b) * XP6 + es * 6;
        float W[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) W[r] = pp[r];
        flux_rows_add<NS>(W, nd + 4 + 11 * i, nd[0], nd[1], nd[2], Sv);
      }
#pragma unroll
      for (int r = 0; r < 9; ++r) q[r * RS] = qv[r] + Sv[r];
      if constexpr (M > 0) {
#pragma unroll
        for (int l = 0; l < M; ++l)
#pragma unroll
          for (int r = 0; r < 6; ++r) q[(9 + 6 * l + r) * RS] = qv[9 + 6 * l + r] + ph.omega[l] * Sv[NS - 6 + r];
      }
    }
  }
}

}  // namespace ltsdev
