// Tensor-core variant of the predict + local kernel (k_predict_tc).
//
// The two contractions of the time and volume kernels with the stiffness matrices
// (Sec. IV, time kernel X K_c^T, volume kernel T K_c, for the 9 elastic rows) run on the
// 5th-generation tensor cores: one tcgen05 MMA chain per derivative computes, for all
// slots of the CTA at once,
//     D[(c, b), (s, r)] = sum_k A[(c, b), k] X_s[r, k],
// M = 128 rows (c, b) (3 B used), N = 9 NE rows (slot s, quantity r) padded to 16, K = B
// modes padded to KP. A (the stacked K_c in either orientation) is a constant operand
// held in tensor memory for the life of the CTA; X is staged in shared memory in the
// K-major core-matrix layout; D accumulates in tensor memory and is moved through
// shared memory to the threads (slot, b) that apply the star matrices, exactly as in
// k_predict_local. With passes = 3 every product is split into tf32 parts,
// A X = A_hi X_hi + A_hi X_lo + A_lo X_hi (FP32-level accuracy); passes = 1 uses the
// rounded tf32 parts only. Everything else (Taylor sums, LTS buffers, anelastic terms,
// local surface kernel, update) is the CUDA-core code of k_predict_local.
#pragma once
#include "kernels.cuh"
#include "tc.cuh"

namespace ltsdev {

template <int O, int M, int FG>
struct TcCfg {
  using C = Cfg<O, M, FG>;
  static constexpr int B = C::B, NE = C::NE, F = C::F;
  static constexpr int KP = rup(B, 8);               // contraction length padded to the MMA K step
  static constexpr int NN = rup(9 * NE, 16);         // MMA N: rows (slot, r)
  static constexpr int COLS = 256;                   // tensor-memory columns per CTA
  static constexpr int T_D = 0;                      // accumulator columns [0, NN)
  static constexpr int T_ACK = NN;                   // time-kernel A: hi at +0, lo at +KP
  static constexpr int T_AVOL = NN + 2 * KP;         // volume A: hi at +0, lo at +KP
  // rows (c, b) must lie in lane quadrants that the CTA's warps can reach (warp w reaches
  // lanes 32 (w % 4) .. + 31)
  static constexpr bool SUPPORTED =
      3 * B <= 128 && NN <= 256 && T_AVOL + 2 * KP <= COLS && (3 * B + 31) / 32 <= C::NT / 32;
  // core matrices 16 bytes apart beyond their 128 bytes along K: consecutive modes of one
  // row then fall on consecutive banks when the threads (slot, b) stage their rows
  static constexpr int LBO = 144;
  static constexpr int SBO = (KP / 4) * LBO;
  static constexpr int XBYTES = (NN / 8) * SBO;      // one operand copy (hi or lo)
  static constexpr int YS = 27;                      // floats per (slot, mode) of the D exchange (odd)
  static constexpr int CW = (NN % 32 == 0) ? 32 : 16;  // accumulator columns per TMEM load
  // shared memory (floats)
  static constexpr int S_X = 0;
  static constexpr int S_Y = S_X + 2 * XBYTES / 4;
  static constexpr int S_FT = rup(S_Y + NE * B * YS, 4);
  static constexpr int S_FH = rup(S_FT + 4 * B * F, 4);
  static constexpr int S_A = rup(S_FH + 4 * F * B, 4);
  static constexpr int S_FL = rup(S_A + NE * B * C::AR, 4);
  static constexpr int S_E = rup(S_FL + NE * C::FLS, 4);
  static constexpr int S_META = rup(S_E + C::NEL * ED, 4);
  static constexpr int S_BAR = rup(S_META + C::NEL, 4);        // mbarrier, then the TMEM address
  static constexpr int S_TOTAL = S_BAR + 4;
  // at least 80 KB per CTA, so that no more than two CTAs (2 x 256 TMEM columns) share an SM
  static constexpr int SMEM_BYTES = (S_TOTAL * 4 > 80 * 1024) ? S_TOTAL * 4 : 80 * 1024;
};

// Default bound of the wait for one MMA chain: about one second at the maximum SM clock.
constexpr long long TC_WAIT_CYCLES = 2000000000LL;

template <int O, int M, int FG>
__global__ void __launch_bounds__(Cfg<O, M, FG>::NT, 2)
    k_predict_tc(DevOps ops, DevState st, PhaseArgs ph, int passes, int* err, long long wait_cycles,
                 int suppress_commit) {
  using C = Cfg<O, M, FG>;
  using TC = TcCfg<O, M, FG>;
  static_assert(TC::SUPPORTED, "shape outside the tensor-core path");
  constexpr int B = C::B, F = C::F, NE = C::NE, NEL = C::NEL, NT = C::NT, AR = C::AR, FR = C::FR;
  constexpr int NQ = C::NQ, NA = C::NA, KP = TC::KP, NN = TC::NN;
  constexpr int NW = NT / 32;
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  char* sXh = reinterpret_cast<char*>(smem + TC::S_X);
  char* sXl = sXh + TC::XBYTES;
  float* sY = smem + TC::S_Y;
  float* sFt = smem + TC::S_FT;
  float* sFh = smem + TC::S_FH;
  float* sA = smem + TC::S_A;
  float* sFl = smem + TC::S_FL;
  float* sE = smem + TC::S_E;
  int* sMeta = reinterpret_cast<int*>(smem + TC::S_META);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + TC::S_BAR);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(smem + TC::S_BAR + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int i = tid; i < 4 * B * F; i += NT) sFt[i] = ops.Ft[i];
  for (int i = tid; i < 4 * F * B; i += NT) sFh[i] = ops.Fh[i];
  // both X copies start at zero: the padding modes (>= B) and rows (>= 9 NE) stay zero
  for (int i = tid; i < 2 * TC::XBYTES / 4; i += NT) smem[TC::S_X + i] = 0.f;
  if (warp == 0) {
    tc::tmem_alloc(taddr_s, TC::COLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *taddr_s;
  // ---- constant A operands into tensor memory, split into tf32 hi / lo: row (c, b) =
  // c B + b; time kernel A[(c,b)][k] = K_c[b][k], volume A[(c,b)][k] = K_c[k][b]. Warp w
  // writes the lanes of its quadrant (w < 4).
  if (warp < 4) {
    const int m = warp * 32 + lane;
    const int c = m / B, bb = m % B;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int which = 0; which < 2; ++which) {
#pragma unroll 1
      for (int k0 = 0; k0 < KP; k0 += 8) {
        float hi[8], lo[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int k = k0 + jj;
          float a = 0.f;
          if (m < 3 * B && k < B) a = (which == 0) ? ops.K[(c * B + bb) * B + k] : ops.K[(c * B + k) * B + bb];
          tc::tf32_split(a, hi[jj], lo[jj]);
        }
        const int col = (which == 0) ? TC::T_ACK : TC::T_AVOL;
        tc::tmem_st8(lane_base + col + k0, hi);
        tc::tmem_st8(lane_base + col + KP + k0, lo);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();

  int e = -1, b = 0, p = 0;
  task_of<O, NE, (FG > 1)>(tid, e, b, p);
  const bool act = e >= 0;
  const int es = act ? e : 0;
  const int fmax = nface(p + 1);
  int fe = -1, fi = 0, ff = 0, fpf = 0;
  const int nelem = ph.end - ph.begin;
  const long long qs = (FG > 1) ? st.qs : C::QS, bs = (FG > 1) ? st.bs : C::BUFS;
  const int nsim = (FG > 1) ? st.nsim : 1;
  const int nsg = nsim / FG;
  const int nbatch = (FG > 1) ? nelem * nsg : (nelem + NE - 1) / NE;
  constexpr int rs = B * FG;
  uint32_t phase = 0;

  // X rows of this thread: n = es * 9 + r at mode k = b, split into the hi / lo copies
  auto stage_x = [&](const float* vals) {
#pragma unroll
    for (int r = 0; r < 9; ++r) {
      const int n = es * 9 + r;
      const int off = (n >> 3) * TC::SBO + (b >> 2) * TC::LBO + (n & 7) * 16 + (b & 3) * 4;
      float hi, lo;
      tc::tf32_split(vals[r], hi, lo);
      *reinterpret_cast<float*>(sXh + off) = hi;
      *reinterpret_cast<float*>(sXl + off) = lo;
    }
  };
  // One MMA chain with A at tensor-memory column a_col, issued by thread 0 after a barrier
  // that publishes the staged X (and anything else written to shared memory before it).
  auto issue = [&](int a_col) {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    // suppress_commit (failure-path test): nothing is issued, so the wait below runs out
    if (tid == 0 && !suppress_commit) {
      tc::fence_after_sync();
      constexpr uint32_t idesc = tc::idesc_tf32(128, NN);
      const uint32_t xh = tc::smem_u32(sXh), xl = tc::smem_u32(sXl);
      uint32_t acc = 0;
      for (int pass = 0; pass < passes; ++pass) {
        const uint32_t xb = (pass == 1) ? xl : xh;                          // pass 1: A_hi X_lo
        const uint32_t at = tmem + a_col + ((pass == 2) ? KP : 0);          // pass 2: A_lo X_hi
#pragma unroll
        for (int s = 0; s < KP / 8; ++s) {
          tc::mma_tf32_ts(tmem + TC::T_D, at + 8 * s, tc::smem_desc(xb + s * 2 * TC::LBO, TC::LBO, TC::SBO), idesc,
                          acc);
          acc = 1;
        }
      }
      tc::commit(bar);
    }
  };
  // Wait for the chain, then move D to sY[(slot B + b) 27 + c 9 + r] (lanes (c, b), columns
  // (slot, r); the column map is resolved at compile time) and end with a barrier.
  // Returns false (in every thread) if the chain did not complete within the bounded wait.
  auto finish = [&]() -> bool {
    bool ok = tc::mbar_wait(bar, phase, wait_cycles);
    ok = __all_sync(0xffffffffu, ok);
    phase ^= 1u;
    tc::fence_after_sync();
    if (ok) {
      constexpr int CW = TC::CW;
      const int q = warp & 3;
      const int m = 32 * q + lane;
      const int c = m / B, bb = m % B;
      const int nwq = (NW - q + 3) / 4;               // warps sharing this lane quadrant
      float* yb = sY + bb * TC::YS + c * 9;
      const bool has_row = m < 3 * B;
#pragma unroll
      for (int ch = 0; ch < NN / CW; ++ch) {
        if (ch % nwq != (warp >> 2)) continue;
        float v[CW];
        if constexpr (CW == 32)
          tc::tmem_ld32(tmem + TC::T_D + ((uint32_t)(32 * q) << 16) + CW * ch, v);
        else
          tc::tmem_ld16(tmem + TC::T_D + ((uint32_t)(32 * q) << 16) + CW * ch, v);
        if (has_row) {
#pragma unroll
          for (int jj = 0; jj < CW; ++jj) {
            const int n = CW * ch + jj;
            if (n < 9 * NE) yb[(n / 9) * B * TC::YS + (n % 9)] = v[jj];
          }
        }
      }
    }
    tc::fence_before_sync();
    return __syncthreads_or(!ok) == 0;
  };
  auto contract = [&](int a_col) -> bool {
    issue(a_col);
    return finish();
  };
  auto read_y = [&](float (&Y)[3][9]) {
    const float* y = sY + (es * B + b) * TC::YS;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < 9; ++r) Y[c][r] = y[c * 9 + r];
  };

  bool alive = true;
  for (int batch = blockIdx.x; alive && batch < nbatch; batch += gridDim.x) {
    const int e0 = (FG > 1) ? ph.begin + batch / nsg : ph.begin + batch * NE;
    const int grp = (FG > 1) ? batch % nsg : 0;
    __syncthreads();
    const int g = e0 + ((FG > 1) ? 0 : e);
    const int eb = (FG > 1) ? 0 : es;
    const int j = (FG > 1) ? es : 0;
    const bool valid = act && g < ph.end;
    const size_t qoff = (size_t)g * qs + (size_t)grp * (NQ * B * FG) + b * FG + j;
    const size_t boff = (size_t)g * bs + (size_t)grp * (9 * B * FG) + b * FG + j;
    float T[NQ], Th[9], Da[NA > 0 ? NA : 1];
    float v[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) v[r] = 0.f;
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
    const float* ed = sE + eb * ED;
    if (act) stage_x(v);
    __syncthreads();
    const int meta = act ? sMeta[eb] : 0;
    const int cl = meta & 0xff;
#pragma unroll
    for (int r = 0; r < 9; ++r) {
      T[r] = ph.coef[cl][0] * v[r];
      Th[r] = ph.hcoef[cl][0] * v[r];
    }
#pragma unroll
    for (int r = 0; r < NA; ++r) T[9 + r] = ph.coef[cl][0] * Da[r];
    // ---- time kernel (Cauchy-Kowalevski), Taylor sums
#pragma unroll 1
    for (int d = 0; d < O - 1; ++d) {
      if (!contract(TC::T_ACK)) {
        alive = false;
        break;
      }
      if (act) {
        float Y[3][9];
        read_y(Y);
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
        stage_x(out);
      }
    }
    if (!alive) break;
    // ---- volume kernel: T staged for the MMA and (rows of 12) for the surface kernel; the
    // volume MMA runs while the LTS buffers are written and the local surface kernel runs
    if (act) {
      stage_x(T);
      float* a = sA + (es * B + b) * AR;
      st4(a, T[0], T[1], T[2], T[3]);
      st4(a + 4, T[4], T[5], T[6], T[7]);
      st4(a + 8, T[8], 0.f, 0.f, 0.f);
    }
    issue(TC::T_AVOL);
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
    // ---- local surface kernel: G_i = T^e F~_i, flux, staged for F^
#pragma unroll 1
    for (int t = tid; t < NE * 4 * F; t += NT) {
      face_task_of<O, NE, (FG > 1)>(t, fe, fi, ff, fpf);
      float gq[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) gq[r] = 0.f;
      const float* Ab = sA + fe * B * AR;
      const float* Fi = sFt + fi * B * F + ff;
#pragma unroll 4
      for (int k = nbasis(fpf); k < B; ++k) {
        const float4 x0 = *reinterpret_cast<const float4*>(Ab + k * AR);
        const float4 x1 = *reinterpret_cast<const float4*>(Ab + k * AR + 4);
        const float x8 = Ab[k * AR + 8];
        const float w = Fi[k * F];
        gq[0] = fmaf(x0.x, w, gq[0]);
        gq[1] = fmaf(x0.y, w, gq[1]);
        gq[2] = fmaf(x0.z, w, gq[2]);
        gq[3] = fmaf(x0.w, w, gq[3]);
        gq[4] = fmaf(x1.x, w, gq[4]);
        gq[5] = fmaf(x1.y, w, gq[5]);
        gq[6] = fmaf(x1.z, w, gq[6]);
        gq[7] = fmaf(x1.w, w, gq[7]);
        gq[8] = fmaf(x8, w, gq[8]);
      }
      float w6[6];
      riemann_state(gq, sE + ((FG > 1) ? 0 : fe) * ED + 20 + 11 * fi, w6);
      store_state(sFl + fe * C::FLS + (fi * F + ff) * FR, w6);
    }
    // the volume chain's barrier also publishes the staged Riemann states
    if (!finish()) {
      alive = false;
      break;
    }
    float acc[NQ];
    if (valid) {
      const float* q = st.Q + qoff;
#pragma unroll
      for (int r = 0; r < NQ; ++r) acc[r] = q[r * rs];
      float Z[3][9];
      read_y(Z);
      float out[9], eps[6];
      star_apply(Z, ed, out, eps);
      float V[9];
#pragma unroll
      for (int r = 0; r < 9; ++r) V[r] = -out[r];
#pragma unroll
      for (int l = 0; l < M; ++l) coupling_add(V, T + 9 + 6 * l, ed[12 + 2 * l], ed[13 + 2 * l]);
#pragma unroll
      for (int r = 0; r < 9; ++r) acc[r] += V[r];
#pragma unroll
      for (int l = 0; l < M; ++l)
#pragma unroll
        for (int r = 0; r < 6; ++r) acc[9 + 6 * l + r] += ph.omega[l] * (-eps[r] - T[9 + 6 * l + r]);
    }
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
  }
  if (!alive && tid == 0) atomicOr(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TC::COLS);
}

}  // namespace ltsdev
