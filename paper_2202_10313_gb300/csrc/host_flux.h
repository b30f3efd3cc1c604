// Closed forms of the per-element operators, templated on the scalar type so that the
// forward set-up (double) and the adjoint's material derivatives (forward-mode dual
// numbers) evaluate the same expressions.
//
// Flux coefficients of one face (Sec. III-A flux solvers, upwind Riemann state in the
// impedance form): interior state (a[4], b[4]) and exterior state (an[4], bn[4]), scaled
// by -2|S|/|det J|. Normal (P) and tangential (S) pairs:
//   v* = (Z- v- + Z+ v+ + t+ - t-)/(Z- + Z+),  t* = (Z+ t- + Z- t+ + Z- Z+ (v+ - v-))/(Z- + Z+)
// free surface: t* = 0, v* = v- - t-/Z-; absorbing: exterior state zero, Z+ = Z-.
#pragma once
#include <cmath>

#include "../../include/ader_lts.h"

// host and device (the adjoint's material-gradient contraction runs on the GPU)
#ifdef __CUDACC__
#define LTS_HD __host__ __device__
#else
#define LTS_HD
#endif

namespace lts {

template <typename T>
LTS_HD void face_coefficients_t(int bc, T zp_i, T zs_i, T zp_o, T zs_o, T scale, T* loc, T* nbc) {
  T a[4], b[4], an[4], bn[4];
  if (bc == LTS_BC_FREE_SURFACE) {
    a[0] = T(1.0); a[1] = T(-1.0) / zp_i; a[2] = T(0.0); a[3] = T(0.0);
    b[0] = T(1.0); b[1] = T(-1.0) / zs_i; b[2] = T(0.0); b[3] = T(0.0);
    for (int i = 0; i < 4; ++i) an[i] = bn[i] = T(0.0);
  } else {
    if (bc == LTS_BC_ABSORBING) {
      zp_o = zp_i;
      zs_o = zs_i;
    }
    const T sp = zp_i + zp_o, ss = zs_i + zs_o;
    a[0] = zp_i / sp; a[1] = T(-1.0) / sp; a[2] = zp_o / sp; a[3] = -(zp_i * zp_o) / sp;
    b[0] = zs_i / ss; b[1] = T(-1.0) / ss; b[2] = zs_o / ss; b[3] = -(zs_i * zs_o) / ss;
    an[0] = zp_o / sp; an[1] = T(1.0) / sp; an[2] = zp_i / sp; an[3] = (zp_i * zp_o) / sp;
    bn[0] = zs_o / ss; bn[1] = T(1.0) / ss; bn[2] = zs_i / ss; bn[3] = (zs_i * zs_o) / ss;
    if (bc == LTS_BC_ABSORBING)
      for (int i = 0; i < 4; ++i) an[i] = bn[i] = T(0.0);
  }
  for (int i = 0; i < 4; ++i) {
    loc[i] = scale * a[i];
    loc[4 + i] = scale * b[i];
    nbc[i] = scale * an[i];
    nbc[4 + i] = scale * bn[i];
  }
}

// Interface state (v*, t*) from a face trace g (9 values) and the 8 coefficients c of one
// side, then the flux rows it adds: S -= flux(w) with the interior element's lam, mu,
// 1/rho (the forward kernels' riemann_state and flux_rows_add).
template <typename T>
LTS_HD void face_flux_apply(const T g[9], const double n[3], const T c[8], T lam, T mu, T rinv, T S[9]) {
  const double nx = n[0], ny = n[1], nz = n[2];
  const T tx = g[0] * nx + g[3] * ny + g[5] * nz;
  const T ty = g[3] * nx + g[1] * ny + g[4] * nz;
  const T tz = g[5] * nx + g[4] * ny + g[2] * nz;
  const T tn = tx * nx + ty * ny + tz * nz;
  const T vn = g[6] * nx + g[7] * ny + g[8] * nz;
  const T tTx = tx - tn * nx, tTy = ty - tn * ny, tTz = tz - tn * nz;
  const T vTx = g[6] - vn * nx, vTy = g[7] - vn * ny, vTz = g[8] - vn * nz;
  const T vsn = c[0] * vn + c[1] * tn;
  const T tsn = c[2] * tn + c[3] * vn;
  T w[6];
  w[0] = vsn * nx + c[4] * vTx + c[5] * tTx;
  w[1] = vsn * ny + c[4] * vTy + c[5] * tTy;
  w[2] = vsn * nz + c[4] * vTz + c[5] * tTz;
  w[3] = tsn * nx + c[6] * tTx + c[7] * vTx;
  w[4] = tsn * ny + c[6] * tTy + c[7] * vTy;
  w[5] = tsn * nz + c[6] * tTz + c[7] * vTz;
  const T nv = w[0] * nx + w[1] * ny + w[2] * nz;
  const T exx = w[0] * nx, eyy = w[1] * ny, ezz = w[2] * nz;
  const T exy = w[1] * nx + w[0] * ny, eyz = w[2] * ny + w[1] * nz, exz = w[2] * nx + w[0] * nz;
  const T ln = lam * nv, m2 = T(2.0) * mu;
  S[0] = S[0] - (ln + m2 * exx);
  S[1] = S[1] - (ln + m2 * eyy);
  S[2] = S[2] - (ln + m2 * ezz);
  S[3] = S[3] - mu * exy;
  S[4] = S[4] - mu * eyz;
  S[5] = S[5] - mu * exz;
  S[6] = S[6] - rinv * w[3];
  S[7] = S[7] - rinv * w[4];
  S[8] = S[8] - rinv * w[5];
}

// 9 x 9 matrix of the face map g -> S (row-major [out][in]).
template <typename T>
LTS_HD void face_flux_matrix(const double n[3], const T c[8], T lam, T mu, T rinv, T M[81]) {
  for (int j = 0; j < 9; ++j) {
    T g[9], S[9];
    for (int q = 0; q < 9; ++q) {
      g[q] = T(q == j ? 1.0 : 0.0);
      S[q] = T(0.0);
    }
    face_flux_apply(g, n, c, lam, mu, rinv, S);
    for (int q = 0; q < 9; ++q) M[q * 9 + j] = S[q];
  }
}

// sum_{q,j} M[q][j] W[q*9 + j] of that matrix, column by column (no 9 x 9 storage).
template <typename T>
LTS_HD T face_flux_dot(const double n[3], const T c[8], T lam, T mu, T rinv, const double* W) {
  T acc(0.0);
  for (int j = 0; j < 9; ++j) {
    T g[9], S[9];
    for (int q = 0; q < 9; ++q) {
      g[q] = T(q == j ? 1.0 : 0.0);
      S[q] = T(0.0);
    }
    face_flux_apply(g, n, c, lam, mu, rinv, S);
    for (int q = 0; q < 9; ++q) acc = acc + S[q] * W[q * 9 + j];
  }
  return acc;
}

// Voigt index of the stress component (i, d).
LTS_HD inline int voigt(int i, int d) {
  return i == d ? i : ((i + d == 1) ? 3 : ((i + d == 3) ? 4 : 5));
}

// The terms of the star matrices (below), each handed to add(c, out * 9 + in, term); an
// entry may receive several terms.
template <typename T, typename Add>
LTS_HD void star_terms_t(const double jinv[9], T lam, T mu, T rinv, Add&& add) {
  for (int c = 0; c < 3; ++c) {
    // stress rows from the velocity gradient g[d][j] = sum_c jinv[c][d] Y_c[6+j]
    for (int d = 0; d < 3; ++d)
      for (int j = 0; j < 3; ++j) {
        const double w = jinv[c * 3 + d];     // dg[d][j] / dY_c[6+j]
        const int col = 6 + j;
        // tr = g00 + g11 + g22
        if (d == j) {
          for (int a = 0; a < 3; ++a) add(c, a * 9 + col, lam * w);
          add(c, d * 9 + col, T(2.0) * mu * w);
        } else {
          // out[3] = mu (g01 + g10), out[4] = mu (g12 + g21), out[5] = mu (g02 + g20)
          add(c, voigt(d, j) * 9 + col, mu * w);
        }
      }
    // velocity rows: rinv * sum_d jinv[c][d] Y_c[SIG[i][d]]
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < 3; ++d) add(c, (6 + i) * 9 + voigt(i, d), rinv * jinv[c * 3 + d]);
  }
}

// Star matrices S_c (row-major [out][in]) of the time kernel's map D_{d+1} = sum_c S_c Y_c,
// Y_c = D_d K_c^T (the forward kernels' star_apply: physical velocity gradient W_d =
// sum_c dxi_c/dx_d Y_c, Hooke's law on the stress rows, stress divergence / rho on the
// velocity rows). jinv[c*3+d] = dxi_c/dx_d.
template <typename T>
LTS_HD void star_matrices_t(const double jinv[9], T lam, T mu, T rinv, T S[3][81]) {
  for (int c = 0; c < 3; ++c)
    for (int q = 0; q < 81; ++q) S[c][q] = T(0.0);
  star_terms_t<T>(jinv, lam, mu, rinv, [&](int c, int q, T v) { S[c][q] = S[c][q] + v; });
}

// sum_c sum_q S_c[q] W[c*81 + q] of the star matrices.
template <typename T>
LTS_HD T star_dot(const double jinv[9], T lam, T mu, T rinv, const double* W) {
  T acc(0.0);
  star_terms_t<T>(jinv, lam, mu, rinv, [&](int c, int q, T v) { acc = acc + v * W[c * 81 + q]; });
  return acc;
}

// Forward-mode dual number with one derivative component.
struct Dual {
  double v, d;
  LTS_HD Dual(double x = 0.0, double dx = 0.0) : v(x), d(dx) {}
};
LTS_HD inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
LTS_HD inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
LTS_HD inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
LTS_HD inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
LTS_HD inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
LTS_HD inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
LTS_HD inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
LTS_HD inline double sqrt_d(double a) {
#ifdef __CUDA_ARCH__
  return ::sqrt(a);
#else
  return std::sqrt(a);
#endif
}
LTS_HD inline Dual sqrt_t(Dual a) {
  const double s = sqrt_d(a.v);
  return Dual(s, a.d / (2.0 * s));
}
LTS_HD inline double sqrt_t(double a) { return sqrt_d(a); }

}  // namespace lts
