// Attenuation fit and rate-2 clustering (Sec. V-A).
#include <cmath>
#include <limits>

#include "host.h"

namespace lts {

void relaxation_frequencies(int m, double f_min, double f_max, double* omega) {
  const double two_pi = 6.283185307179586476925286766559;
  if (m == 1) {
    omega[0] = two_pi * std::sqrt(f_min * f_max);
    return;
  }
  for (int l = 0; l < m; ++l) omega[l] = two_pi * f_min * std::pow(f_max / f_min, l / (m - 1.0));
}

// Y_l for a constant target Q: collocation of
//   Q^-1 = sum_l Y_l (omega_l w + omega_l^2 Q^-1) / (omega_l^2 + w^2)   at w = omega_k
// (the generalised Maxwell body modulus M_u (1 - sum_l Y_l omega_l / (omega_l + i w))),
// solved by Gaussian elimination with partial pivoting.
int fit_y(int m, double q, const double* omega, double* y) {
  if (std::isinf(q)) {
    for (int l = 0; l < m; ++l) y[l] = 0.0;
    return 0;
  }
  double qi = 1.0 / q;
  std::vector<double> A(m * (m + 1));
  for (int k = 0; k < m; ++k) {
    for (int l = 0; l < m; ++l) {
      double wl = omega[l], wk = omega[k];
      A[k * (m + 1) + l] = (wl * wk + wl * wl * qi) / (wl * wl + wk * wk);
    }
    A[k * (m + 1) + m] = qi;
  }
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(A[r * (m + 1) + c]) > std::fabs(A[piv * (m + 1) + c])) piv = r;
    if (A[piv * (m + 1) + c] == 0.0) return -1;
    if (piv != c)
      for (int t = 0; t <= m; ++t) std::swap(A[c * (m + 1) + t], A[piv * (m + 1) + t]);
    for (int r = c + 1; r < m; ++r) {
      double f = A[r * (m + 1) + c] / A[c * (m + 1) + c];
      for (int t = c; t <= m; ++t) A[r * (m + 1) + t] -= f * A[c * (m + 1) + t];
    }
  }
  for (int r = m - 1; r >= 0; --r) {
    double s = A[r * (m + 1) + m];
    for (int t = r + 1; t < m; ++t) s -= A[r * (m + 1) + t] * y[t];
    y[r] = s / A[r * (m + 1) + r];
  }
  return 0;
}

void cfl_time_steps(const Mesh& m, const Material& mat, int order, double cfl, std::vector<double>& dt) {
  dt.resize(m.K);
  for (int64_t k = 0; k < m.K; ++k) dt[k] = cfl * m.dins[k] / ((2.0 * order - 1.0) * mat.vp[k]);
}

void assign_clusters(const std::vector<double>& dt, double lam, int nc, std::vector<int32_t>& c) {
  double dmin = std::numeric_limits<double>::infinity();
  for (double v : dt) dmin = std::min(dmin, v);
  double base = lam * dmin;
  c.assign(dt.size(), 0);
  for (size_t k = 0; k < dt.size(); ++k) {
    int l = 0;
    while (l + 1 < nc && dt[k] >= base * std::ldexp(1.0, l + 1)) ++l;
    c[k] = l;
  }
}

void normalise_clusters(const Mesh& m, std::vector<int32_t>& c) {
  // fixed point of c(k) <- min(c(k), min_nbr c(nbr) + 1), in Jacobi sweeps
  std::vector<int32_t> nxt(c.size());
  for (;;) {
    bool changed = false;
    for (int64_t k = 0; k < m.K; ++k) {
      int32_t v = c[k];
      for (int f = 0; f < 4; ++f) {
        int64_t nb = m.nbr[4 * k + f];
        if (nb >= 0) v = std::min(v, c[nb] + 1);
      }
      nxt[k] = v;
      changed |= (v != c[k]);
    }
    c.swap(nxt);
    if (!changed) return;
  }
}

double theoretical_speedup(const std::vector<int32_t>& c, double lam) {
  double s = 0.0;
  for (int32_t v : c) s += std::ldexp(1.0, -v);
  return c.size() * lam / s;
}

double search_lambda(const Mesh& m, const std::vector<double>& dt, int nc, std::vector<int32_t>& c, double* speedup) {
  double best_lam = 1.0, best_s = -1.0;
  std::vector<int32_t> cur;
  for (int i = 51; i <= 100; ++i) {
    double lam = i / 100.0;
    assign_clusters(dt, lam, nc, cur);
    normalise_clusters(m, cur);
    double s = theoretical_speedup(cur, lam);
    if (s >= best_s) {
      best_s = s;
      best_lam = lam;
      c = cur;
    }
  }
  if (speedup) *speedup = best_s;
  return best_lam;
}

}  // namespace lts
