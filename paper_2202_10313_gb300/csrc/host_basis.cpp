// Reference operators by exact polynomial algebra.
//
// Each basis function is expanded into monomials xi1^a xi2^b xi3^c (dense table up to
// degree 2*(O-1)); products, derivatives and face restrictions stay polynomials, and
// integrals over the reference tetrahedron / triangle are exact:
//   int_tet xi1^a xi2^b xi3^c = a! b! c! / (a+b+c+3)!,   int_tri chi1^a chi2^b = a! b! / (a+b+2)!.
// The projection quadrature is a collapsed Gauss-Jacobi rule whose nodes come from
// Newton iteration on Jacobi polynomials.
#include <cmath>
#include <stdexcept>

#include "host.h"

namespace lts {

int n_basis(int o) { return o * (o + 1) * (o + 2) / 6; }
int n_face_basis(int o) { return o * (o + 1) / 2; }

namespace {

// ---------------------------------------------------------------- 3-variable polynomials
struct P3 {
  int D;                        // max degree stored
  std::vector<double> c;        // c[(a*(D+1)+b)*(D+1)+cc]
  explicit P3(int d = 0) : D(d), c((d + 1) * (d + 1) * (d + 1), 0.0) {}
  double& at(int a, int b, int cc) { return c[(a * (D + 1) + b) * (D + 1) + cc]; }
  double at(int a, int b, int cc) const { return c[(a * (D + 1) + b) * (D + 1) + cc]; }
};

P3 p3_const(int D, double v) { P3 p(D); p.at(0, 0, 0) = v; return p; }
P3 p3_var(int D, int var) {
  P3 p(D);
  if (var == 0) p.at(1, 0, 0) = 1.0;
  if (var == 1) p.at(0, 1, 0) = 1.0;
  if (var == 2) p.at(0, 0, 1) = 1.0;
  return p;
}
P3 operator+(const P3& x, const P3& y) { P3 r(x.D); for (size_t i = 0; i < r.c.size(); ++i) r.c[i] = x.c[i] + y.c[i]; return r; }
P3 operator-(const P3& x, const P3& y) { P3 r(x.D); for (size_t i = 0; i < r.c.size(); ++i) r.c[i] = x.c[i] - y.c[i]; return r; }
P3 operator*(double s, const P3& x) { P3 r(x.D); for (size_t i = 0; i < r.c.size(); ++i) r.c[i] = s * x.c[i]; return r; }
P3 mul(const P3& x, const P3& y) {
  P3 r(x.D);
  const int D = x.D;
  for (int a = 0; a <= D; ++a)
    for (int b = 0; a + b <= D; ++b)
      for (int c = 0; a + b + c <= D; ++c) {
        double xv = x.at(a, b, c);
        if (xv == 0.0) continue;
        for (int a2 = 0; a + a2 <= D; ++a2)
          for (int b2 = 0; a + a2 + b + b2 <= D; ++b2)
            for (int c2 = 0; a + a2 + b + b2 + c + c2 <= D; ++c2) {
              double yv = y.at(a2, b2, c2);
              if (yv != 0.0) r.at(a + a2, b + b2, c + c2) += xv * yv;
            }
      }
  return r;
}
P3 deriv(const P3& x, int var) {
  P3 r(x.D);
  for (int a = 0; a <= x.D; ++a)
    for (int b = 0; a + b <= x.D; ++b)
      for (int c = 0; a + b + c <= x.D; ++c) {
        double v = x.at(a, b, c);
        if (v == 0.0) continue;
        if (var == 0 && a > 0) r.at(a - 1, b, c) += a * v;
        if (var == 1 && b > 0) r.at(a, b - 1, c) += b * v;
        if (var == 2 && c > 0) r.at(a, b, c - 1) += c * v;
      }
  return r;
}
double fact(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; }
double integrate_tet(const P3& x) {
  double s = 0.0;
  for (int a = 0; a <= x.D; ++a)
    for (int b = 0; a + b <= x.D; ++b)
      for (int c = 0; a + b + c <= x.D; ++c) {
        double v = x.at(a, b, c);
        if (v != 0.0) s += v * fact(a) * fact(b) * fact(c) / fact(a + b + c + 3);
      }
  return s;
}
double eval3(const P3& x, const double* xi) {
  double s = 0.0;
  for (int a = 0; a <= x.D; ++a)
    for (int b = 0; a + b <= x.D; ++b)
      for (int c = 0; a + b + c <= x.D; ++c) {
        double v = x.at(a, b, c);
        if (v != 0.0) s += v * std::pow(xi[0], a) * std::pow(xi[1], b) * std::pow(xi[2], c);
      }
  return s;
}

// ---------------------------------------------------------------- 2-variable polynomials
struct P2 {
  int D;
  std::vector<double> c;   // c[a*(D+1)+b]
  explicit P2(int d = 0) : D(d), c((d + 1) * (d + 1), 0.0) {}
  double& at(int a, int b) { return c[a * (D + 1) + b]; }
  double at(int a, int b) const { return c[a * (D + 1) + b]; }
};
P2 mul2(const P2& x, const P2& y) {
  P2 r(x.D);
  for (int a = 0; a <= x.D; ++a)
    for (int b = 0; a + b <= x.D; ++b) {
      double xv = x.at(a, b);
      if (xv == 0.0) continue;
      for (int a2 = 0; a + a2 <= x.D; ++a2)
        for (int b2 = 0; a + a2 + b + b2 <= x.D; ++b2) r.at(a + a2, b + b2) += xv * y.at(a2, b2);
    }
  return r;
}
double integrate_tri(const P2& x) {
  double s = 0.0;
  for (int a = 0; a <= x.D; ++a)
    for (int b = 0; a + b <= x.D; ++b)
      if (x.at(a, b) != 0.0) s += x.at(a, b) * fact(a) * fact(b) / fact(a + b + 2);
  return s;
}
// substitute xi_i = alpha_i + beta_i chi1 + gamma_i chi2 into a P3 -> P2 (degree D)
P2 restrict_to_face(const P3& p, const double alpha[3], const double beta[3], const double gamma[3]) {
  const int D = p.D;
  // powers of each affine form
  std::vector<P2> pw[3];
  for (int i = 0; i < 3; ++i) {
    P2 lin(D);
    lin.at(0, 0) = alpha[i];
    if (D >= 1) { lin.at(1, 0) = beta[i]; lin.at(0, 1) = gamma[i]; }
    P2 one(D);
    one.at(0, 0) = 1.0;
    pw[i].push_back(one);
    for (int k = 1; k <= D; ++k) pw[i].push_back(mul2(pw[i].back(), lin));
  }
  P2 r(D);
  for (int a = 0; a <= D; ++a)
    for (int b = 0; a + b <= D; ++b)
      for (int c = 0; a + b + c <= D; ++c) {
        double v = p.at(a, b, c);
        if (v == 0.0) continue;
        P2 t = mul2(mul2(pw[0][a], pw[1][b]), pw[2][c]);
        for (size_t q = 0; q < r.c.size(); ++q) r.c[q] += v * t.c[q];
      }
  return r;
}

// s^n P_n^(alpha,0)(x/s) for n = 0..nmax, as polynomials (x, s given as polynomials)
template <class P, class Mul>
std::vector<P> jacobi_h(int nmax, double alpha, const P& x, const P& s, const P& one, Mul mulf) {
  std::vector<P> out;
  out.push_back(one);
  if (nmax >= 1) out.push_back(0.5 * ((alpha + 2.0) * x + alpha * s));
  for (int n = 2; n <= nmax; ++n) {
    double a1 = 2.0 * n * (n + alpha) * (2.0 * n + alpha - 2.0);
    double a2 = 2.0 * n + alpha - 1.0;
    double a3 = (2.0 * n + alpha) * (2.0 * n + alpha - 2.0);
    double a4 = 2.0 * (n + alpha - 1.0) * (n - 1.0) * (2.0 * n + alpha);
    P t1 = mulf(a2 * (a3 * x + (alpha * alpha) * s), out[n - 1]);
    P t2 = mulf(mulf(s, s), out[n - 2]);
    out.push_back((1.0 / a1) * (t1 - a4 * t2));
  }
  return out;
}
P2 operator+(const P2& x, const P2& y) { P2 r(x.D); for (size_t i = 0; i < r.c.size(); ++i) r.c[i] = x.c[i] + y.c[i]; return r; }
P2 operator-(const P2& x, const P2& y) { P2 r(x.D); for (size_t i = 0; i < r.c.size(); ++i) r.c[i] = x.c[i] - y.c[i]; return r; }
P2 operator*(double s, const P2& x) { P2 r(x.D); for (size_t i = 0; i < r.c.size(); ++i) r.c[i] = s * x.c[i]; return r; }

const double kRefV[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
const int kFaceV[4][3] = {{0, 2, 1}, {0, 1, 3}, {0, 3, 2}, {1, 2, 3}};

double jacobi_eval(int n, double a, double b, double x, double* dp) {
  // general Jacobi P_n^(a,b)(x) and derivative by the standard recurrence
  double p0 = 1.0, p1 = 0.5 * (a - b + (a + b + 2.0) * x);
  if (n == 0) { if (dp) *dp = 0.0; return 1.0; }
  double pm = p0, p = p1;
  for (int k = 2; k <= n; ++k) {
    double c = 2.0 * k + a + b;
    double a1 = 2.0 * k * (k + a + b) * (c - 2.0);
    double a2 = (c - 1.0) * (a * a - b * b);
    double a3 = (c - 2.0) * (c - 1.0) * c;
    double a4 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * c;
    double pn = ((a2 + a3 * x) * p - a4 * pm) / a1;
    pm = p;
    p = pn;
  }
  if (dp) {
    // d/dx P_n^(a,b) = (n+a+b+1)/2 P_{n-1}^(a+1,b+1)
    *dp = 0.5 * (n + a + b + 1.0) * jacobi_eval(n - 1, a + 1.0, b + 1.0, x, nullptr);
  }
  return p;
}

}  // namespace

void gauss_jacobi(int n, double alpha, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    // Chebyshev-like initial guess, refined by Newton with deflation of found roots
    double r = -std::cos((2.0 * i + 1.0) * pi / (2.0 * n));
    if (i > 0 && r <= x[i - 1]) r = 0.5 * (x[i - 1] + 1.0);
    for (int it = 0; it < 100; ++it) {
      double dp;
      double p = jacobi_eval(n, alpha, 0.0, r, &dp);
      double s = 0.0;
      for (int j = 0; j < i; ++j) s += 1.0 / (r - x[j]);
      double dr = p / (dp - s * p);
      r -= dr;
      if (std::fabs(dr) < 1e-16) break;
    }
    x[i] = r;
  }
  for (int i = 0; i < n; ++i) {
    double dp;
    jacobi_eval(n, alpha, 0.0, x[i], &dp);
    w[i] = std::pow(2.0, alpha + 1.0) / ((1.0 - x[i] * x[i]) * dp * dp);
  }
}

void RefOps::build(int o) {
  order = o;
  B = n_basis(o);
  F = n_face_basis(o);
  deg = o - 1;
  const int D = 2 * deg;        // room for products
  // modes in storage order: degree p, then k, then j (i = p - j - k)
  std::vector<std::array<int, 3>> modes;
  for (int p = 0; p < o; ++p)
    for (int k = 0; k <= p; ++k)
      for (int j = 0; j <= p - k; ++j) modes.push_back({p - j - k, j, k});
  P3 one = p3_const(D, 1.0);
  P3 x1 = p3_var(D, 0), x2 = p3_var(D, 1), x3 = p3_var(D, 2);
  P3 s1 = one - x2 - x3, s2 = one - x3;
  auto m3 = [](const P3& a, const P3& b) { return mul(a, b); };
  std::vector<P3> phi;
  degree.clear();
  for (auto& md : modes) {
    int i = md[0], j = md[1], k = md[2];
    P3 hi = jacobi_h(i, 0.0, 2.0 * x1 - s1, s1, one, m3)[i];
    P3 hj = jacobi_h(j, 2.0 * i + 1.0, 2.0 * x2 - s2, s2, one, m3)[j];
    P3 hk = jacobi_h(k, 2.0 * i + 2.0 * j + 2.0, 2.0 * x3 - one, one, one, m3)[k];
    P3 f = mul(mul(hi, hj), hk);
    double nrm = std::sqrt(integrate_tet(mul(f, f)));
    phi.push_back((1.0 / nrm) * f);
    degree.push_back(i + j + k);
  }
  poly.clear();
  for (auto& p : phi) poly.push_back(p.c);
  // triangle basis psi_ij, ordered by degree then j
  P2 one2(D);
  one2.at(0, 0) = 1.0;
  P2 c1(D), c2(D);
  c1.at(1, 0) = 1.0;
  c2.at(0, 1) = 1.0;
  P2 s = one2 - c2;
  auto m2 = [](const P2& a, const P2& b) { return mul2(a, b); };
  std::vector<P2> psi;
  for (int p = 0; p < o; ++p)
    for (int j = 0; j <= p; ++j) {
      int i = p - j;
      P2 hi = jacobi_h(i, 0.0, 2.0 * c1 - s, s, one2, m2)[i];
      P2 hj = jacobi_h(j, 2.0 * i + 1.0, 2.0 * c2 - one2, one2, one2, m2)[j];
      P2 f = mul2(hi, hj);
      double nrm = std::sqrt(integrate_tri(mul2(f, f)));
      psi.push_back((1.0 / nrm) * f);
    }
  // K_c[i][j] = int phi_i d phi_j / d xi_c
  for (int c = 0; c < 3; ++c) {
    K[c].assign(B * B, 0.0);
    for (int j = 0; j < B; ++j) {
      P3 dj = deriv(phi[j], c);
      for (int i = 0; i < B; ++i) K[c][i * B + j] = integrate_tet(mul(phi[i], dj));
    }
  }
  // face maps
  auto face_affine = [&](int f, double al[3], double be[3], double ga[3]) {
    const double* va = kRefV[kFaceV[f][0]];
    const double* vb = kRefV[kFaceV[f][1]];
    const double* vc = kRefV[kFaceV[f][2]];
    for (int d = 0; d < 3; ++d) { al[d] = va[d]; be[d] = vb[d] - va[d]; ga[d] = vc[d] - va[d]; }
  };
  for (int f = 0; f < 4; ++f) {
    double al[3], be[3], ga[3];
    face_affine(f, al, be, ga);
    Ft[f].assign(B * F, 0.0);
    for (int k = 0; k < B; ++k) {
      P2 tr = restrict_to_face(phi[k], al, be, ga);
      for (int m = 0; m < F; ++m) Ft[f][k * F + m] = integrate_tri(mul2(tr, psi[m]));
    }
  }
  // neighbour matrices: local face barycentrics (1-c1-c2, c1, c2) at neighbour positions
  // pi = (h, h+2, h+1) mod 3; neighbour face coords chi'_1 = lam'_1, chi'_2 = lam'_2.
  for (int j = 0; j < 4; ++j) {
    double al[3], be[3], ga[3];
    face_affine(j, al, be, ga);
    for (int h = 0; h < 3; ++h) {
      int pi[3] = {h % 3, (h + 2) % 3, (h + 1) % 3};
      // lam'_q as affine functions of (c1, c2): coefficients (const, c1, c2)
      double lamc[3][3] = {{1.0, -1.0, -1.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
      double lp[3][3];
      for (int m = 0; m < 3; ++m)
        for (int t = 0; t < 3; ++t) lp[pi[m]][t] = lamc[m][t];
      // xi_d = al_d + be_d chi'_1 + ga_d chi'_2, chi'_1 = lp[1], chi'_2 = lp[2]
      double A[3], Bc[3], G[3];
      for (int d = 0; d < 3; ++d) {
        A[d] = al[d] + be[d] * lp[1][0] + ga[d] * lp[2][0];
        Bc[d] = be[d] * lp[1][1] + ga[d] * lp[2][1];
        G[d] = be[d] * lp[1][2] + ga[d] * lp[2][2];
      }
      std::vector<double>& Fm = Fb[j * 3 + h];
      Fm.assign(B * F, 0.0);
      for (int k = 0; k < B; ++k) {
        P2 tr = restrict_to_face(phi[k], A, Bc, G);
        for (int m = 0; m < F; ++m) Fm[k * F + m] = integrate_tri(mul2(tr, psi[m]));
      }
    }
  }
  // projection rule: collapsed Gauss-Jacobi (alpha 0, 1, 2), exact to degree 2n-1 per direction
  const int nq = o + 2;
  std::vector<double> xa, wa, xb, wb, xc, wc;
  gauss_jacobi(nq, 0.0, xa, wa);
  gauss_jacobi(nq, 1.0, xb, wb);
  gauss_jacobi(nq, 2.0, xc, wc);
  qp.clear();
  qw.clear();
  for (int ia = 0; ia < nq; ++ia)
    for (int ib = 0; ib < nq; ++ib)
      for (int ic = 0; ic < nq; ++ic) {
        double a = xa[ia], b = xb[ib], c = xc[ic];
        double xi3 = 0.5 * (1.0 + c);
        double xi2 = 0.25 * (1.0 + b) * (1.0 - c);
        double xi1 = 0.125 * (1.0 + a) * (1.0 - b) * (1.0 - c);
        qp.push_back({xi1, xi2, xi3});
        qw.push_back(wa[ia] * wb[ib] * wc[ic] / 64.0);
      }
}

void RefOps::eval(const double xi[3], double* out) const {
  for (int b = 0; b < B; ++b) {
    P3 p(2 * deg);
    p.c = poly[b];
    out[b] = eval3(p, xi);
  }
}

}  // namespace lts
