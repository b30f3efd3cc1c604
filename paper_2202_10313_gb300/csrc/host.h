// Host-side set-up of the ADER-DG LTS solver (FP64): reference operators, geometry,
// face neighbours, per-element kernel data, clustering and the schedule's tables.
#pragma once
#include <array>
#include <cstdint>
#include <string>
#include <vector>

namespace lts {

struct Error {
  int code;
  std::string msg;
};

int n_basis(int order);
int n_face_basis(int order);

// Reference operators of one order, exact (monomial integration), orthonormal basis.
//   K[c][i*B + j]      = int phi_i d(phi_j)/d(xi_c)                 (Sec. III-A K_c)
//   Ft[f][k*F + m]     = int_{face f} phi_k psi_m                   (F~_f)
//   Fb[j*3+h][k*F + m] = int psi_m(chi) phi_k(xi_j(chi'(chi,h)))   (F-_{j,h})
// F^_f = F~_f^T because the mass matrix is the identity.
struct RefOps {
  int order = 0, B = 0, F = 0;
  std::vector<double> K[3];
  std::vector<double> Ft[4];
  std::vector<double> Fb[12];
  std::vector<int> degree;                 // total degree of each mode
  // projection rule: points (xi) and weights on the reference tetrahedron
  std::vector<std::array<double, 3>> qp;
  std::vector<double> qw;
  void build(int order);
  // phi_b(xi) for b = 0..B-1
  void eval(const double xi[3], double* out) const;
  // internal: polynomial coefficients of each mode
  int deg = 0;                              // max polynomial degree (order-1)
  std::vector<std::vector<double>> poly;    // poly[b][idx(a,b,c)]
};

// Gauss-Jacobi nodes/weights for weight (1-x)^alpha on [-1,1] (beta = 0).
void gauss_jacobi(int n, double alpha, std::vector<double>& x, std::vector<double>& w);

struct Mesh {
  int64_t nv = 0, K = 0;
  std::vector<double> xyz;       // 3 nv
  std::vector<int64_t> tet;      // 4 K
  std::vector<int32_t> bc;       // 4 K
  bool periodic = false;
  double period[3] = {0, 0, 0};
  // geometry
  std::vector<double> detJ, Jinv, J, x0;     // K, 9K (Jinv[c*3+d] = dxi_c/dx_d), 9K (J[d*3+c] = dx_d/dxi_c), 3K
  std::vector<double> normal, area, dins;    // 12K, 4K, K
  // neighbours
  std::vector<int64_t> nbr;                  // 4K, -1 if none
  std::vector<int8_t> nbr_face, nbr_orient;  // 4K
};

// Builds geometry + neighbours. Returns 0 or fills err.
int build_mesh(Mesh& m, Error& err);

// Element containing point x (lowest index with barycentric coords >= -tol), -1 if none.
int64_t locate(const Mesh& m, const double x[3], double xi_out[3]);

struct Material {
  std::vector<double> rho, vp, vs, qp, qs;
  double f_min = 0.1, f_max = 5.0;
};

// Relaxation frequencies and the constant-Q fit (Y per mechanism) by Gaussian elimination.
void relaxation_frequencies(int m, double f_min, double f_max, double* omega);
int fit_y(int m, double q, const double* omega, double* y);

// Rate-2 clustering (Sec. V-A).
void cfl_time_steps(const Mesh& m, const Material& mat, int order, double cfl, std::vector<double>& dt);
void assign_clusters(const std::vector<double>& dt, double lam, int nc, std::vector<int32_t>& c);
void normalise_clusters(const Mesh& m, std::vector<int32_t>& c);
double theoretical_speedup(const std::vector<int32_t>& c, double lam);
double search_lambda(const Mesh& m, const std::vector<double>& dt, int nc, std::vector<int32_t>& c, double* speedup);

}  // namespace lts
