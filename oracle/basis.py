"""Oracle: modal basis, quadrature and reference operators (test infrastructure).

Sec. III-A of the paper: the DOFs of a tetrahedron are the coefficients of
B(O) = O(O+1)(O+2)/6 modal basis functions built by the Karniadakis-Sherwin
(Dubiner) tetrahedral expansion; faces carry F(O) = O(O+1)/2 triangle functions.

Conventions (the paper prints none; these readings are shared by contract with the
product library, which implements them independently):

* reference tetrahedron: vertices v0=(0,0,0), v1=(1,0,0), v2=(0,1,0), v3=(0,0,1);
* tetrahedral mode (i, j, k), degree p=i+j+k, modes ordered by p, then k, then j;
  phi_ijk = [s1^i P_i(a)] [s2^j P_j^(2i+1,0)(b)] P_k^(2i+2j+2,0)(c) with
  s1 = 1-xi2-xi3, s2 = 1-xi3, a = 2 xi1/s1 - 1, b = 2 xi2/s2 - 1, c = 2 xi3 - 1,
  scaled to unit L2 norm on the reference tetrahedron (so the mass matrix is I);
* triangle mode (i, j), ordered by p=i+j then j: psi_ij = [s^i P_i(a)] P_j^(2i+1,0)(b),
  s = 1-chi2, a = 2 chi1/s - 1, b = 2 chi2 - 1, unit L2 norm on the reference
  triangle (0,0),(1,0),(0,1);
* face i of the reference tetrahedron is the vertex triple FACE_VERTS[i]
  (outward orientation), parametrised as x = V_a + chi1 (V_b - V_a) + chi2 (V_c - V_a).

Quadrature here is collapsed-coordinate Gauss-Legendre (Duffy transform), a route
independent of the product library's exact monomial integration.
"""
import numpy as np
from numpy.polynomial.legendre import leggauss

REF_VERTS = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
FACE_VERTS = ((0, 2, 1), (0, 1, 3), (0, 3, 2), (1, 2, 3))


def n_basis(order):
    """B(O) of Sec. III-A (B(4)=20, B(5)=35)."""
    return order * (order + 1) * (order + 2) // 6


def n_face_basis(order):
    """F(O) of Sec. III-A "Surface Kernel" (F(5)=15)."""
    return order * (order + 1) // 2


def tet_modes(order):
    """Mode triples (i, j, k) in storage order: degree, then k, then j."""
    modes = []
    for p in range(order):
        for k in range(p + 1):
            for j in range(p - k + 1):
                modes.append((p - j - k, j, k))
    return modes


def tri_modes(order):
    """Triangle mode pairs (i, j) in storage order: degree, then j."""
    return [(p - j, j) for p in range(order) for j in range(p + 1)]


class Dual:
    """Forward-mode value + gradient (w.r.t. the 3 reference coordinates)."""

    __slots__ = ("v", "d")

    def __init__(self, v, d):
        self.v = np.asarray(v, dtype=float)
        self.d = np.asarray(d, dtype=float)

    @staticmethod
    def const(c, n):
        return Dual(np.full(n, float(c)), np.zeros((n, 3)))

    def __add__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v + o.v, self.d + o.d)
        return Dual(self.v + o, self.d)

    __radd__ = __add__

    def __sub__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v - o.v, self.d - o.d)
        return Dual(self.v - o, self.d)

    def __rsub__(self, o):
        return Dual(o - self.v, -self.d)

    def __mul__(self, o):
        if isinstance(o, Dual):
            return Dual(self.v * o.v, self.d * o.v[:, None] + o.d * self.v[:, None])
        return Dual(self.v * o, self.d * o)

    __rmul__ = __mul__

    def __truediv__(self, c):
        return Dual(self.v / c, self.d / c)


def jacobi_homogeneous(nmax, alpha, x, s):
    """[s^n P_n^(alpha,0)(x/s) for n = 0..nmax].

    Standard three-term Jacobi recurrence (beta = 0) multiplied through by s^n, so
    the result is a polynomial in (x, s) and stays finite where s -> 0. Works on
    floats, arrays or Dual numbers.
    """
    out = [x * 0.0 + 1.0]
    if nmax >= 1:
        out.append(((alpha + 2.0) * x + alpha * s) / 2.0)
    for n in range(2, nmax + 1):
        a1 = 2.0 * n * (n + alpha) * (2.0 * n + alpha - 2.0)
        a2 = (2.0 * n + alpha - 1.0)
        a3 = (2.0 * n + alpha) * (2.0 * n + alpha - 2.0)
        a4 = 2.0 * (n + alpha - 1.0) * (n - 1.0) * (2.0 * n + alpha)
        out.append((a2 * (a3 * x + alpha * alpha * s) * out[n - 1] - a4 * (s * s) * out[n - 2]) / a1)
    return out


def _tet_unnormalised(order, xi, dual):
    """Unnormalised phi_ijk at points xi (N,3); Dual-valued if dual."""
    n = xi.shape[0]
    if dual:
        x1 = Dual(xi[:, 0], np.tile([1.0, 0.0, 0.0], (n, 1)))
        x2 = Dual(xi[:, 1], np.tile([0.0, 1.0, 0.0], (n, 1)))
        x3 = Dual(xi[:, 2], np.tile([0.0, 0.0, 1.0], (n, 1)))
        one = Dual.const(1.0, n)
    else:
        x1, x2, x3, one = xi[:, 0], xi[:, 1], xi[:, 2], 1.0
    s1 = one - x2 - x3
    s2 = one - x3
    vals = []
    for (i, j, k) in tet_modes(order):
        hi = jacobi_homogeneous(i, 0.0, 2.0 * x1 - s1, s1)[i]
        hj = jacobi_homogeneous(j, 2.0 * i + 1.0, 2.0 * x2 - s2, s2)[j]
        hk = jacobi_homogeneous(k, 2.0 * i + 2.0 * j + 2.0, 2.0 * x3 - one, one)[k]
        vals.append(hi * hj * hk)
    return vals


def _tri_unnormalised(order, chi):
    c1, c2 = chi[:, 0], chi[:, 1]
    s = 1.0 - c2
    vals = []
    for (i, j) in tri_modes(order):
        hi = jacobi_homogeneous(i, 0.0, 2.0 * c1 - s, s)[i]
        hj = jacobi_homogeneous(j, 2.0 * i + 1.0, 2.0 * c2 - 1.0, 1.0)[j]
        vals.append(hi * hj)
    return vals


def tet_quadrature(n):
    """Collapsed Gauss-Legendre rule on the reference tetrahedron, n^3 points.

    xi3 = (1+c)/2, xi2 = (1+b)(1-c)/4, xi1 = (1+a)(1-b)(1-c)/8, Jacobian
    (1-b)(1-c)^2/64. Exact for polynomials of degree <= 2n-3 in xi.
    """
    g, w = leggauss(n)
    a, b, c = np.meshgrid(g, g, g, indexing="ij")
    wa, wb, wc = np.meshgrid(w, w, w, indexing="ij")
    xi3 = (1.0 + c) / 2.0
    xi2 = (1.0 + b) * (1.0 - c) / 4.0
    xi1 = (1.0 + a) * (1.0 - b) * (1.0 - c) / 8.0
    wt = wa * wb * wc * (1.0 - b) * (1.0 - c) ** 2 / 64.0
    pts = np.stack([xi1.ravel(), xi2.ravel(), xi3.ravel()], axis=1)
    return pts, wt.ravel()


def tri_quadrature(n):
    """Collapsed Gauss-Legendre rule on the reference triangle, n^2 points."""
    g, w = leggauss(n)
    a, b = np.meshgrid(g, g, indexing="ij")
    wa, wb = np.meshgrid(w, w, indexing="ij")
    c2 = (1.0 + b) / 2.0
    c1 = (1.0 + a) * (1.0 - b) / 4.0
    wt = wa * wb * (1.0 - b) / 8.0
    return np.stack([c1.ravel(), c2.ravel()], axis=1), wt.ravel()


class Basis:
    """Orthonormal tetrahedral and triangle bases of one order, with operators.

    Attributes (all FP64, orthonormal basis so the mass matrix is the identity):
      K[c][b, a]   = int phi_b d(phi_a)/d(xi_c)             (Sec. III-A, K_c; the
                     time kernel uses Q K_c^T, the volume kernel Q K_c)
      Ft[i][b, f]  = int_face_i phi_b psi_f dchi             (F~_i, volume -> face)
      Fh[i][f, a]  = int_face_i psi_f phi_a dchi             (F^_i = F~_i^T, M = I)
      Fb[j][h][b, f] = int psi_f(chi) phi_b(xi_j(chi'(chi,h))) dchi  (F-_{j,h})
    """

    def __init__(self, order):
        self.order = order
        self.nb = n_basis(order)
        self.nf = n_face_basis(order)
        self.qp, self.qw = tet_quadrature(order + 2)
        self.fqp, self.fqw = tri_quadrature(order + 2)
        raw = _tet_unnormalised(order, self.qp, dual=False)
        self.norm2 = np.array([np.sum(self.qw * r * r) for r in raw])
        self.scale = 1.0 / np.sqrt(self.norm2)
        rawf = _tri_unnormalised(order, self.fqp)
        self.fnorm2 = np.array([np.sum(self.fqw * r * r) for r in rawf])
        self.fscale = 1.0 / np.sqrt(self.fnorm2)
        self._build_operators()

    # -- evaluation ---------------------------------------------------------
    def phi(self, xi):
        """phi_b(xi) for points xi (N,3) -> (N, B)."""
        xi = np.atleast_2d(np.asarray(xi, dtype=float))
        raw = _tet_unnormalised(self.order, xi, dual=False)
        return np.stack(raw, axis=1) * self.scale[None, :]

    def grad_phi(self, xi):
        """d phi_b / d xi_c at points xi -> (N, B, 3)."""
        xi = np.atleast_2d(np.asarray(xi, dtype=float))
        raw = _tet_unnormalised(self.order, xi, dual=True)
        return np.stack([r.d for r in raw], axis=1) * self.scale[None, :, None]

    def psi(self, chi):
        """psi_f(chi) for face points chi (N,2) -> (N, F)."""
        chi = np.atleast_2d(np.asarray(chi, dtype=float))
        raw = _tri_unnormalised(self.order, chi)
        return np.stack(raw, axis=1) * self.fscale[None, :]

    # -- reference operators ------------------------------------------------
    @staticmethod
    def face_point(i, chi):
        """Reference-tet coordinates of face-i parameter points chi (N,2)."""
        a, b, c = FACE_VERTS[i]
        va, vb, vc = REF_VERTS[a], REF_VERTS[b], REF_VERTS[c]
        return va[None, :] + chi[:, :1] * (vb - va)[None, :] + chi[:, 1:2] * (vc - va)[None, :]

    @staticmethod
    def neighbour_chi(h, chi):
        """Neighbour face parameters of local face parameters chi for orientation h.

        Local face vertices (a, b, c) carry barycentric weights (1-chi1-chi2, chi1,
        chi2). The neighbour's face lists the same three vertices in reversed cyclic
        order with its vertex number h equal to the local vertex a, so local vertex
        m sits at neighbour position pi(m) with pi = (h, h+2, h+1) mod 3.
        """
        lam = np.stack([1.0 - chi[:, 0] - chi[:, 1], chi[:, 0], chi[:, 1]], axis=1)
        perm = (h % 3, (h + 2) % 3, (h + 1) % 3)
        lamn = np.zeros_like(lam)
        for m in range(3):
            lamn[:, perm[m]] = lam[:, m]
        return lamn[:, 1:3]

    def _build_operators(self):
        qp, qw = self.qp, self.qw
        ph = self.phi(qp)                      # (N, B)
        gp = self.grad_phi(qp)                 # (N, B, 3)
        self.mass = (ph * qw[:, None]).T @ ph
        self.K = [(ph * qw[:, None]).T @ gp[:, :, c] for c in range(3)]
        fq, fw = self.fqp, self.fqw
        ps = self.psi(fq)                       # (Nf, F)
        self.Ft = []
        for i in range(4):
            phf = self.phi(self.face_point(i, fq))
            self.Ft.append((phf * fw[:, None]).T @ ps)
        self.Fh = [ft.T.copy() for ft in self.Ft]
        self.Fb = []
        for j in range(4):
            row = []
            for h in range(3):
                phn = self.phi(self.face_point(j, self.neighbour_chi(h, fq)))
                row.append((phn * fw[:, None]).T @ ps)
            self.Fb.append(row)

    # -- projection -----------------------------------------------------------
    def project(self, values_at_qp):
        """L2 projection onto the orthonormal basis: (..., N) values -> (..., B)."""
        ph = self.phi(self.qp)
        return values_at_qp @ (ph * self.qw[:, None])


def closed_form_tet_norm2(i, j, k):
    """Textbook norm of the unnormalised mode on the [0,1] reference tetrahedron.

    From int_{-1}^{1} (1-x)^alpha P_n^(alpha,0)(x)^2 dx = 2^(alpha+1)/(2n+alpha+1)
    and the collapsed-coordinate Jacobian: 1 / ((2i+1)(2i+2j+2)(2i+2j+2k+3)).
    """
    return 1.0 / ((2 * i + 1) * (2 * i + 2 * j + 2) * (2 * i + 2 * j + 2 * k + 3))


def closed_form_tri_norm2(i, j):
    """Norm of the unnormalised triangle mode: 1 / ((2i+1)(2i+2j+2))."""
    return 1.0 / ((2 * i + 1) * (2 * i + 2 * j + 2))
