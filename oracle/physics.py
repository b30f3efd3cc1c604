"""Oracle: PDE coefficients, attenuation fit and flux solvers (test infrastructure).

Sec. III, Eq. (1): q_t + A q_x + B q_y + C q_z = E q with q = [q^e, q^a],
q^e = (sxx, syy, szz, sxy, syz, sxz, u, v, w) and, per relaxation mechanism l,
q^{a,l} = (txx, tyy, tzz, txy, tyz, txz) (memory variables, tensor components).

The paper does not print the matrices (it cites Dumbser & Kaeser 2006 and Kaeser
et al. 2007). Readings used here, written from the physics:

* elastic: sigma_t = lambda div(v) I + mu (grad v + grad v^T), rho v_t = div sigma,
  written as q_t + A_d q_{x_d} = 0;
* anelastic (generalised Maxwell body, unrelaxed lambda, mu from the given vp, vs):
  theta^l_t = omega_l (eps_dot - theta^l), eps_dot = sym grad v, and
  sigma_t gains - sum_l (lambda Y^lam_l tr(theta^l) I + 2 mu Y^mu_l theta^l).
  Hence A^a_l = omega_l Abar^a (Abar^a: -1 / -1/2 entries from -eps_dot),
  E^l = -(lambda Y^lam_l tr I + 2 mu Y^mu_l) on stress rows, E' = -omega_l I.
  The anelastic time derivative is read with -omega_l on the memory term (the
  time-kernel equation prints +omega_l; the volume kernel prints -omega_l, and
  relaxation requires the minus sign).
* relaxation fit: omega_l log-spaced over [f_min, f_max]; Y_l from collocating
  Q^-1(w) = sum_l Y_l (omega_l w + omega_l^2 Q^-1)/(omega_l^2 + w^2) at w = omega_l
  (exact for M(w) = M_u (1 - sum_l Y_l omega_l/(omega_l + i w))), solved for Q_s on
  mu and Q_p on the P modulus; Y^lam = ((lam+2mu) Y^P - 2 mu Y^S)/lam.
* flux: exact upwind (Godunov) solver with possibly different materials on the two
  sides, built here by eigen-decomposition of the normal Jacobians on both sides and
  continuity of velocity and traction at the interface; the interior element's
  Jacobian is applied to the interior Riemann state. Free surface: zero traction.
  Absorbing: exterior state zero with the interior material. Anelastic rows use the
  elastic Riemann state's velocity: A^a_n q^e*.
"""
import numpy as np
from scipy.linalg import matrix_balance

NQE = 9
SXX, SYY, SZZ, SXY, SYZ, SXZ, U, V, W = range(9)
# index of stress component (a,b) in Voigt storage
_VOIGT = {(0, 0): SXX, (1, 1): SYY, (2, 2): SZZ, (0, 1): SXY, (1, 0): SXY,
          (1, 2): SYZ, (2, 1): SYZ, (0, 2): SXZ, (2, 0): SXZ}


def lame(rho, vp, vs):
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    return lam, mu


def elastic_jacobians(lam, mu, rho):
    """A_x, A_y, A_z (9x9) of the elastic block A^e, B^e, C^e (Eq. 1)."""
    A = np.zeros((3, 9, 9))
    vel = (U, V, W)
    for d in range(3):
        # stress rows: sigma_ab,t - lam delta_ab dv_d/dx_d ... written as + A_d q_d
        for a in range(3):
            A[d, _VOIGT[(a, a)], vel[d]] -= lam
        # 2 mu eps_ab with eps_ab = (d_a v_b + d_b v_a)/2, derivative direction d
        for a in range(3):
            for b in range(a, 3):
                s = _VOIGT[(a, b)]
                if a == b:
                    if a == d:
                        A[d, s, vel[a]] -= 2.0 * mu
                else:
                    if a == d:
                        A[d, s, vel[b]] -= mu
                    if b == d:
                        A[d, s, vel[a]] -= mu
        # velocity rows: rho v_a,t - d sigma_ad / dx_d
        for a in range(3):
            A[d, vel[a], _VOIGT[(a, d)]] -= 1.0 / rho
    return A


def anelastic_jacobians():
    """Abar^a_x, _y, _z (6x9): the anelastic Jacobians with omega_l factored out."""
    A = np.zeros((3, 6, 9))
    vel = (U, V, W)
    for d in range(3):
        for a in range(3):
            for b in range(a, 3):
                s = _VOIGT[(a, b)]
                if a == b:
                    if a == d:
                        A[d, s, vel[a]] -= 1.0
                else:
                    if a == d:
                        A[d, s, vel[b]] -= 0.5
                    if b == d:
                        A[d, s, vel[a]] -= 0.5
    return A


def coupling_matrix(lam, mu, ylam, ymu):
    """E^l (9x6): stress rows -(lam Y^lam tr(theta) I + 2 mu Y^mu theta)."""
    E = np.zeros((9, 6))
    for a in range(3):
        for b in range(3):
            E[a, b] -= lam * ylam
        E[a, a] -= 2.0 * mu * ymu
    for s in (SXY, SYZ, SXZ):
        E[s, s] -= 2.0 * mu * ymu
    return E


def relaxation_frequencies(m, f_min, f_max):
    """omega_l = 2 pi f_min (f_max/f_min)^((l-1)/(m-1)), l = 1..m."""
    if m == 1:
        return np.array([2.0 * np.pi * np.sqrt(f_min * f_max)])
    return np.array([2.0 * np.pi * f_min * (f_max / f_min) ** (l / (m - 1.0)) for l in range(m)])


def fit_y(q, omega):
    """Y_l for a constant target Q by collocation at w = omega_l."""
    m = len(omega)
    qi = 1.0 / q
    M = np.zeros((m, m))
    for k in range(m):
        wk = omega[k]
        for l in range(m):
            wl = omega[l]
            M[k, l] = (wl * wk + wl * wl * qi) / (wl * wl + wk * wk)
    return np.linalg.solve(M, np.full(m, qi))


def anelastic_coefficients(lam, mu, qp, qs, omega):
    """(Y^lam_l, Y^mu_l) for one element."""
    ys = fit_y(qs, omega)
    yp = fit_y(qp, omega)
    ylam = ((lam + 2.0 * mu) * yp - 2.0 * mu * ys) / lam
    return ylam, ys


def star_matrices(jac, Jinv):
    """Abar_c = sum_d A_d dxi_c/dx_d (Sec. III-A, "element-local linear combinations")."""
    return np.einsum("dij,cd->cij", jac, Jinv)


def _traction(q, n):
    """Traction sigma n of a (..., 9) state."""
    s = q
    return np.stack([s[..., SXX] * n[0] + s[..., SXY] * n[1] + s[..., SXZ] * n[2],
                     s[..., SXY] * n[0] + s[..., SYY] * n[1] + s[..., SYZ] * n[2],
                     s[..., SXZ] * n[0] + s[..., SYZ] * n[1] + s[..., SZZ] * n[2]], axis=-1)


def _waves(An, speeds, sign):
    """Basis of the eigenvectors of An with eigenvalue sign * c, c in speeds.

    speeds = {c_p: 1, c_s: 2} (wave speed: multiplicity), the textbook eigenvalues
    of the elastic normal Jacobian. An is first balanced by a diagonal similarity
    (scipy.linalg.matrix_balance: stresses and velocities differ by ~rho c); each
    eigenspace is the null space of (An_bal - lambda I) from an SVD, mapped back
    through the balancing scale. The computed eigenvalues are checked against the
    speeds.
    """
    Ab, bal = matrix_balance(An, permute=False, separate=True)
    dscale = bal[0]
    ev = np.sort(np.linalg.eigvals(Ab).real)
    want = np.sort([sign * c for c, m in speeds.items() for _ in range(m)])
    got = ev[sign * ev > 0.5 * min(speeds)]
    if len(got) != len(want) or np.max(np.abs(np.sort(got) - want)) > 1e-8 * max(speeds):
        raise ValueError("normal Jacobian eigenvalues do not match the wave speeds")
    cols = []
    for c, mult in speeds.items():
        _, _, vt = np.linalg.svd(Ab - sign * c * np.eye(An.shape[0]))
        cols.append(dscale[:, None] * vt[-mult:, :].T)
    return np.concatenate(cols, axis=1)


def _speeds(lam, mu, rho):
    return {np.sqrt((lam + 2.0 * mu) / rho): 1, np.sqrt(mu / rho): 2}


def riemann_state_maps(n, mat_in, mat_out, kind):
    """Linear maps (M_in, M_out), 9x9, with q*_in = M_in q_in + M_out q_out.

    q*_in is the interior-side Godunov state of the linear Riemann problem along
    the outward unit normal n: q*_in - q_in is a combination of the interior's
    waves that travel into the interior (eigenvalues < 0 of A_n^-); q*_out - q_out
    a combination of the exterior's waves travelling outward (eigenvalues > 0 of
    A_n^+); velocity and traction are continuous. kind: 'interior' (incl.
    periodic), 'absorbing' (q_out = 0, exterior = interior material) or 'free'
    (traction of q*_in is zero).
    """
    lam_i, mu_i, rho_i = mat_in
    jac_i = elastic_jacobians(lam_i, mu_i, rho_i)
    An_i = np.einsum("d,dij->ij", n, jac_i)
    Rm = _waves(An_i, _speeds(lam_i, mu_i, rho_i), -1.0)  # (9, 3) into the interior
    if Rm.shape[1] != 3:
        raise ValueError("expected 3 incoming waves")
    eye = np.eye(9)
    if kind == "free":
        T = _traction(Rm.T, n).T                            # (3, 3): traction of each wave
        Tq = _traction(eye, n).T                            # (3, 9): traction of unit states
        alpha = -np.linalg.solve(T, Tq)                     # (3, 9)
        return eye + Rm @ alpha, np.zeros((9, 9))
    if kind == "absorbing":
        mat_out = mat_in
    lam_o, mu_o, rho_o = mat_out
    jac_o = elastic_jacobians(lam_o, mu_o, rho_o)
    An_o = np.einsum("d,dij->ij", n, jac_o)
    Rp = _waves(An_o, _speeds(lam_o, mu_o, rho_o), 1.0)
    if Rp.shape[1] != 3:
        raise ValueError("expected 3 outgoing waves")
    # unknowns (alpha (3), beta (3)): v(q_in + Rm a) = v(q_out - Rp b), same for traction
    Mv = np.concatenate([Rm[U:W + 1, :], Rp[U:W + 1, :]], axis=1)           # (3, 6)
    Mt = np.concatenate([_traction(Rm.T, n).T, _traction(Rp.T, n).T], axis=1)
    Msys = np.concatenate([Mv, Mt], axis=0)                                   # (6, 6)
    Pv = eye[U:W + 1, :]
    Pt = _traction(eye, n).T
    P = np.concatenate([Pv, Pt], axis=0)                                      # (6, 9)
    sol_in = np.linalg.solve(Msys, -P)            # coefficient of q_in
    sol_out = np.linalg.solve(Msys, P)            # coefficient of q_out
    if kind == "absorbing":
        sol_out = np.zeros_like(sol_out)
    M_in = eye + Rm @ sol_in[:3, :]
    M_out = Rm @ sol_out[:3, :]
    return M_in, M_out


def flux_solvers(n, area, detJ, mat_in, mat_out, kind):
    """Flux solvers (A~e-, A~e+, A~a-, A~a+) of one element face (Sec. III-A).

    S^{e_L} adds A~e- (T^e F~_i) F^_i and S^{e_N} adds A~e+ (T^e_nbr F-_{j,h}) F^_i, so
    A~ = -(2 |S_i| / |det J|) * A_n q*(.) with the reference face of area 1/2.
    """
    lam, mu, rho = mat_in
    An = np.einsum("d,dij->ij", n, elastic_jacobians(lam, mu, rho))
    Aan = np.einsum("d,dij->ij", n, anelastic_jacobians())
    M_in, M_out = riemann_state_maps(n, mat_in, mat_out, kind)
    s = -2.0 * area / detJ
    return s * An @ M_in, s * An @ M_out, s * Aan @ M_in, s * Aan @ M_out


def compliance_energy_density(sig, lam, mu):
    """1/2 sigma : C^-1 sigma for Voigt stress arrays (..., 6)."""
    sxx, syy, szz, sxy, syz, sxz = (sig[..., i] for i in range(6))
    tr = sxx + syy + szz
    ss = sxx ** 2 + syy ** 2 + szz ** 2 + 2.0 * (sxy ** 2 + syz ** 2 + sxz ** 2)
    return 0.5 * (ss / (2.0 * mu) - lam / (2.0 * mu * (3.0 * lam + 2.0 * mu)) * tr ** 2)
