"""Pins for the oracle's PDE coefficients, attenuation fit and flux solvers."""
import numpy as np
import pytest
from scipy.linalg import eig

from oracle import physics as ph


def _mat(rng):
    rho = rng.uniform(2000.0, 3000.0)
    vs = rng.uniform(500.0, 4000.0)
    lam, mu = ph.lame(rho, np.sqrt(3.0) * vs, vs)
    return lam, mu, rho


def test_plane_wave_eigenvectors():
    """Textbook P and S plane waves are eigenvectors of A_n with speeds vp, vs."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        lam, mu, rho = _mat(rng)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        An = np.einsum("d,dij->ij", n, ph.elastic_jacobians(lam, mu, rho))
        vp, vs = np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho)
        S = -(lam * np.eye(3) + 2 * mu * np.outer(n, n)) / vp
        rp = np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[1, 2], S[0, 2], *n])
        assert np.allclose(An @ rp, vp * rp, rtol=1e-12, atol=1e-12 * np.abs(vp * rp).max())
        p = np.cross(n, rng.normal(size=3))
        p /= np.linalg.norm(p)
        S = -mu * (np.outer(n, p) + np.outer(p, n)) / vs
        rs = np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[1, 2], S[0, 2], *p])
        assert np.allclose(An @ rs, vs * rs, rtol=1e-12, atol=1e-12 * np.abs(vs * rs).max())


def _closed_form_flux(n, mi, mo, kind):
    """Impedance form of the exact elastic Riemann solution (normal / tangential pairs):
    v* = (Z- v- + Z+ v+ + t+ - t-)/(Z- + Z+), t* = (Z+ t- + Z- t+ + Z- Z+ (v+ - v-))/(Z- + Z+),
    free surface t* = 0, v* = v- - t-/Z-; absorbing = zero exterior state. Flux =
    interior Jacobian applied to (v*, t*). Returns 9x9 maps of q_in and q_out."""
    lam, mu, rho = mi
    if kind == "absorbing":
        mo = mi
    lo, muo, ro = mo
    zpi, zsi = np.sqrt((lam + 2 * mu) * rho), np.sqrt(mu * rho)
    zpo, zso = np.sqrt((lo + 2 * muo) * ro), np.sqrt(muo * ro)

    def tv(q):
        t = np.array([q[0] * n[0] + q[3] * n[1] + q[5] * n[2], q[3] * n[0] + q[1] * n[1] + q[4] * n[2],
                      q[5] * n[0] + q[4] * n[1] + q[2] * n[2]])
        return t, q[6:9]

    def flux(qi, qo):
        ti, vi = tv(qi)
        to, vo = tv(qo)
        if kind == "absorbing":
            to, vo = 0 * to, 0 * vo
        tin, vin, ton, von = ti @ n, vi @ n, to @ n, vo @ n
        tiT, viT, toT, voT = ti - tin * n, vi - vin * n, to - ton * n, vo - von * n
        if kind == "free":
            vsn, vsT, tsn, tsT = vin - tin / zpi, viT - tiT / zsi, 0.0, 0 * n
        else:
            vsn = (zpi * vin + zpo * von + ton - tin) / (zpi + zpo)
            tsn = (zpo * tin + zpi * ton + zpi * zpo * (von - vin)) / (zpi + zpo)
            vsT = (zsi * viT + zso * voT + toT - tiT) / (zsi + zso)
            tsT = (zso * tiT + zsi * toT + zsi * zso * (voT - viT)) / (zsi + zso)
        vs_, ts_ = vsn * n + vsT, tsn * n + tsT
        nv = n @ vs_
        F = np.zeros(9)
        for a in range(3):
            F[a] = -(lam * nv + 2 * mu * n[a] * vs_[a])
        F[3] = -mu * (n[0] * vs_[1] + n[1] * vs_[0])
        F[4] = -mu * (n[1] * vs_[2] + n[2] * vs_[1])
        F[5] = -mu * (n[0] * vs_[2] + n[2] * vs_[0])
        F[6:9] = -ts_ / rho
        Fa = -np.array([n[0] * vs_[0], n[1] * vs_[1], n[2] * vs_[2], 0.5 * (n[0] * vs_[1] + n[1] * vs_[0]),
                        0.5 * (n[1] * vs_[2] + n[2] * vs_[1]), 0.5 * (n[0] * vs_[2] + n[2] * vs_[0])])
        return F, Fa

    I = np.eye(9)
    cols_in = [flux(I[c], 0 * I[c]) for c in range(9)]
    cols_out = [flux(0 * I[c], I[c]) for c in range(9)]
    return (np.stack([c[0] for c in cols_in], 1), np.stack([c[0] for c in cols_out], 1),
            np.stack([c[1] for c in cols_in], 1), np.stack([c[1] for c in cols_out], 1))


@pytest.mark.parametrize("kind", ["interior", "free", "absorbing"])
def test_eigen_route_flux_equals_closed_form(kind):
    rng = np.random.default_rng({"interior": 1, "free": 2, "absorbing": 3}[kind])
    for _ in range(60):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        mi, mo = _mat(rng), _mat(rng)
        area, detj = rng.uniform(0.5, 2.0), rng.uniform(1.0, 5.0)
        em, ep, am, ap = ph.flux_solvers(n, area, detj, mi, mo, kind)
        Fi, Fo, Fai, Fao = _closed_form_flux(n, mi, mo, kind)
        s = -2.0 * area / detj
        # compare in units where stresses are scaled by the interior P impedance
        z = np.sqrt((mi[0] + 2 * mi[1]) * mi[2])
        D = np.diag([1 / z] * 6 + [1.0] * 3)
        Di = np.linalg.inv(D)
        for got, want in ((em, s * Fi), (ep, s * Fo)):
            assert np.abs(D @ (got - want) @ Di).max() <= 1e-12 * np.abs(D @ want @ Di).max() + 1e-300
        for got, want in ((am, s * Fai), (ap, s * Fao)):
            assert np.abs((got - want) @ Di).max() <= 1e-12 * max(np.abs(want @ Di).max(), 1e-300)
        if kind != "interior":
            assert np.all(ep == 0) and np.all(ap == 0)


def test_homogeneous_flux_is_half_sum_and_abs():
    """Equal materials: A~- + A~+ = s A_n and (A~- - A~+)^2 = (s A_n)^2 (|A_n| = A+ - A-)."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        m = _mat(rng)
        em, ep, _, _ = ph.flux_solvers(n, 0.5, 1.0, m, m, "interior")
        An = -1.0 * np.einsum("d,dij->ij", n, ph.elastic_jacobians(*m))
        z = np.sqrt((m[0] + 2 * m[1]) * m[2])
        D = np.diag([1 / z] * 6 + [1.0] * 3)
        Di = np.linalg.inv(D)
        assert np.abs(D @ (em + ep - An) @ Di).max() < 1e-12 * np.abs(D @ An @ Di).max()
        Aabs = em - ep
        assert np.abs(D @ (Aabs @ Aabs - An @ An) @ Di).max() < 1e-10 * np.abs(D @ An @ An @ Di).max()


def _qs_from_symbol(lam, mu, rho, ylam, ymu, omega, w, wave):
    """Q of P or S waves at angular frequency w from the 9+6m system's dispersion
    relation: (i w I - i k A_x - E_hat) q = 0 solved for complex k (generalised
    eigenproblem); M_eff = rho w^2 / k^2 and Q = Re M_eff / Im M_eff."""
    m = len(omega)
    nq = 9 + 6 * m
    A = np.zeros((nq, nq))
    A[:9, :9] = ph.elastic_jacobians(lam, mu, rho)[0]
    Aa = ph.anelastic_jacobians()[0]
    Ehat = np.zeros((nq, nq))
    for l in range(m):
        A[9 + 6 * l:15 + 6 * l, :9] = omega[l] * Aa
        Ehat[:9, 9 + 6 * l:15 + 6 * l] = ph.coupling_matrix(lam, mu, ylam[l], ymu[l])
        Ehat[9 + 6 * l:15 + 6 * l, 9 + 6 * l:15 + 6 * l] = -omega[l] * np.eye(6)
    # balance units (stresses ~ rho vp |v|, memory variables ~ |v| / vp) before solving
    d = np.ones(nq)
    d[:6] = rho * np.sqrt((lam + 2 * mu) / rho)
    d[9:] = 1.0 / np.sqrt((lam + 2 * mu) / rho)
    ks, vecs = eig((1j * w * np.eye(nq) - Ehat) * d[None, :] / d[:, None], (1j * A) * d[None, :] / d[:, None])
    fin = np.isfinite(ks) & (np.abs(ks) > 1e-12)
    ks, vecs = ks[fin], vecs[:, fin]
    # P: particle velocity along x (u); S: along y (v)
    comp = 6 if wave == "P" else 7
    dom = np.abs(vecs[comp, :]) / np.linalg.norm(vecs[6:9, :], axis=0)
    k = ks[np.argmax(dom * (ks.real > 0))]
    Meff = rho * w * w / k ** 2
    return abs(Meff.real / Meff.imag)


def test_attenuation_fit_reproduces_target_q_at_relaxation_frequencies():
    """Collocation is exact: the PDE symbol's Q equals the target at w = omega_l."""
    rho, vs = 2700.0, 1500.0
    vp = np.sqrt(3.0) * vs
    lam, mu = ph.lame(rho, vp, vs)
    qs = 50.0 * vs / 1000.0
    qp = 2.0 * qs
    omega = ph.relaxation_frequencies(3, 0.1, 5.0)
    assert np.allclose(omega / (2 * np.pi), [0.1, np.sqrt(0.5), 5.0], rtol=1e-14)
    ylam, ymu = ph.anelastic_coefficients(lam, mu, qp, qs, omega)
    for w in omega:
        assert abs(_qs_from_symbol(lam, mu, rho, ylam, ymu, omega, w, "S") / qs - 1) < 1e-9
        assert abs(_qs_from_symbol(lam, mu, rho, ylam, ymu, omega, w, "P") / qp - 1) < 1e-9
    # between the collocation points the constant-Q fit stays close (reported band)
    dev = max(abs(_qs_from_symbol(lam, mu, rho, ylam, ymu, omega, w, "S") / qs - 1)
              for w in 2 * np.pi * np.geomspace(0.1, 5.0, 25))
    assert dev < 0.15


def test_high_frequency_limit_is_unrelaxed():
    rho, vs = 2700.0, 1000.0
    lam, mu = ph.lame(rho, np.sqrt(3) * vs, vs)
    omega = ph.relaxation_frequencies(3, 0.1, 5.0)
    ylam, ymu = ph.anelastic_coefficients(lam, mu, 100.0, 50.0, omega)
    w = 1e7
    m = len(omega)
    nq = 9 + 6 * m
    A = np.zeros((nq, nq))
    A[:9, :9] = ph.elastic_jacobians(lam, mu, rho)[0]
    for l in range(m):
        A[9 + 6 * l:15 + 6 * l, :9] = omega[l] * ph.anelastic_jacobians()[0]
    ev = np.linalg.eigvals(A[:9, :9]).real
    assert np.isclose(ev.max(), np.sqrt((lam + 2 * mu) / rho), rtol=1e-12)
    assert w > 0


def test_coupling_structure():
    lam, mu = 3.0e9, 2.0e9
    E = ph.coupling_matrix(lam, mu, 0.1, 0.2)
    theta = np.array([1.0, 2.0, 3.0, 0.5, 0.25, 0.125])
    s = E @ theta
    tr = theta[:3].sum()
    for a in range(3):
        assert np.isclose(s[a], -(lam * 0.1 * tr + 2 * mu * 0.2 * theta[a]))
    assert np.allclose(s[3:6], -2 * mu * 0.2 * theta[3:6])
    assert np.all(s[6:] == 0)
    # Q = infinity gives Y = 0
    omega = ph.relaxation_frequencies(3, 0.1, 5.0)
    assert np.all(ph.fit_y(np.inf, omega) == 0)
