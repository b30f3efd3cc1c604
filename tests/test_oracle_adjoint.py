"""Pins for the oracle's discrete adjoint (global time stepping, elastic): the gradient of the
seismogram misfit w.r.t. every element's (rho, lambda, mu) and w.r.t. the initial DOFs
against central finite differences of the oracle's own misfit (time step held fixed)."""
import numpy as np
import pytest

from oracle.adjoint import misfit_gradient
from oracle.mesh import Mesh
from oracle.scheme import Solver as Oracle
from paper_2202_10313_gb300 import synth


def _setup(order=3, seed=4):
    m = synth.graded_box(2, 2, 1, 200.0, 100.0, seed=seed)
    mat = synth.random_layers(m, n_layers=2, seed=3)
    mesh = Mesh(m["xyz"], m["tet"], m["face_bc"])
    K = mesh.K
    rng = np.random.default_rng(seed)
    q0 = rng.normal(size=(K, 9, order * (order + 1) * (order + 2) // 6))
    q0[:, :6] *= 1e6
    rec_x = [np.array([120.0, 150.0, -30.0]), np.array([290.0, 260.0, -60.0])]
    return mesh, mat, q0, rec_x


def _solver(order, mesh, rho, lam, mu):
    vp = np.sqrt((lam + 2 * mu) / rho)
    vs = np.sqrt(mu / rho)
    return Oracle(order, 0, mesh, rho, vp, vs)


def _misfit(order, mesh, rho, lam, mu, q0, rec, data, dt, n):
    s = _solver(order, mesh, rho, lam, mu)
    s.Q = q0.copy()
    syn = []
    for step in range(n + 1):
        syn.append(np.stack([s.Q[k, 6:9] @ phi for k, phi in rec]))
        if step < n:
            s.run_gts(dt, 1)
    return 0.5 * float(np.sum((np.stack(syn) - data) ** 2))


@pytest.mark.parametrize("order", [3, 4])
def test_adjoint_gradient_matches_finite_differences(order):
    mesh, mat, q0, rec_x = _setup(order)
    K = mesh.K
    lam0, mu0 = mat["rho"] * (mat["vp"] ** 2 - 2 * mat["vs"] ** 2), mat["rho"] * mat["vs"] ** 2
    rho0 = mat["rho"].astype(float)
    base = _solver(order, mesh, rho0, lam0, mu0)
    dt = base.time_step_gts(0.5)
    rec = []
    for x in rec_x:
        k = mesh.locate(x)
        rec.append((k, base.basis.phi(mesh.xi_of(k, x)[None, :])[0]))
    n = 5
    # observed data: the same run in a model with mu perturbed by 1 %
    data = np.zeros((n + 1, len(rec), 3))
    s = _solver(order, mesh, rho0, lam0, mu0 * 1.01)
    s.Q = q0.copy()
    for step in range(n + 1):
        data[step] = np.stack([s.Q[k, 6:9] @ phi for k, phi in rec])
        if step < n:
            s.run_gts(dt, 1)
    base.Q = q0.copy()
    J, grad, lam_q0, syn = misfit_gradient(base, dt, n, [r[0] for r in rec], [r[1] for r in rec], data)
    assert abs(J - _misfit(order, mesh, rho0, lam0, mu0, q0, rec, data, dt, n)) <= 1e-12 * J
    params = [rho0, lam0, mu0]
    fd = np.zeros((K, 3))
    for k in range(K):
        for p in range(3):
            # relative step 1e-4: the oracle's flux maps (eigen route) carry ~1e-10 relative
            # rounding, so smaller steps let it dominate the difference quotient
            h = 1e-4 * params[p][k]
            up = [x.copy() for x in params]
            dn = [x.copy() for x in params]
            up[p][k] += h
            dn[p][k] -= h
            fd[k, p] = (_misfit(order, mesh, *up, q0, rec, data, dt, n) - _misfit(order, mesh, *dn, q0, rec, data, dt, n)) / (2 * h)
    for p in range(3):
        err = np.linalg.norm(grad[:, p] - fd[:, p]) / np.linalg.norm(fd[:, p])
        assert err <= 1e-5, (p, err)
    # w.r.t. the initial DOFs (J is quadratic in Q^0): a few entries
    rng = np.random.default_rng(1)
    for _ in range(4):
        k, r, bb = rng.integers(K), rng.integers(9), rng.integers(q0.shape[2])
        h = 1e-3 * np.abs(q0[:, r]).max()
        qp, qm = q0.copy(), q0.copy()
        qp[k, r, bb] += h
        qm[k, r, bb] -= h
        g = (_misfit(order, mesh, rho0, lam0, mu0, qp, rec, data, dt, n) -
             _misfit(order, mesh, rho0, lam0, mu0, qm, rec, data, dt, n)) / (2 * h)
        assert abs(g - lam_q0[k, r, bb]) <= 1e-6 * np.abs(lam_q0).max() + 1e-9 * abs(g), (k, r, bb, g, lam_q0[k, r, bb])


def test_lts_adjoint_gradient_matches_finite_differences():
    """Clustered LTS with three forced clusters (B1, B2, B1 - B2 and B3 reads all occur):
    the phase-level reverse sweep against central differences of the LTS misfit."""
    from oracle.adjoint import misfit_gradient_lts
    order = 3
    mesh, mat, q0, rec_x = _setup(order, seed=7)
    K = mesh.K
    lam0, mu0 = mat["rho"] * (mat["vp"] ** 2 - 2 * mat["vs"] ** 2), mat["rho"] * mat["vs"] ** 2
    rho0 = mat["rho"].astype(float)
    from oracle import lts as olts
    cx = mesh.centroid[:, 0]
    raw = np.digitize(cx, np.quantile(cx, [0.3, 0.65]))
    cl = olts.normalise(raw, mesh.nbr)
    assert len(np.unique(cl)) == 3

    def make(rho, lam, mu):
        s = _solver(order, mesh, rho, lam, mu)
        s.setup_clusters(3, 0.5, lam=1.0, clusters=cl)
        s.delta = 2.0e-4
        s.Q = q0.copy()
        return s

    base = make(rho0, lam0, mu0)
    assert np.any(base.has_finer) and np.any(base.has_coarser)
    rec = []
    for x in rec_x:
        k = mesh.locate(x)
        rec.append((k, base.basis.phi(mesh.xi_of(k, x)[None, :])[0]))
    n_macro = 3
    ref = make(rho0, lam0, mu0 * 1.01)
    data = [np.stack([ref.Q[k, 6:9] @ phi for k, phi in rec])]
    for _ in range(n_macro):
        ref.run_lts(4)
        data.append(np.stack([ref.Q[k, 6:9] @ phi for k, phi in rec]))
    data = np.stack(data)
    J, grad, lq0, syn = misfit_gradient_lts(base, n_macro, [r[0] for r in rec], [r[1] for r in rec], data)

    def misfit(rho, lam, mu, q=None):
        s = make(rho, lam, mu)
        if q is not None:
            s.Q = q.copy()
        out = [np.stack([s.Q[k, 6:9] @ phi for k, phi in rec])]
        for _ in range(n_macro):
            s.run_lts(4)
            out.append(np.stack([s.Q[k, 6:9] @ phi for k, phi in rec]))
        return 0.5 * float(np.sum((np.stack(out) - data) ** 2))

    assert abs(J - misfit(rho0, lam0, mu0)) <= 1e-12 * J
    params = [rho0, lam0, mu0]
    fd = np.zeros((K, 3))
    for k in range(K):
        for p in range(3):
            h = 1e-4 * params[p][k]
            up = [x.copy() for x in params]
            dn = [x.copy() for x in params]
            up[p][k] += h
            dn[p][k] -= h
            fd[k, p] = (misfit(*up) - misfit(*dn)) / (2 * h)
    for p in range(3):
        err = np.linalg.norm(grad[:, p] - fd[:, p]) / np.linalg.norm(fd[:, p])
        assert err <= 1e-5, (p, err)
    rng = np.random.default_rng(3)
    for _ in range(4):
        k, r, bb = rng.integers(K), rng.integers(9), rng.integers(q0.shape[2])
        h = 1e-3 * np.abs(q0[:, r]).max()
        qp, qm = q0.copy(), q0.copy()
        qp[k, r, bb] += h
        qm[k, r, bb] -= h
        g = (misfit(rho0, lam0, mu0, qp) - misfit(rho0, lam0, mu0, qm)) / (2 * h)
        assert abs(g - lq0[k, r, bb]) <= 1e-6 * np.abs(lq0).max() + 1e-9 * abs(g), (k, r, bb, g, lq0[k, r, bb])
