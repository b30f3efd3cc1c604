"""Oracle: discrete adjoint of the global-time-stepping loop, elastic (test infrastructure).

Objective (the seismogram misfit of Sec. VII-B, summed instead of normalised):
    J = 1/2 sum_{n=0..N} sum_r |v_r(t_n) - d_r^n|^2,   v_r(t_n) = Q^n_{k_r}[u, v, w] phi(xi_r),
the velocity at receiver r sampled at the step boundaries t_n = n dt of N steps of the
oracle's GTS scheme (predict + volume + local surface for all elements, then the
neighbour surface with T of the neighbours; sources add terms independent of Q and of
the material). One step is linear in Q:
    D_0 = Q, D_{d+1} = L(D_d) = -sum_c Abar_c D_d K_c^T,   T = sum_d c_d D_d, c_d = dt^(d+1)/(d+1)!,
    Q' = Q + sum_c Abar_c T K_c + sum_i A~-_i (T F~_i) F^_i + sum_i A~+_i (T_{k_i} F-_{j,h}) F^_i.
Its transpose gives the adjoint recursion lambda^n = lambda^{n+1} + G_0 (+ the misfit's
source at t_n) with mu = dJ/dT,
    mu_k = sum_c Abar_c^T lambda_k K_c^T + sum_i ((A~-_i^T lambda_k) F^_i^T) F~_i^T
           + sum over faces (k', i') whose neighbour is k of ((A~+_{k',i'}^T lambda_k') F^_{i'}^T) F-_{j,h}^T,
    G_{O-1} = c_{O-1} mu,  G_d = c_d mu + L^T(G_{d+1}),  L^T(Z) = -sum_c Abar_c^T Z K_c.
The material enters only through the 9 x 9 matrices Abar_c (element k's own lambda, mu,
rho) and A~-, A~+ (both sides of the face), so
    dJ/dp = sum_n [ sum_c <dAbar_c/dp, -sum_{d<O-1} G_{d+1} (D_d K_c^T)^T + lambda (T K_c)^T>
                    + sum_i <dA~-_i/dp, lambda (T F~_i F^_i)^T> + sum_i <dA~+_i/dp, lambda (T_{k_i} F-_{j,h} F^_i)^T> ],
with lambda = lambda^{n+1} and D, T of step n; the time step is held fixed. The
derivatives of the 9 x 9 matrices are central differences of their FP64 constructions with
a relative step of 1e-4 (the flux maps come from an eigen decomposition with ~1e-10 relative
rounding, which smaller steps would amplify).
"""
import math

import numpy as np

from . import physics as ph
from .mesh import BC_ABSORBING, BC_FREE


def _face_matrices(solver, k, i, mat_k, mat_o):
    mesh = solver.mesh
    bc = mesh.face_bc[k, i]
    kind = "free" if bc == BC_FREE else ("absorbing" if bc == BC_ABSORBING else "interior")
    if kind != "interior":
        mat_o = mat_k
    em, ep, _, _ = ph.flux_solvers(mesh.normal[k, i], mesh.area[k, i], mesh.detJ[k], mat_k, mat_o, kind)
    return em, ep


def derivative_matrices(solver, rel=1e-4):
    """Central differences of Abar_c (w.r.t. the element's rho, lambda, mu) and of A~-, A~+
    (w.r.t. the element's and the neighbour's rho, lambda, mu).

    Returns dAe (K, 3 params, 3 c, 9, 9), dAm, dAp (K, 4 faces, 6 params, 9, 9): params
    0-2 the element's (rho, lambda, mu), 3-5 the neighbour's."""
    s = solver
    mesh = s.mesh
    K = mesh.K
    mats = np.stack([s.rho, s.lam, s.mu], axis=1)
    dAe = np.zeros((K, 3, 3, 9, 9))
    dAm = np.zeros((K, 4, 6, 9, 9))
    dAp = np.zeros((K, 4, 6, 9, 9))

    def star(m, k):
        rho, lam, mu = m
        return ph.star_matrices(ph.elastic_jacobians(lam, mu, rho), mesh.Jinv[k])

    for k in range(K):
        for p in range(3):
            h = rel * abs(mats[k, p])
            mp, mm = mats[k].copy(), mats[k].copy()
            mp[p] += h
            mm[p] -= h
            dAe[k, p] = (star(mp, k) - star(mm, k)) / (2 * h)
        for i in range(4):
            nb = mesh.nbr[k, i]
            own = mats[k]
            oth = mats[nb] if nb >= 0 else mats[k]
            for p in range(6):
                a, b = own.copy(), oth.copy()
                c, d = own.copy(), oth.copy()
                if p < 3:
                    h = rel * abs(own[p])
                    a[p] += h
                    c[p] -= h
                else:
                    if nb < 0:
                        continue
                    h = rel * abs(oth[p - 3])
                    b[p - 3] += h
                    d[p - 3] -= h
                emp, epp = _face_matrices(s, k, i, (a[1], a[2], a[0]), (b[1], b[2], b[0]))
                emm, epm = _face_matrices(s, k, i, (c[1], c[2], c[0]), (d[1], d[2], d[0]))
                dAm[k, i, p] = (emp - emm) / (2 * h)
                dAp[k, i, p] = (epp - epm) / (2 * h)
    return dAe, dAm, dAp


def _samples(Q, rec_elem, rec_phi):
    return np.stack([Q[k, 6:9, :] @ phi for k, phi in zip(rec_elem, rec_phi)])


def misfit_gradient(solver, dt, n_steps, rec_elem, rec_phi, data):
    """J, dJ/d(rho, lambda, mu) per element (K, 3), dJ/dQ^0, and the synthetic samples
    (N+1, n_rec, 3), from the solver's current state; the solver ends at t_N."""
    s = solver
    if s.m != 0:
        raise ValueError("the oracle adjoint is written for the elastic equations")
    mesh = s.mesh
    b = s.basis
    K, O = mesh.K, s.order
    Qs = [s.Q.copy()]
    for _ in range(n_steps):
        s.run_gts(dt, 1)
        Qs.append(s.Q.copy())
    synth = np.stack([_samples(Q, rec_elem, rec_phi) for Q in Qs])
    res = synth - data
    J = 0.5 * float(np.sum(res ** 2))
    cd = [dt ** (d + 1) / math.factorial(d + 1) for d in range(O)]
    idx = np.arange(K)
    lam = np.zeros((K, 9, b.nb))

    def add_source(n):
        for r, (k, phi) in enumerate(zip(rec_elem, rec_phi)):
            lam[k, 6:9, :] += np.outer(res[n, r], phi)

    add_source(n_steps)
    Wc = np.zeros((K, 3, 9, 9))
    Wm = np.zeros((K, 4, 9, 9))
    Wp = np.zeros((K, 4, 9, 9))
    nbr, nbf, nbo = mesh.nbr, mesh.nbr_face, mesh.nbr_orient
    Ae, Aem, Aep = s.Ae, s.Aem, s.Aep
    K3 = b.K
    for n in range(n_steps - 1, -1, -1):
        s.Q = Qs[n].copy()
        D = [d[:, :9, :] for d in s.derivatives(idx)]
        T = sum(cd[d] * D[d] for d in range(O))
        mu = sum(np.transpose(Ae[:, c], (0, 2, 1)) @ lam @ K3[c].T for c in range(3))
        for i in range(4):
            mu += ((np.transpose(Aem[:, i], (0, 2, 1)) @ lam) @ b.Fh[i].T) @ b.Ft[i].T
        for k in range(K):
            for i in range(4):
                kn = nbr[k, i]
                if kn < 0:
                    continue
                mu[kn] += ((Aep[k, i].T @ lam[k]) @ b.Fh[i].T) @ b.Fb[nbf[k, i]][nbo[k, i]].T
        G = [None] * O
        G[O - 1] = cd[O - 1] * mu
        for d in range(O - 2, -1, -1):
            G[d] = cd[d] * mu - sum(np.transpose(Ae[:, c], (0, 2, 1)) @ G[d + 1] @ K3[c] for c in range(3))
        for c in range(3):
            acc = lam @ np.transpose(T @ K3[c], (0, 2, 1))
            for d in range(O - 1):
                acc -= G[d + 1] @ np.transpose(D[d] @ K3[c].T, (0, 2, 1))
            Wc[:, c] += acc
        for i in range(4):
            Wm[:, i] += lam @ np.transpose((T @ b.Ft[i]) @ b.Fh[i], (0, 2, 1))
            H = np.zeros((K, 9, b.nf))
            for k in range(K):
                kn = nbr[k, i]
                if kn >= 0:
                    H[k] = T[kn] @ b.Fb[nbf[k, i]][nbo[k, i]]
            Wp[:, i] += lam @ np.transpose(H @ b.Fh[i], (0, 2, 1))
        lam = lam + G[0]
        add_source(n)
    s.Q = Qs[-1].copy()
    return J, _contract(s, Wc, Wm, Wp), lam, synth


def _contract(solver, Wc, Wm, Wp):
    """dJ/d(rho, lambda, mu) from the per-element correlations."""
    nbr = solver.mesh.nbr
    dAe, dAm, dAp = derivative_matrices(solver)
    grad = np.einsum("kpcij,kcij->kp", dAe, Wc)
    grad += np.einsum("kipab,kiab->kp", dAm[:, :, :3], Wm) + np.einsum("kipab,kiab->kp", dAp[:, :, :3], Wp)
    for k in range(solver.mesh.K):
        for i in range(4):
            kn = nbr[k, i]
            if kn >= 0:
                grad[kn] += np.einsum("pab,ab->p", dAm[k, i, 3:], Wm[k, i]) + np.einsum("pab,ab->p", dAp[k, i, 3:], Wp[k, i])
    return grad


def misfit_gradient_lts(solver, n_macro, rec_elem, rec_phi, data):
    """Clustered LTS (Sec. V-B): J = 1/2 sum_m sum_r |v_r(t_m) - d_r^m|^2 over the macro-step
    boundaries t_m (every cluster has completed its steps there), m = 0..n_macro, from the
    solver's current state with its clusters set up. The LTS state is (Q, B1, B2, B3); the
    reverse sweep takes the phases backwards:
    * a neighbour pass of cluster l (step n) added S_N(X_i) to Q_k with X_i the neighbour's
      B1, B3, B2 or B1 - B2 (cluster relation, parity of n); its transpose adds
      ((A~+^T lambda_Q_k) F^_i^T) F-_{j,h}^T to the adjoint of that buffer;
    * a predict pass (step n) wrote B1 = T, B2 = T(dt/2) (finer neighbour), B3 = T or
      B3 += T (coarser neighbour, even / odd n) and added V(T) + S_L(T) to Q; so
      mu = dJ/dT = V^T + S_L^T + lambda_B1 (+ lambda_B3), mu_half = lambda_B2, the
      buffer adjoints reset except lambda_B3 after an accumulation, and the transposed
      time kernel G_d = c_d mu + c'_d mu_half + L^T(G_{d+1}) adds G_0 to lambda_Q.
    Returns J, dJ/d(rho, lambda, mu) (K, 3), dJ/dQ at the start, samples (M+1, n_rec, 3)."""
    s = solver
    if s.m != 0:
        raise ValueError("the oracle adjoint is written for the elastic equations")
    mesh = s.mesh
    b = s.basis
    K, O = mesh.K, s.order
    nc = s.n_clusters
    period = 2 ** (nc - 1)
    nbr, nbf, nbo = mesh.nbr, mesh.nbr_face, mesh.nbr_orient
    Ae, Aem, Aep = s.Ae, s.Aem, s.Aep
    K3 = b.K
    records = [("S", 0)]
    orig_p, orig_n = s._predict_local, s._neighbour

    def rec_p(l, n):
        idx = np.nonzero(s.clusters == l)[0]
        if len(idx):
            records.append(("P", l, n, idx, s.Q[idx].copy()))
        orig_p(l, n)

    def rec_n(l, n):
        idx = np.nonzero(s.clusters == l)[0]
        if len(idx):
            X = np.zeros((len(idx), 4, 9, b.nb))
            for p_, k in enumerate(idx):
                for i in range(4):
                    kn = nbr[k, i]
                    if kn < 0:
                        continue
                    cn = s.clusters[kn]
                    if cn == l - 1:
                        X[p_, i] = s.B3[kn]
                    elif cn == l + 1:
                        X[p_, i] = s.B2[kn] if n % 2 == 0 else s.B1[kn] - s.B2[kn]
                    else:
                        X[p_, i] = s.B1[kn]
            records.append(("N", l, n, idx, X))
        orig_n(l, n)

    s._predict_local, s._neighbour = rec_p, rec_n
    samples = [_samples(s.Q, rec_elem, rec_phi)]
    try:
        for m in range(n_macro):
            s.run_lts(period)
            samples.append(_samples(s.Q, rec_elem, rec_phi))
            records.append(("S", m + 1))
    finally:
        s._predict_local, s._neighbour = orig_p, orig_n
    synth = np.stack(samples)
    res = synth - data
    J = 0.5 * float(np.sum(res ** 2))
    lq = np.zeros((K, 9, b.nb))
    lb1, lb2, lb3 = np.zeros_like(lq), np.zeros_like(lq), np.zeros_like(lq)
    Wc = np.zeros((K, 3, 9, 9))
    Wm = np.zeros((K, 4, 9, 9))
    Wp = np.zeros((K, 4, 9, 9))
    for rec in reversed(records):
        if rec[0] == "S":
            for r, (k, phi) in enumerate(zip(rec_elem, rec_phi)):
                lq[k, 6:9, :] += np.outer(res[rec[1], r], phi)
        elif rec[0] == "N":
            _, l, n, idx, X = rec
            for p_, k in enumerate(idx):
                for i in range(4):
                    kn = nbr[k, i]
                    if kn < 0:
                        continue
                    Fb = b.Fb[nbf[k, i]][nbo[k, i]]
                    Y = ((Aep[k, i].T @ lq[k]) @ b.Fh[i].T) @ Fb.T
                    cn = s.clusters[kn]
                    if cn == l - 1:
                        lb3[kn] += Y
                    elif cn == l + 1:
                        lb2[kn] += Y if n % 2 == 0 else -Y
                        if n % 2 == 1:
                            lb1[kn] += Y
                    else:
                        lb1[kn] += Y
                    Wp[k, i] += lq[k] @ ((X[p_, i] @ Fb) @ b.Fh[i]).T
        else:
            _, l, n, idx, Qb = rec
            dl = s.delta * 2.0 ** l
            cd = [dl ** (d + 1) / math.factorial(d + 1) for d in range(O)]
            ch = [(0.5 * dl) ** (d + 1) / math.factorial(d + 1) for d in range(O)]
            s_q = s.Q
            s.Q = s.Q.copy()
            s.Q[idx] = Qb
            D = [d[:, :9, :] for d in s.derivatives(idx)]
            s.Q = s_q
            T = sum(cd[d] * D[d] for d in range(O))
            lam = lq[idx]
            mu = sum(np.transpose(Ae[idx, c], (0, 2, 1)) @ lam @ K3[c].T for c in range(3))
            for i in range(4):
                mu += ((np.transpose(Aem[idx, i], (0, 2, 1)) @ lam) @ b.Fh[i].T) @ b.Ft[i].T
            mu += lb1[idx]
            coa = s.has_coarser[idx]
            fin = s.has_finer[idx]
            mu[coa] += lb3[idx[coa]]
            muh = np.zeros_like(mu)
            muh[fin] = lb2[idx[fin]]
            lb1[idx] = 0.0
            lb2[idx[fin]] = 0.0
            if n % 2 == 0:
                lb3[idx[coa]] = 0.0
            G = [None] * O
            G[O - 1] = cd[O - 1] * mu + ch[O - 1] * muh
            for d in range(O - 2, -1, -1):
                G[d] = cd[d] * mu + ch[d] * muh - sum(np.transpose(Ae[idx, c], (0, 2, 1)) @ G[d + 1] @ K3[c]
                                                      for c in range(3))
            for c in range(3):
                acc = lam @ np.transpose(T @ K3[c], (0, 2, 1))
                for d in range(O - 1):
                    acc -= G[d + 1] @ np.transpose(D[d] @ K3[c].T, (0, 2, 1))
                Wc[idx, c] += acc
            for i in range(4):
                Wm[idx, i] += lam @ np.transpose((T @ b.Ft[i]) @ b.Fh[i], (0, 2, 1))
            lq[idx] = lam + G[0]
    return J, _contract(s, Wc, Wm, Wp), lq, synth
