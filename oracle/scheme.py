"""Oracle: ADER-DG time, volume and surface kernels with clustered LTS (test infrastructure).

Follows Sec. III-A and Sec. V-B of the paper in their order and notation:

* time kernel: Cauchy-Kowalevski derivatives (Eqs. ader_derivative_elastic and
  ader_derivative_anelastic, read with -omega_l on the memory term) and the Taylor
  integral T_k(t0, dt) = sum_d dt^(d+1)/(d+1)! d^d Q_k (Eq. ader_taylor);
* volume kernel: V^e = sum_c Abar^e_c T^e K_c + sum_l E^l T^{a,l},
  V^{a,l} = omega_l (sum_c Abar^a_c T^e K_c - T^{a,l});
* local surface kernel: S^{e_L} = sum_i A~e-_i (T^e F~_i) F^_i and
  S^{a_L,l} = omega_l sum_i A~a-_i (T^e F~_i) F^_i;
* neighbour surface kernel: the same with A~+, the neighbour's buffer and F-_{j,h};
* update (Eq. update): Q <- ((Q + V) + S^L) in the local step, Q <- Q + S^N in the
  neighbouring step;
* LTS buffers (Eq. lts_buffers): B1 = T^e(dt_k), B2 = T^e(dt_k/2) for elements with a
  finer neighbour, B3 = T^e(dt_k) at even step index n_k and B3 += T^e(dt_k) at odd
  n_k for elements with a coarser neighbour; a neighbour update reads B1 (same
  cluster), B3 (finer neighbour), B2 (coarser neighbour, first half of its step)
  or B1 - B2 (second half). All neighbour steps ending at a time level run before
  the time predictions starting there (the Fig. 5 walk-through).

Readings for what the paper leaves open: the moment-tensor point source adds
-M_ij (int s dt) phi_b(xi_s) / |det J| to the stress DOFs of the source element in
its neighbouring step (the time integral by O-point Gauss-Legendre); receivers are
sampled at t_j = j dt_rec inside each predicted step [t_n, t_n + dt) by the Taylor
series sum_d (t_j - t_n)^d / d! d^d Q evaluated at the receiver; the discrete energy
is sum_k |det J_k| sum_b (rho |v_b|^2 / 2 + sigma_b : C^-1 sigma_b / 2).

Elements of one phase are processed as a batch with numpy matmuls; each element's
arithmetic is independent of the others, so this equals an element-by-element loop.
"""
import math

import numpy as np
from numpy.polynomial.legendre import leggauss

from .basis import Basis
from .mesh import Mesh, BC_ABSORBING, BC_FREE
from . import physics as ph
from . import lts as ltsmod


def ricker(t, f0, t0):
    a = (np.pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


class Solver:
    """FP64 ADER-DG solver for one mesh.

    order O in {3,4,5}; n_mech m in {0, 3, ...}; material arrays per element
    (rho, vp, vs, and qp, qs when m > 0); relaxation band [f_min, f_max] in Hz.
    """

    def __init__(self, order, n_mech, mesh, rho, vp, vs, qp=None, qs=None, f_min=0.1, f_max=5.0):
        self.order = order
        self.m = n_mech
        self.mesh = mesh
        self.basis = Basis(order)
        self.nb = self.basis.nb
        self.nq = 9 + 6 * n_mech
        K = mesh.K
        self.rho = np.asarray(rho, dtype=float)
        self.vp = np.asarray(vp, dtype=float)
        self.vs = np.asarray(vs, dtype=float)
        self.lam, self.mu = ph.lame(self.rho, self.vp, self.vs)
        # star matrices (Sec. III-A)
        self.Ae = np.zeros((K, 3, 9, 9))
        for k in range(K):
            jac = ph.elastic_jacobians(self.lam[k], self.mu[k], self.rho[k])
            self.Ae[k] = ph.star_matrices(jac, mesh.Jinv[k])
        if n_mech > 0:
            self.omega = ph.relaxation_frequencies(n_mech, f_min, f_max)
            aj = ph.anelastic_jacobians()
            self.Aa = np.einsum("dij,kcd->kcij", aj, mesh.Jinv)
            self.E = np.zeros((K, n_mech, 9, 6))
            for k in range(K):
                ylam, ymu = ph.anelastic_coefficients(self.lam[k], self.mu[k], qp[k], qs[k], self.omega)
                for l in range(n_mech):
                    self.E[k, l] = ph.coupling_matrix(self.lam[k], self.mu[k], ylam[l], ymu[l])
        # flux solvers per face (Sec. III-A, "element-local flux solvers")
        self.Aem = np.zeros((K, 4, 9, 9))
        self.Aep = np.zeros((K, 4, 9, 9))
        self.Aam = np.zeros((K, 4, 6, 9))
        self.Aap = np.zeros((K, 4, 6, 9))
        for k in range(K):
            mat_k = (self.lam[k], self.mu[k], self.rho[k])
            for i in range(4):
                bc = mesh.face_bc[k, i]
                nb = mesh.nbr[k, i]
                if bc == BC_FREE:
                    kind, mat_o = "free", mat_k
                elif bc == BC_ABSORBING:
                    kind, mat_o = "absorbing", mat_k
                else:
                    kind, mat_o = "interior", (self.lam[nb], self.mu[nb], self.rho[nb])
                em, ep, am, ap = ph.flux_solvers(mesh.normal[k, i], mesh.area[k, i], mesh.detJ[k],
                                                 mat_k, mat_o, kind)
                self.Aem[k, i], self.Aep[k, i], self.Aam[k, i], self.Aap[k, i] = em, ep, am, ap
        self.Q = np.zeros((K, self.nq, self.nb))
        self.sources = []
        self.receivers = []
        # one part of a partitioned run (oracle.partitioned): the elements this solver
        # updates (None: all) and the supplier of face-local messages for faces whose
        # neighbour lies in another part (None: none)
        self.owned = None
        self.remote_h = None

    # ---------------------------------------------------------------- set-up
    def quadrature_points(self):
        """Physical quadrature points (K, n_qp, 3) of the projection rule."""
        m = self.mesh
        return m.x0[:, None, :] + np.einsum("kdc,qc->kqd", m.J, self.basis.qp)

    def project(self, fn):
        """Q_k = L2 projection of fn(x) -> (N, nq) onto each element's basis."""
        pts = self.quadrature_points()
        K, nqp, _ = pts.shape
        vals = np.asarray(fn(pts.reshape(-1, 3)), dtype=float).reshape(K, nqp, self.nq)
        phq = self.basis.phi(self.basis.qp) * self.basis.qw[:, None]     # (nqp, B)
        self.Q = np.einsum("kpq,pb->kqb", vals, phq)

    def add_point_source(self, x, m6, f0, t0, m0=1.0):
        k = self.mesh.locate(x)
        xi = self.mesh.xi_of(k, x)
        phi = self.basis.phi(xi[None, :])[0]
        self.sources.append(dict(elem=k, phi=phi, m6=np.asarray(m6, dtype=float) * m0, f0=f0, t0=t0))

    def add_receiver(self, x, dt_rec):
        k = self.mesh.locate(x)
        xi = self.mesh.xi_of(k, x)
        phi = self.basis.phi(xi[None, :])[0]
        self.receivers.append(dict(elem=k, phi=phi, dt=dt_rec, t=[], v=[]))
        return len(self.receivers) - 1

    # ----------------------------------------------------------- time kernel
    def derivatives(self, idx):
        """[d^d Q / dt^d for d = 0..O-1] of elements idx (Cauchy-Kowalevski)."""
        K3 = self.basis.K
        D = [self.Q[idx].copy()]
        m = self.m
        for d in range(self.order - 1):
            X = D[d]
            Xe = X[:, :9, :]
            Y = [Xe @ K3[c].T for c in range(3)]
            nxt = np.zeros_like(X)
            nxt[:, :9, :] = -(self.Ae[idx, 0] @ Y[0] + self.Ae[idx, 1] @ Y[1] + self.Ae[idx, 2] @ Y[2])
            if m > 0:
                for l in range(m):
                    nxt[:, :9, :] += self.E[idx, l] @ X[:, 9 + 6 * l:15 + 6 * l, :]
                S = self.Aa[idx, 0] @ Y[0] + self.Aa[idx, 1] @ Y[1] + self.Aa[idx, 2] @ Y[2]
                for l in range(m):
                    nxt[:, 9 + 6 * l:15 + 6 * l, :] = self.omega[l] * (-S - X[:, 9 + 6 * l:15 + 6 * l, :])
            D.append(nxt)
        return D

    def taylor(self, D, tau):
        """T(t0, tau) = sum_d tau^(d+1)/(d+1)! D_d (Eq. ader_taylor)."""
        T = np.zeros_like(D[0])
        for d in range(self.order):
            T += (tau ** (d + 1) / math.factorial(d + 1)) * D[d]
        return T

    # --------------------------------------------------------- volume kernel
    def volume(self, idx, T):
        K3 = self.basis.K
        Te = T[:, :9, :]
        Z = [Te @ K3[c] for c in range(3)]
        V = np.zeros_like(T)
        V[:, :9, :] = self.Ae[idx, 0] @ Z[0] + self.Ae[idx, 1] @ Z[1] + self.Ae[idx, 2] @ Z[2]
        if self.m > 0:
            for l in range(self.m):
                V[:, :9, :] += self.E[idx, l] @ T[:, 9 + 6 * l:15 + 6 * l, :]
            S = self.Aa[idx, 0] @ Z[0] + self.Aa[idx, 1] @ Z[1] + self.Aa[idx, 2] @ Z[2]
            for l in range(self.m):
                V[:, 9 + 6 * l:15 + 6 * l, :] = self.omega[l] * (S - T[:, 9 + 6 * l:15 + 6 * l, :])
        return V

    # -------------------------------------------------------- surface kernels
    def _surface_to_dofs(self, Se, Sa):
        out = np.zeros((Se.shape[0], self.nq, self.nb))
        out[:, :9, :] = Se
        for l in range(self.m):
            out[:, 9 + 6 * l:15 + 6 * l, :] = self.omega[l] * Sa
        return out

    def local_surface(self, idx, T):
        b = self.basis
        Te = T[:, :9, :]
        Se = np.zeros((len(idx), 9, self.nb))
        Sa = np.zeros((len(idx), 6, self.nb))
        for i in range(4):
            G = Te @ b.Ft[i]
            Se += (self.Aem[idx, i] @ G) @ b.Fh[i]
            if self.m > 0:
                Sa += (self.Aam[idx, i] @ G) @ b.Fh[i]
        return self._surface_to_dofs(Se, Sa)

    def neighbour_surface(self, idx, buffers, given=None):
        """buffers[i]: (len(idx), 9, B) time-integrated neighbour DOFs for face i
        (rows of boundary faces are ignored). given[i], if not None: (mask over idx, H)
        with H = X F-_{j,h} (9 x F) already formed by the neighbour's part for the masked
        faces (Sec. V-C face-local messages); their buffer rows are not used."""
        b = self.basis
        mesh = self.mesh
        Se = np.zeros((len(idx), 9, self.nb))
        Sa = np.zeros((len(idx), 6, self.nb))
        for i in range(4):
            nb = mesh.nbr[idx, i]
            has = nb >= 0
            if not np.any(has):
                continue
            sel = idx[has]
            H = np.zeros((len(sel), 9, b.nf))
            jj = mesh.nbr_face[sel, i]
            hh = mesh.nbr_orient[sel, i]
            X = buffers[i][has]
            msg = np.zeros(len(sel), dtype=bool)
            if given is not None and given[i] is not None:
                gmask, gH = given[i]
                msg = gmask[has]
                H[msg] = gH[np.cumsum(gmask)[has][msg] - 1]
            for j in range(4):
                for h in range(3):
                    mk = (jj == j) & (hh == h) & ~msg
                    if np.any(mk):
                        H[mk] = X[mk] @ b.Fb[j][h]
            Se[has] += (self.Aep[sel, i] @ H) @ b.Fh[i]
            if self.m > 0:
                Sa[has] += (self.Aap[sel, i] @ H) @ b.Fh[i]
        return self._surface_to_dofs(Se, Sa)

    # ------------------------------------------------------- source / receiver
    def _apply_sources(self, idx, t_a, t_b):
        if not self.sources:
            return
        gx, gw = leggauss(self.order)
        tm = 0.5 * (t_a + t_b) + 0.5 * (t_b - t_a) * gx
        members = set(int(k) for k in idx)
        for s in self.sources:
            k = s["elem"]
            if k not in members:
                continue
            integ = 0.5 * (t_b - t_a) * np.sum(gw * ricker(tm, s["f0"], s["t0"]))
            self.Q[k, :6, :] += (-s["m6"] * integ)[:, None] * (s["phi"] / self.mesh.detJ[k])[None, :]

    def _sample_receivers(self, idx, D, t_a, t_b):
        if not self.receivers:
            return
        members = {int(k): p for p, k in enumerate(idx)}
        for r in self.receivers:
            p = members.get(r["elem"])
            if p is None:
                continue
            j = max(int(math.floor(t_a / r["dt"])) - 1, 0)
            while j * r["dt"] < t_b:
                tj = j * r["dt"]
                if tj >= t_a:
                    val = np.zeros(9)
                    for d in range(self.order):
                        val += ((tj - t_a) ** d / math.factorial(d)) * (D[d][p, :9, :] @ r["phi"])
                    r["t"].append(tj)
                    r["v"].append(val)
                j += 1

    def seismogram(self, rid):
        r = self.receivers[rid]
        return np.array(r["t"]), np.array(r["v"]).reshape(-1, 9)

    # --------------------------------------------------------------- energy
    def energy(self):
        """Discrete elastic energy sum_k |det J| sum_b (rho|v_b|^2/2 + sig_b:C^-1 sig_b/2)."""
        Q = self.Q
        kin = 0.5 * self.rho[:, None] * np.sum(Q[:, 6:9, :] ** 2, axis=1)
        sig = np.moveaxis(Q[:, :6, :], 1, 2)
        pot = ph.compliance_energy_density(sig, self.lam[:, None], self.mu[:, None])
        return float(np.sum(self.mesh.detJ[:, None] * (kin + pot)))

    # ------------------------------------------------------ global time stepping
    def time_step_gts(self, cfl):
        dt = ltsmod.cfl_time_steps(self.mesh.dins, self.vp, self.order, cfl)
        return float(dt.min())

    def run_gts(self, dt, n_steps):
        """Global time stepping: predict+local for all, then neighbour for all.

        Step number n (counted over all calls) covers [n dt, (n+1) dt]."""
        K = self.mesh.K
        idx = np.arange(K)
        n0 = getattr(self, "gts_steps_done", 0)
        for n in range(n0, n0 + n_steps):
            t_a = n * dt
            t_b = (n + 1) * dt
            D = self.derivatives(idx)
            self._sample_receivers(idx, D, t_a, t_b)
            T = self.taylor(D, dt)
            B1 = T[:, :9, :].copy()
            self.Q[idx] = (self.Q[idx] + self.volume(idx, T)) + self.local_surface(idx, T)
            bufs = [B1[np.maximum(self.mesh.nbr[idx, i], 0)] for i in range(4)]
            self.Q[idx] = self.Q[idx] + self.neighbour_surface(idx, bufs)
            self._apply_sources(idx, t_a, t_b)
        self.gts_steps_done = n0 + n_steps

    # ------------------------------------------------------- local time stepping
    def setup_clusters(self, n_clusters, cfl, lam=None, clusters=None):
        """Cluster set-up (Sec. V-A). lam None: search; clusters given: forced."""
        dt = ltsmod.cfl_time_steps(self.mesh.dins, self.vp, self.order, cfl)
        self.dt_min = float(dt.min())
        if clusters is not None:
            self.clusters = np.asarray(clusters, dtype=np.int64)
            self.lam_lts = 1.0 if lam is None else lam
            self.n_clusters = n_clusters
        elif lam is None:
            self.lam_lts, self.clusters, _ = ltsmod.search_lambda(dt, self.mesh.nbr, n_clusters)
            self.n_clusters = n_clusters
        else:
            self.lam_lts = lam
            self.clusters = ltsmod.normalise(ltsmod.assign_clusters(dt, lam, n_clusters), self.mesh.nbr)
            self.n_clusters = n_clusters
        self.speedup = ltsmod.theoretical_speedup(self.clusters, self.lam_lts)
        self.delta = self.lam_lts * self.dt_min
        nbr = self.mesh.nbr
        c = self.clusters
        cn = np.where(nbr >= 0, c[np.maximum(nbr, 0)], c[:, None])
        if np.any(np.abs(cn - c[:, None]) > 1):
            raise ValueError("clusters are not normalised")
        self.has_finer = np.any(cn < c[:, None], axis=1)
        self.has_coarser = np.any(cn > c[:, None], axis=1)
        K = self.mesh.K
        self.B1 = np.full((K, 9, self.nb), np.nan)
        self.B2 = np.full((K, 9, self.nb), np.nan)
        self.B3 = np.full((K, 9, self.nb), np.nan)
        self.s_now = 0

    def _predict_local(self, l, n):
        idx = np.nonzero(self.clusters == l)[0]
        if self.owned is not None:
            idx = idx[self.owned[idx]]
        if len(idx) == 0:
            return
        dl = self.delta * 2.0 ** l
        s0 = n * 2 ** l
        t_a = s0 * self.delta
        t_b = (s0 + 2 ** l) * self.delta
        D = self.derivatives(idx)
        self._sample_receivers(idx, D, t_a, t_b)
        T = self.taylor(D, dl)
        self.B1[idx] = T[:, :9, :]
        fin = self.has_finer[idx]
        if np.any(fin):
            Th = self.taylor([d[fin] for d in D], 0.5 * dl)
            self.B2[idx[fin]] = Th[:, :9, :]
        coa = self.has_coarser[idx]
        if np.any(coa):
            if n % 2 == 0:
                self.B3[idx[coa]] = T[coa, :9, :]
            else:
                self.B3[idx[coa]] = self.B3[idx[coa]] + T[coa, :9, :]
        self.Q[idx] = (self.Q[idx] + self.volume(idx, T)) + self.local_surface(idx, T)

    def _neighbour(self, l, n):
        idx = np.nonzero(self.clusters == l)[0]
        if self.owned is not None:
            idx = idx[self.owned[idx]]
        # the message exchange runs even when this part has no element of cluster l
        given = self.remote_h(l, n, idx) if self.remote_h is not None else None
        if len(idx) == 0:
            return
        nbr = self.mesh.nbr
        bufs = []
        for i in range(4):
            nb = np.maximum(nbr[idx, i], 0)
            cn = self.clusters[nb]
            X = self.B1[nb].copy()
            fin = cn == l - 1
            X[fin] = self.B3[nb[fin]]
            coa = cn == l + 1
            if n % 2 == 0:
                X[coa] = self.B2[nb[coa]]
            else:
                X[coa] = self.B1[nb[coa]] - self.B2[nb[coa]]
            X[nbr[idx, i] < 0] = 0.0
            bufs.append(X)
        self.Q[idx] = self.Q[idx] + self.neighbour_surface(idx, bufs, given)
        s0 = n * 2 ** l
        self._apply_sources(idx, s0 * self.delta, (s0 + 2 ** l) * self.delta)

    def run_lts(self, n_finest):
        """Advance n_finest finest steps (a multiple of 2^(N_c-1)) from time level s_now."""
        period = 2 ** (self.n_clusters - 1)
        if n_finest % period != 0:
            raise ValueError("n_finest must be a multiple of 2^(N_c-1)")
        s_begin = self.s_now
        s_end = s_begin + n_finest
        for s in range(s_begin, s_end + 1):
            for l in range(self.n_clusters):
                if s > s_begin and s % 2 ** l == 0:
                    self._neighbour(l, s // 2 ** l - 1)
            if s < s_end:
                for l in range(self.n_clusters):
                    if s % 2 ** l == 0:
                        self._predict_local(l, s // 2 ** l)
        self.s_now = s_end

    def element_updates(self, n_finest):
        """Element updates performed by n_finest finest steps of LTS."""
        return int(np.sum(n_finest // 2 ** self.clusters))
