"""Pins for the oracle's clustering (Sec. V-A) and LTS buffers/schedule (Sec. V-B, Fig. 5)."""
import json
import math
import os

import numpy as np

from oracle import lts
from oracle.mesh import Mesh
from oracle.scheme import Solver

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))


def test_lambda_example_intervals():
    g = GOLD["lambda_example"]
    lam = g["lambda"]
    # C1 = [lam, 2 lam), C2 = [2 lam, 4 lam) in units of dt_min (dt_min = 1 here)
    assert g["C1"] == [lam, 2 * lam] and g["C2"] == [2 * lam, 4 * lam]
    dt = np.array([1.0, g["C1"][1] - 1e-9, g["C2"][0], g["C2"][1] - 1e-9, g["C2"][1]])
    c = lts.assign_clusters(dt, lam, 3)
    assert list(c) == [0, 0, 1, 1, 2]
    # the bulk in (3, 4) advances with 3.0 (lam=0.75) instead of 2.0 (lam=1)
    bulk = np.array([1.0, 3.5])
    for lam_, want in ((lam, g["bulk_step"]), (1.0, g["bulk_step_lambda1"])):
        cl = lts.assign_clusters(bulk, lam_, 3)[1]
        assert math.isclose(2.0 ** cl * lam_ * 1.0, want)


def test_cluster_example_three_lambda_dtmin():
    g = GOLD["cluster_example"]
    for lam in (0.51, 0.75, 1.0):
        dt = np.array([1.0, g["dt_over_lambda_dtmin"] * lam])
        assert lts.assign_clusters(dt, lam, 5)[1] + 1 == g["cluster_1based"]


def test_half_open_intervals_and_open_last_cluster():
    dt = np.array([1.0, 2.0, 4.0, 1000.0])
    assert list(lts.assign_clusters(dt, 1.0, 3)) == [0, 1, 2, 2]


def test_normalisation_example():
    g = GOLD["normalisation_example"]
    # chain a - b - c with a in C1 (index 0) and c initially C3 next to a
    nbr = np.array([[1, 2, -1, -1], [0, -1, -1, -1], [0, -1, -1, -1]])
    c = lts.normalise(np.array([g["neighbour"] - 1, 0, g["from"] - 1]), nbr)
    assert c[2] + 1 == g["to"]
    # fixed point propagates along chains
    nbr = np.array([[1, -1, -1, -1], [0, 2, -1, -1], [1, 3, -1, -1], [2, -1, -1, -1]])
    assert list(lts.normalise(np.array([0, 4, 4, 4]), nbr)) == [0, 1, 2, 3]


def test_lambda_search():
    assert GOLD["lambda_step"]["step"] == 0.01
    nbr = -np.ones((101, 4), dtype=np.int64)
    dt = np.array([1.0] + [3.5] * 100)
    lam, c, s = lts.search_lambda(dt, nbr, 3)
    # 4*lam <= 3.5 puts the bulk into C3: lam = 0.87 is the largest on the 0.01 grid
    assert math.isclose(lam, 0.87) and c[1] == 2 and c[0] == 0
    assert math.isclose(s, 101 * 0.87 / (1 + 100 / 4))
    # one cluster: lam = 1, speedup 1
    lam, c, s = lts.search_lambda(dt, nbr, 1)
    assert lam == 1.0 and np.all(c == 0) and s == 1.0


def _star_mesh():
    """Tetrahedron k (index 0) with four face neighbours glued on its faces."""
    core = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    xyz = list(core)
    tets = [[0, 1, 2, 3]]
    faces = ((0, 2, 1), (0, 1, 3), (0, 3, 2), (1, 2, 3))
    cen = core.mean(axis=0)
    for f in faces:
        fc = core[list(f)].mean(axis=0)
        apex = fc + 1.2 * (fc - cen)
        xyz.append(apex)
        t = [f[0], f[1], f[2], len(xyz) - 1]
        x = np.array(xyz)[t]
        if np.linalg.det(np.stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]], 1)) < 0:
            t[1], t[2] = t[2], t[1]
        tets.append(t)
    tets = np.array(tets)
    bc = np.zeros((5, 4), dtype=np.int64)
    for e in range(1, 5):
        for i, f in enumerate(faces):
            if not set(tets[e, list(f)]) <= {0, 1, 2, 3}:
                bc[e, i] = 1
    return np.array(xyz) * 100.0, tets, bc


def test_fig5_walkthrough_buffers_and_reads():
    """k steps 2dt, k1 dt, k2/k3 2dt, k4 4dt (Fig. 5). Checks what k stores in
    B1/B2/B3 and which data each neighbour reads, against Taylor integrals of k's own
    derivatives recorded at t0 and t2."""
    xyz, tet, bc = _star_mesh()
    mesh = Mesh(xyz, tet, bc)
    K = mesh.K
    s = Solver(3, 0, mesh, np.full(K, 2700.0), np.full(K, 6000.0), np.full(K, 3464.0))
    rng = np.random.default_rng(0)
    s.Q = rng.normal(size=s.Q.shape)
    s.Q[:, :6] *= 1e6
    kf = {int(mesh.nbr[0, i]): i for i in range(4)}          # neighbour element -> face of k
    k1, k2, k3, k4 = sorted(kf)
    clusters = np.array([1, 0, 1, 1, 2])
    clusters[[k1, k2, k3, k4]] = [0, 1, 1, 2]
    s.setup_clusters(3, 0.5, lam=1.0, clusters=clusters)
    dt = s.delta
    recorded_D = {}
    reads = []
    orig_deriv, orig_nbr = s.derivatives, s.neighbour_surface

    def deriv(idx):
        D = orig_deriv(idx)
        if 0 in set(idx.tolist()):
            p = list(idx).index(0)
            recorded_D[s.s_clock] = [d[p].copy() for d in D]
        return D

    def nbr_surface(idx, bufs, given=None):
        for p, e in enumerate(idx):
            for i in range(4):
                if mesh.nbr[e, i] == 0:
                    reads.append((s.s_clock, int(e), bufs[i][p].copy()))
        return orig_nbr(idx, bufs)

    s.derivatives, s.neighbour_surface = deriv, nbr_surface
    # drive the schedule step by step to know the time level of every call
    orig_pl, orig_nb = s._predict_local, s._neighbour

    def pl(l, n):
        s.s_clock = n * 2 ** l
        orig_pl(l, n)

    def nb(l, n):
        s.s_clock = (n + 1) * 2 ** l
        orig_nb(l, n)

    s._predict_local, s._neighbour = pl, nb
    s.run_lts(4)
    assert np.all(np.isfinite(s.Q))                         # no unset (NaN) buffer was read

    def T(s0, a, b):
        """int_{a}^{b} of k's Taylor expansion about time level s0 (units of dt), elastic rows."""
        D = recorded_D[s0]
        out = np.zeros_like(D[0][:9])
        for d in range(len(D)):
            out += ((b - s0) ** (d + 1) - (a - s0) ** (d + 1)) * dt ** (d + 1) / math.factorial(d + 1) * D[d][:9]
        return out

    assert sorted(recorded_D) == [0, 2]
    by = {}
    for tl, e, buf in reads:
        by.setdefault(e, []).append((tl, buf))
    tol = 1e-12
    # k1 (dt): [t0,t1] from B2 = T(t0, dt); [t1,t2] from B1 - B2 = T(t1, dt); then from k's prediction at t2
    exp_k1 = [(1, T(0, 0, 1)), (2, T(0, 1, 2)), (3, T(2, 2, 3)), (4, T(2, 3, 4))]
    # k2, k3 (2dt): B1 = T(t0, 2dt), then T(t2, 2dt)
    exp_k2 = [(2, T(0, 0, 2)), (4, T(2, 2, 4))]
    # k4 (4dt): B3 = T(t0, 2dt) + T(t2, 2dt) = T(t0, 4dt) accumulated
    exp_k4 = [(4, T(0, 0, 2) + T(2, 2, 4))]
    for e, exp in ((k1, exp_k1), (k2, exp_k2), (k3, exp_k2), (k4, exp_k4)):
        got = by[e]
        assert [g[0] for g in got] == [x[0] for x in exp]
        for (tl, buf), (_, want) in zip(got, exp):
            assert np.abs(buf - want).max() <= tol * np.abs(want).max()


def test_dependency_cone_of_n_finest_steps():
    """After n finest LTS steps an element depends only on data within n face hops: the
    oracle on the (n+1)-hop ball (cut faces absorbing) reproduces the full-mesh result at
    the ball's centre. This is the basis of the full-size sampled GPU parity test."""
    from paper_2202_10313_gb300 import synth
    m = synth.graded_box(6, 6, 4, 250.0, 125.0, seed=4)
    mat = synth.random_layers(m, n_layers=3, seed=6)
    om = Mesh(m["xyz"], m["tet"], m["face_bc"])
    full = Solver(3, 3, om, mat["rho"], mat["vp"], mat["vs"], mat["qp"], mat["qs"])
    full.setup_clusters(3, 0.5)
    n = 4
    init = np.random.default_rng(1).normal(size=full.Q.shape)
    full.Q = init.copy()
    full.run_lts(n)
    for k in (100, 400, 700):
        seen, front = {k}, [k]
        for _ in range(n + 1):
            nxt = []
            for e in front:
                for nb in om.nbr[e]:
                    if nb >= 0 and int(nb) not in seen:
                        seen.add(int(nb))
                        nxt.append(int(nb))
            front = nxt
        ball = np.array(sorted(seen))
        assert len(ball) < om.K
        tet = m["tet"][ball]
        uv, inv = np.unique(tet, return_inverse=True)
        bc = m["face_bc"][ball].copy()
        bc[(om.nbr[ball] >= 0) & ~np.isin(om.nbr[ball], ball)] = 1
        sm = Mesh(m["xyz"][uv], inv.reshape(tet.shape), bc)
        sub = Solver(3, 3, sm, mat["rho"][ball], mat["vp"][ball], mat["vs"][ball], mat["qp"][ball], mat["qs"][ball])
        sub.setup_clusters(3, 0.5, lam=full.lam_lts, clusters=full.clusters[ball])
        sub.delta = full.delta
        sub.Q = init[ball].copy()
        sub.run_lts(n)
        got = sub.Q[np.searchsorted(ball, k)]
        assert np.abs(got - full.Q[k]).max() <= 1e-12 * np.abs(full.Q[k]).max()
