"""Pins for the oracle's full ADER-DG scheme: convergence, LTS, energy, attenuation,
receivers and source (Sec. III-A, Sec. V-B)."""
import math

import numpy as np
import pytest

from oracle.lts import normalise
from oracle.mesh import Mesh
from oracle.scheme import Solver, ricker
from paper_2202_10313_gb300 import synth

RHO, VP, VS = 2700.0, 6000.0, 3464.0
KVEC = 2 * np.pi * np.array([1.0, 1.0, 1.0])


def _cube_solver(n, order, m=0, qs=None):
    mm = synth.periodic_cube(n)
    mesh = Mesh(mm["xyz"], mm["tet"], mm["face_bc"], mm["period"])
    K = mesh.K
    kw = {}
    if m:
        kw = dict(qp=np.full(K, 2 * qs), qs=np.full(K, qs))
    return Solver(order, m, mesh, np.full(K, RHO), np.full(K, VP), np.full(K, VS), **kw), mesh


def _rel_err(a, b, rows):
    return np.sqrt(np.sum((a[:, rows] - b[:, rows]) ** 2) / np.sum(b[:, rows] ** 2))


@pytest.mark.parametrize("order", [3, 4, 5])
def test_plane_wave_convergence(order):
    """P plane wave on the periodic cube: L2 error drops at rate ~O (3x3x3 -> 6x6x6 hexes)."""
    pw = synth.p_plane_wave(RHO, VP, VS, KVEC)
    tend = 0.25 / (VP * np.linalg.norm(KVEC) / (2 * np.pi))
    errs = []
    for n in (3, 6):
        s, mesh = _cube_solver(n, order)
        s.project(lambda x: pw(x, 0.0))
        dt = s.time_step_gts(0.5)
        nst = int(math.ceil(tend / dt))
        s.run_gts(tend / nst, nst)
        ex, _ = _cube_solver(n, order)
        ex.project(lambda x: pw(x, tend))
        errs.append(_rel_err(s.Q, ex.Q, slice(6, 9)))
    rate = math.log2(errs[0] / errs[1])
    assert rate > order - 0.6, (errs, rate)


@pytest.mark.parametrize("order", [3, 4, 5])
def test_s_plane_wave_convergence(order):
    """S plane wave (velocity along (1, -1, 0), k = 2 pi (1, 1, 1)) on the periodic cube:
    the L2 error of the velocities and of the stresses drops at rate ~O (3x3x3 -> 6x6x6)."""
    sw = synth.s_plane_wave(RHO, VS, KVEC, [1.0, -1.0, 0.0])
    tend = 0.25 / (VS * np.linalg.norm(KVEC) / (2 * np.pi))
    errs_v, errs_s = [], []
    for n in (3, 6):
        s, mesh = _cube_solver(n, order)
        s.project(lambda x: sw(x, 0.0))
        dt = s.time_step_gts(0.5)
        nst = int(math.ceil(tend / dt))
        s.run_gts(tend / nst, nst)
        ex, _ = _cube_solver(n, order)
        ex.project(lambda x: sw(x, tend))
        errs_v.append(_rel_err(s.Q, ex.Q, slice(6, 9)))
        errs_s.append(_rel_err(s.Q, ex.Q, slice(0, 6)))
    for errs in (errs_v, errs_s):
        rate = math.log2(errs[0] / errs[1])
        assert rate > order - 0.6, (errs, rate)


def test_lts_single_cluster_equals_gts_bitwise():
    pw = synth.p_plane_wave(RHO, VP, VS, KVEC)
    a, _ = _cube_solver(3, 3)
    b, _ = _cube_solver(3, 3)
    a.project(lambda x: pw(x, 0.0))
    b.project(lambda x: pw(x, 0.0))
    dt = a.time_step_gts(0.5)
    a.run_gts(dt, 7)
    b.setup_clusters(1, 0.5)
    assert b.lam_lts == 1.0 and b.delta == dt
    b.run_lts(7)
    assert np.array_equal(a.Q, b.Q)


def test_forced_three_cluster_lts_converges_and_tracks_gts():
    pw = synth.p_plane_wave(RHO, VP, VS, KVEC)
    tend = 0.25 / (VP * np.sqrt(3))
    errs, gaps = [], []
    for n in (3, 6):
        s, mesh = _cube_solver(n, 3)
        s.project(lambda x: pw(x, 0.0))
        x = mesh.centroid[:, 0]
        c = normalise(np.digitize(x, [1 / 3, 2 / 3]), mesh.nbr)
        assert set(c.tolist()) == {0, 1, 2}
        s.setup_clusters(3, 0.125, lam=1.0, clusters=c)
        nper = int(math.ceil(tend / (4 * s.delta)))
        s.delta = tend / (4 * nper)
        s.run_lts(4 * nper)
        g, _ = _cube_solver(n, 3)
        g.project(lambda x: pw(x, 0.0))
        g.run_gts(tend / (4 * nper), 4 * nper)
        ex, _ = _cube_solver(n, 3)
        ex.project(lambda x: pw(x, tend))
        errs.append(_rel_err(s.Q, ex.Q, slice(6, 9)))
        gaps.append(_rel_err(s.Q, g.Q, slice(6, 9)))
    assert math.log2(errs[0] / errs[1]) > 2.4
    # LTS differs from GTS by less than the discretisation error
    assert gaps[1] < errs[1]


@pytest.mark.parametrize("order", [3, 4])
def test_energy_non_increasing_periodic(order):
    pw = synth.p_plane_wave(RHO, VP, VS, KVEC)
    s, _ = _cube_solver(3, order)
    s.project(lambda x: pw(x, 0.0))
    dt = s.time_step_gts(0.5)
    e = [s.energy()]
    for _ in range(30):
        s.run_gts(dt, 1)
        e.append(s.energy())
    assert np.all(np.diff(e) <= 1e-13 * e[0])
    assert e[-1] < e[0]


def test_energy_non_increasing_free_surface_and_absorbing_box():
    m = synth.graded_box(3, 3, 3, 100.0, 60.0, seed=9)
    mesh = Mesh(m["xyz"], m["tet"], m["face_bc"])
    mat = synth.layered(m, [60.0], [1500.0, 2500.0])
    s = Solver(3, 0, mesh, mat["rho"], mat["vp"], mat["vs"])
    s.project(synth.gaussian_pulse([150.0, 150.0, -100.0], 80.0, 9))
    dt = s.time_step_gts(0.5)
    e = [s.energy()]
    for _ in range(30):
        s.run_gts(dt, 1)
        e.append(s.energy())
    assert np.all(np.diff(e) <= 1e-13 * e[0])
    assert e[-1] < 0.999 * e[0]


def test_infinite_q_anelastic_equals_elastic_bitwise():
    pw = synth.p_plane_wave(RHO, VP, VS, KVEC)
    a, _ = _cube_solver(3, 3)
    b, _ = _cube_solver(3, 3, m=3, qs=np.inf)
    a.project(lambda x: pw(x, 0.0))
    b.project(lambda x: np.concatenate([pw(x, 0.0), np.zeros((len(x), 18))], axis=1))
    dt = a.time_step_gts(0.5)
    a.run_gts(dt, 5)
    b.run_gts(dt, 5)
    assert np.array_equal(a.Q, b.Q[:, :9])


def test_anelastic_plane_wave_decays_at_target_q():
    """Uniform attenuating medium: an S plane wave's velocity amplitude decays like
    exp(-w t / (2 Q)) up to discretisation error (low-loss limit)."""
    qs = 20.0
    kvec = 2 * np.pi * np.array([1.0, 0.0, 0.0])
    w = np.linalg.norm(kvec) * VS
    s, mesh = _cube_solver(3, 4, m=3, qs=qs)
    # relaxation band around the wave frequency
    from oracle import physics as ph
    s.omega = ph.relaxation_frequencies(3, 0.1 * w / (2 * np.pi), 10 * w / (2 * np.pi))
    lam, mu = ph.lame(RHO, VP, VS)
    ylam, ymu = ph.anelastic_coefficients(lam, mu, 2 * qs, qs, s.omega)
    for k in range(mesh.K):
        for l in range(3):
            s.E[k, l] = ph.coupling_matrix(lam, mu, ylam[l], ymu[l])
    sw = synth.s_plane_wave(RHO, VS, kvec, [0.0, 1.0, 0.0])
    s.project(lambda x: np.concatenate([sw(x, 0.0), np.zeros((len(x), 18))], axis=1))
    a0 = np.sqrt(np.sum(s.Q[:, 6:9] ** 2) + np.sum(s.Q[:, :6] ** 2) / (RHO * VS) ** 2)
    tend = 2 * 2 * np.pi / w
    dt = s.time_step_gts(0.4)
    nst = int(math.ceil(tend / dt))
    s.run_gts(tend / nst, nst)
    a1 = np.sqrt(np.sum(s.Q[:, 6:9] ** 2) + np.sum(s.Q[:, :6] ** 2) / (RHO * VS) ** 2)
    want = math.exp(-w * tend / (2 * qs))
    assert abs(a1 / a0 / want - 1) < 0.05, (a1 / a0, want)


@pytest.mark.parametrize("order", [3])
def test_anelastic_s_plane_wave_convergence(order):
    """Attenuating medium (Q_s = 20, Q_p = 40, three mechanisms around the wave frequency), S
    wave along x polarised along y (Sec. III, anelastic equations with memory variables): one
    Fourier mode of the continuum equations is a 5 x 5 linear ODE in (v_y, sigma_xy,
    theta^l_xy),
        rho v_y'       = d_x sigma_xy,
        sigma_xy'      = mu d_x v_y - 2 mu sum_l Y^mu_l theta^l_xy,
        theta^l_xy'    = omega_l (1/2 d_x v_y - theta^l_xy),
    solved exactly by a matrix exponential. Starting from the elastic S wave with zero memory
    variables, the oracle's velocity, stress and memory-variable errors against that solution
    drop at rate ~O from 3x3x3 to 6x6x6 hexes; a wrong strain factor or coupling sign leaves
    them flat."""
    from scipy.linalg import expm
    from oracle import physics as ph
    qs = 20.0
    k = 2 * np.pi
    w = k * VS
    lam, mu = ph.lame(RHO, VP, VS)
    rows = (7, 3, 12, 18, 24)                 # v_y, sigma_xy, theta^1..3_xy in the state vector

    def setup(n):
        s, mesh = _cube_solver(n, order, m=3, qs=qs)
        s.omega = ph.relaxation_frequencies(3, 0.1 * w / (2 * np.pi), 10 * w / (2 * np.pi))
        ylam, ymu = ph.anelastic_coefficients(lam, mu, 2 * qs, qs, s.omega)
        for e in range(mesh.K):
            for l in range(3):
                s.E[e, l] = ph.coupling_matrix(lam, mu, ylam[l], ymu[l])
        return s, ymu

    def exact(omega, ymu, t):
        # amplitudes of exp(i k x); the field is their imaginary part (sin(k x) at t = 0)
        M = np.zeros((5, 5), complex)
        M[0, 1] = 1j * k / RHO
        M[1, 0] = 1j * k * mu
        for l in range(3):
            M[1, 2 + l] = -2 * mu * ymu[l]
            M[2 + l, 0] = 0.5j * k * omega[l]
            M[2 + l, 2 + l] = -omega[l]
        y = expm(M * t) @ np.array([1.0, -mu / VS, 0.0, 0.0, 0.0], complex)

        def fn(x):
            out = np.zeros((len(x), 27))
            c, sn = np.cos(k * x[:, 0]), np.sin(k * x[:, 0])
            for r, yy in zip(rows, y):
                out[:, r] = yy.imag * c + yy.real * sn
            return out
        return fn

    tend = 0.25 / VS
    errs = []
    for n in (3, 6):
        s, ymu = setup(n)
        s.project(exact(s.omega, ymu, 0.0))
        dt = s.time_step_gts(0.5)
        nst = int(math.ceil(tend / dt))
        s.run_gts(tend / nst, nst)
        ex, _ = setup(n)
        ex.project(exact(s.omega, ymu, tend))
        errs.append([_rel_err(s.Q, ex.Q, sl) for sl in (slice(6, 9), slice(0, 6), slice(9, 27))])
    for e3, e6 in zip(*errs):
        rate = math.log2(e3 / e6)
        assert rate > order - 0.6, (errs, rate)


@pytest.mark.parametrize("kind", ["s", "p"])
@pytest.mark.parametrize("order", [3, 4])
def test_free_surface_standing_waves_converge(kind, order):
    """Traction-free planes z = 0 and z = 1 (free-surface faces, Sec. III), periodic in x and
    y: the standing waves v = cos(k z) cos(w t) with k = 2 pi (S: v_x with sigma_xz; P: v_z
    with sigma_zz and sigma_xx = sigma_yy = lam / (lam + 2 mu) sigma_zz) satisfy the boundary
    condition exactly (their traction sin(k z) vanishes on both planes). The oracle's velocity
    and stress errors against them drop at rate ~O from 3x3x3 to 6x6x6 hexes; an absorbing or
    a rigid treatment of those faces leaves the error flat."""
    lam, mu = RHO * (VP ** 2 - 2 * VS ** 2), RHO * VS ** 2
    c = VS if kind == "s" else VP
    k = 2 * np.pi
    w = k * c

    def standing(t):
        def fn(x):
            out = np.zeros((len(x), 9))
            z = x[:, 2]
            v = np.cos(k * z) * np.cos(w * t)
            sg = -RHO * c * np.sin(k * z) * np.sin(w * t)   # from rho v_t = d_z sigma
            if kind == "s":
                out[:, 6], out[:, 5] = v, sg
            else:
                out[:, 8], out[:, 2] = v, sg
                out[:, 0] = out[:, 1] = sg * lam / (lam + 2 * mu)
            return out
        return fn

    def solver(n):
        m = synth.periodic_slab(n, z_code=2)
        mesh = Mesh(m["xyz"], m["tet"], m["face_bc"], m["period"])
        K = mesh.K
        return Solver(order, 0, mesh, np.full(K, RHO), np.full(K, VP), np.full(K, VS))

    tend = 0.125 / c
    errs = []
    for n in (3, 6):
        s = solver(n)
        s.project(standing(0.0))
        dt = s.time_step_gts(0.5)
        nst = int(math.ceil(tend / dt))
        s.run_gts(tend / nst, nst)
        ex = solver(n)
        ex.project(standing(tend))
        errs.append([_rel_err(s.Q, ex.Q, sl) for sl in (slice(6, 9), slice(0, 6))])
    for e3, e6 in zip(*errs):
        rate = math.log2(e3 / e6)
        assert rate > order - 0.6, (errs, rate)


@pytest.mark.parametrize("kind", ["s", "p"])
@pytest.mark.parametrize("order", [3, 4])
def test_absorbing_planes_pass_a_normally_incident_pulse(kind, order):
    """Absorbing planes z = 0 and z = 1 (Sec. III boundary faces), periodic in x and y: a
    Gaussian P or S pulse travelling along +z (width 0.12, centre 0.6) crosses z = 1 at normal
    incidence, where the absorbing boundary lets it out without reflection, so the field
    inside stays the travelling pulse. After it has moved 0.3 (half of it gone), the oracle's
    velocity and stress errors against that pulse drop at rate ~O from 8 to 16 hexes along z;
    a reflecting (free-surface) treatment leaves a 22 % error."""
    lam, mu = RHO * (VP ** 2 - 2 * VS ** 2), RHO * VS ** 2
    c = VS if kind == "s" else VP

    def pulse(t):
        def fn(x):
            out = np.zeros((len(x), 9))
            f = np.exp(-((x[:, 2] - 0.6 - c * t) / 0.12) ** 2)
            if kind == "s":
                out[:, 6], out[:, 5] = f, -RHO * c * f
            else:
                out[:, 8], out[:, 2] = f, -RHO * c * f
                out[:, 0] = out[:, 1] = -RHO * c * f * lam / (lam + 2 * mu)
            return out
        return fn

    def solver(n):
        m = synth.periodic_slab(n, z_code=1, nxy=2)
        mesh = Mesh(m["xyz"], m["tet"], m["face_bc"], m["period"])
        K = mesh.K
        return Solver(order, 0, mesh, np.full(K, RHO), np.full(K, VP), np.full(K, VS))

    tend = 0.3 / c
    errs = []
    for n in (8, 16):
        s = solver(n)
        s.project(pulse(0.0))
        dt = s.time_step_gts(0.5)
        nst = int(math.ceil(tend / dt))
        s.run_gts(tend / nst, nst)
        ex = solver(n)
        ex.project(pulse(tend))
        errs.append([_rel_err(s.Q, ex.Q, sl) for sl in (slice(6, 9), slice(0, 6))])
    for e8, e16 in zip(*errs):
        rate = math.log2(e8 / e16)
        assert rate > order - 0.6, (errs, rate)


@pytest.mark.parametrize("kind", ["s", "p"])
def test_material_interface_reflects_and_transmits_at_normal_incidence(kind):
    """Welded interface z = 1/2 between two materials (upwind flux with each side's own
    impedance, Sec. III), absorbing planes z = 0 and z = 1, periodic in x and y. A Gaussian P
    or S pulse (width 0.1, centre 0.3) travels along +z and meets the interface at normal
    incidence; continuity of velocity and traction gives the reflected and transmitted
    velocity amplitudes R = (Z1 - Z2) / (Z1 + Z2), T = 2 Z1 / (Z1 + Z2), Z = rho c, the
    transmitted pulse compressed by c2 / c1. After the incident pulse has moved 0.3, the order-4
    oracle's velocity and stress errors against that solution drop at rate ~4 from 12 to 24
    hexes along z. (Any consistent interface flux converges here, one built with a single
    side's impedance too: the Godunov states themselves are pinned against the closed-form
    Riemann solution in the physics tests.)"""
    order = 4
    m1, m2 = (2700.0, 6000.0, 3464.0), (2000.0, 3000.0, 1732.0)      # rho, vp, vs per side

    def side(m):
        rho, vp, vs = m
        mu = rho * vs * vs
        lam = rho * vp * vp - 2 * mu
        c = vs if kind == "s" else vp
        return rho * c, c, lam / (lam + 2 * mu)

    Z1, c1, q1 = side(m1)
    Z2, c2, q2 = side(m2)
    R, T = (Z1 - Z2) / (Z1 + Z2), 2 * Z1 / (Z1 + Z2)

    def f(s):
        return np.exp(-((s - 0.3) / 0.1) ** 2)

    def exact(t):
        def fn(x):
            z = x[:, 2]
            lo = z < 0.5
            inc, ref = f(z - c1 * t), R * f(1.0 - z - c1 * t)
            tra = T * f(0.5 - c1 * t + c1 * (z - 0.5) / c2)
            v = np.where(lo, inc + ref, tra)
            sg = np.where(lo, -Z1 * inc + Z1 * ref, -Z2 * tra)      # sigma = -Z v along +z, +Z v along -z
            out = np.zeros((len(x), 9))
            if kind == "s":
                out[:, 6], out[:, 5] = v, sg
            else:
                out[:, 8], out[:, 2] = v, sg
                out[:, 0] = out[:, 1] = sg * np.where(lo, q1, q2)
            return out
        return fn

    def solver(n):
        m = synth.periodic_slab(n, z_code=1, nxy=2)
        mesh = Mesh(m["xyz"], m["tet"], m["face_bc"], m["period"])
        lo = mesh.centroid[:, 2] < 0.5
        rho, vp, vs = (np.where(lo, a, b) for a, b in zip(m1, m2))
        return Solver(order, 0, mesh, rho, vp, vs)

    tend = 0.3 / c1
    errs = []
    for n in (12, 24):
        s = solver(n)
        s.project(exact(0.0))
        dt = s.time_step_gts(0.5)
        nst = int(math.ceil(tend / dt))
        s.run_gts(tend / nst, nst)
        ex = solver(n)
        ex.project(exact(tend))
        errs.append([_rel_err(s.Q, ex.Q, sl) for sl in (slice(6, 9), slice(0, 6))])
    for e12, e24 in zip(*errs):
        rate = math.log2(e12 / e24)
        assert rate > order - 0.6, (errs, rate)


def test_lts_across_material_interface_converges():
    """Two LTS clusters split by a material interface (Sec. V): the P pulse of the interface
    test above, with the slow side (vp 2,900 against 6,000, so twice the CFL step) in the
    coarser cluster and lam = 1. The pulse crosses from the fine cluster into the coarse one
    through the LTS buffer reads across the interface; the error against the closed-form
    reflection and transmission drops at rate ~4 (order 4, 12 -> 24 hexes along z), and LTS
    stays within the discretisation error of GTS. (A mistake whose effect is below the
    discretisation error here, such as the second half-step reading B2 instead of B1 - B2,
    is caught by the exact buffer checks of the Fig. 5 walkthrough test.)"""
    order = 4
    m1, m2 = (2700.0, 6000.0, 3464.0), (2000.0, 2900.0, 1674.0)      # rho, vp, vs per side

    def side(m):
        rho, vp, vs = m
        mu = rho * vs * vs
        lam = rho * vp * vp - 2 * mu
        return rho * vp, vp, lam / (lam + 2 * mu)

    Z1, c1, q1 = side(m1)
    Z2, c2, q2 = side(m2)
    R, T = (Z1 - Z2) / (Z1 + Z2), 2 * Z1 / (Z1 + Z2)

    def f(s):
        return np.exp(-((s - 0.3) / 0.1) ** 2)

    def exact(t):
        def fn(x):
            z = x[:, 2]
            lo = z < 0.5
            inc, ref = f(z - c1 * t), R * f(1.0 - z - c1 * t)
            tra = T * f(0.5 - c1 * t + c1 * (z - 0.5) / c2)
            out = np.zeros((len(x), 9))
            out[:, 8] = np.where(lo, inc + ref, tra)
            out[:, 2] = np.where(lo, -Z1 * inc + Z1 * ref, -Z2 * tra)
            out[:, 0] = out[:, 1] = out[:, 2] * np.where(lo, q1, q2)
            return out
        return fn

    def solver(n):
        m = synth.periodic_slab(n, z_code=1, nxy=2)
        mesh = Mesh(m["xyz"], m["tet"], m["face_bc"], m["period"])
        lo = mesh.centroid[:, 2] < 0.5
        rho, vp, vs = (np.where(lo, a, b) for a, b in zip(m1, m2))
        return Solver(order, 0, mesh, rho, vp, vs), lo

    tend = 0.3 / c1
    errs, gaps = [], []
    for n in (12, 24):
        s, lo = solver(n)
        s.project(exact(0.0))
        s.setup_clusters(2, 0.5, lam=1.0)
        assert np.array_equal(s.clusters, np.where(lo, 0, 1))
        nper = int(math.ceil(tend / (2 * s.delta)))
        s.delta = tend / (2 * nper)
        s.run_lts(2 * nper)
        ex, _ = solver(n)
        ex.project(exact(tend))
        g, _ = solver(n)
        g.project(exact(0.0))
        g.run_gts(tend / (2 * nper), 2 * nper)
        errs.append([_rel_err(s.Q, ex.Q, sl) for sl in (slice(6, 9), slice(0, 6))])
        gaps.append(_rel_err(s.Q, g.Q, slice(0, 9)))
    for e12, e24 in zip(*errs):
        rate = math.log2(e12 / e24)
        assert rate > order - 0.6, (errs, rate)
    assert gaps[1] < min(errs[1])


def test_receiver_is_exact_point_evaluation():
    """Sampled at the start of each step, the receiver equals the DG polynomial of
    Q^n at the receiver point; mid-step samples come from the Taylor series."""
    pw = synth.p_plane_wave(RHO, VP, VS, KVEC)
    s, mesh = _cube_solver(3, 3)
    s.project(lambda x: pw(x, 0.0))
    dt = s.time_step_gts(0.5)
    xr = np.array([0.31, 0.47, 0.62])
    rid = s.add_receiver(xr, dt)
    k = mesh.locate(xr)
    phi = s.basis.phi(mesh.xi_of(k, xr)[None, :])[0]
    vals = []
    for _ in range(4):
        vals.append(s.Q[k, :9] @ phi)
        s.run_gts(dt, 1)
    t, v = s.seismogram(rid)
    assert np.allclose(t, dt * np.arange(4))
    assert np.abs(v - np.array(vals)).max() <= 1e-13 * np.abs(vals).max()
    # Taylor evaluation at mid-step approximates the exact wave to discretisation error
    s2, _ = _cube_solver(3, 3)
    s2.project(lambda x: pw(x, 0.0))
    rid = s2.add_receiver(xr, dt / 2)
    s2.run_gts(dt, 4)
    t, v = s2.seismogram(rid)
    ex = np.array([pw(xr[None, :], ti)[0] for ti in t])
    assert np.abs(v[:, 6:] - ex[:, 6:]).max() < 0.1


def test_source_injection_matches_closed_form_time_integral():
    """Q = 0, one step: the source element gains -M (int s dt) phi(xi_s)/|det J|; the
    O-point Gauss-Legendre integral matches the Ricker antiderivative t e^(-pi^2 f0^2 t^2)."""
    s, mesh = _cube_solver(3, 3)
    dt = s.time_step_gts(0.5)
    xs = np.array([0.52, 0.41, 0.33])
    m6 = np.array([1.0, -0.5, 0.25, 0.3, -0.2, 0.1])
    f0, t0 = 2000.0, 2.5e-4
    s.add_point_source(xs, m6, f0, t0, m0=1e9)
    s.run_gts(dt, 1)
    k = mesh.locate(xs)
    phi = s.basis.phi(mesh.xi_of(k, xs)[None, :])[0]

    def anti(t):
        tau = t - t0
        return tau * np.exp(-(np.pi * f0 * tau) ** 2)

    integ = anti(dt) - anti(0.0)
    want = -(m6 * 1e9 * integ)[:, None] * (phi / mesh.detJ[k])[None, :]
    assert np.abs(s.Q[k, :6] - want).max() <= 1e-6 * np.abs(want).max()
    others = np.delete(np.arange(mesh.K), k)
    assert np.all(s.Q[others] == 0)
    assert abs(ricker(t0, f0, t0) - 1.0) < 1e-15


@pytest.mark.parametrize("order", [3, 4, 5])
def test_elastic_time_derivatives_lose_one_degree_each(order):
    """Cauchy-Kowalevski (Sec. III-A): every time derivative of the elastic state is one
    spatial derivative, so d^d Q has degree <= O-1-d and its modes beyond the first
    nbasis(O-d) vanish (the truncation the elastic time kernel uses). The anelastic coupling
    E theta carries the memory variables' full degree into every derivative."""
    a, mesh = _cube_solver(3, order)
    b, _ = _cube_solver(3, order, m=3, qs=40.0)
    rng = np.random.default_rng(order)
    B = order * (order + 1) * (order + 2) // 6
    a.Q = rng.standard_normal((mesh.K, 9, B))
    b.Q = rng.standard_normal((mesh.K, 27, B))
    idx = np.arange(mesh.K)
    Da, Db = a.derivatives(idx), b.derivatives(idx)
    for d in range(1, order):
        keep = (order - d) * (order - d + 1) * (order - d + 2) // 6
        scale = np.abs(Da[d]).max()
        assert scale > 0
        assert np.abs(Da[d][:, :, keep:]).max() <= 1e-12 * scale, d
        # anelastic: far above rounding (the coupling is weaker than the stiffness terms)
        assert np.abs(Db[d][:, :9, keep:]).max() > 1e-8 * np.abs(Db[d][:, :9]).max(), d
