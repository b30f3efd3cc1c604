"""Discrete adjoint on the GPU (global time stepping, elastic): misfit, samples, material
gradient and dJ/dQ0 against the FP64 oracle's adjoint; invariance to the checkpoint
spacing; central differences of the GPU's own misfit; the torch.autograd.Function."""
import numpy as np
import pytest

from oracle.adjoint import misfit_gradient as oracle_misfit_gradient
from oracle.mesh import Mesh
from oracle.scheme import Solver as Oracle
from paper_2202_10313_gb300 import binding, build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _case(order, seed=6):
    m = synth.permute_vertex_order(synth.graded_box(3, 3, 2, 200.0, 100.0, seed=seed), seed=5)
    mat = synth.random_layers(m, n_layers=2, seed=3)
    K = m["tet"].shape[0]
    nb = order * (order + 1) * (order + 2) // 6
    q0 = synth.random_dofs(K, 9, nb, seed=seed)
    rec = [np.array([150.0, 200.0, -40.0]), np.array([420.0, 330.0, -90.0]), np.array([300.0, 480.0, -20.0])]
    src = (np.array([310.0, 290.0, -120.0]), np.array([0.2, -0.4, 0.2, 1.0, 0.1, -0.3]), 10.0, 0.02, 1e12)
    return m, mat, q0, rec, src


def _rlm(mat):
    rho = mat["rho"].astype(float)
    mu = rho * mat["vs"] ** 2
    lam = rho * mat["vp"] ** 2 - 2 * mu
    return rho, lam, mu


def _oracle(order, m, rho, lam, mu, q0, rec, src, data, dt, n):
    om = Mesh(m["xyz"], m["tet"], m["face_bc"])
    o = Oracle(order, 0, om, rho, np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho))
    o.add_point_source(*src)
    o.Q = q0.copy()
    re = [om.locate(x) for x in rec]
    rp = [o.basis.phi(om.xi_of(k, x)[None, :])[0] for k, x in zip(re, rec)]
    return oracle_misfit_gradient(o, dt, n, re, rp, data), o


def _gpu(order, m, rho, lam, mu, q0, rec, src, dt, engine="sparse"):
    s = binding.Solver(order, 0, device=0)
    s.set_contraction(engine)
    s.set_mesh(m["xyz"], m["tet"], m["face_bc"])
    s.set_material(rho, np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho))
    s.add_point_source(*src)
    for x in rec:
        s.add_receiver(x, dt)
    s.setup_clusters(1, 0.5)
    s.set_finest_dt(dt)
    s.set_dofs(q0)
    return s


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _central_difference(make, params, p, k, misfit, J, g, noise):
    """Central difference of the GPU misfit w.r.t. parameter p of element k, with the floor
    it can resolve. The relative step is h = min(0.1, 5e-3 J / |g p|), so that J moves by about
    1 % (J is a sum of squares of FP32 samples, smooth in the parameter, but strongly
    non-linear for the few elements next to the source). Each evaluation of J carries FP32
    rounding of about `noise` J; the quotient turns that into noise J / h. Per element and
    parameter the adjoint must agree within 2e-2 |g| + noise J / h."""
    pk = params[p][k]
    h = min(0.1, 5e-3 * J / max(abs(g * pk), 1e-300)) * pk
    vals = []
    for sgn in (1, -1):
        pp = [x.copy() for x in params]
        pp[p][k] += sgn * h
        t = make(pp)
        vals.append(misfit(t))
        t.close()
    fd = (vals[0] - vals[1]) / (2 * h)
    return fd, abs(fd - g) <= 2e-2 * abs(g) + noise * J / h, noise * J / h


@pytest.mark.parametrize("engine", ["sparse", "fp32"])
@pytest.mark.parametrize("order", [3, 4])
def test_gpu_adjoint_matches_oracle_adjoint(order, engine):
    """Both reverse predict kernels: generated sparse products (engine 'sparse', the default
    for one simulation) and dense degree blocks ('fp32')."""
    m, mat, q0, rec, src = _case(order)
    rho, lam, mu = _rlm(mat)
    n = 8
    om = Mesh(m["xyz"], m["tet"], m["face_bc"])
    dt = Oracle(order, 0, om, rho, mat["vp"], mat["vs"]).time_step_gts(0.5)
    # observed data: the oracle in a model with mu 2 % higher
    (_, _, _, data), _ = _oracle(order, m, rho, lam, mu * 1.02, q0, rec, src, np.zeros((n + 1, 3, 3)), dt, n)
    (J0, g0, dq0_o, syn0), _ = _oracle(order, m, rho, lam, mu, q0, rec, src, data, dt, n)
    s = _gpu(order, m, rho, lam, mu, q0, rec, src, dt, engine)
    J, g, syn, dq0 = s.misfit_gradient(n, data, every=3, want_dq0=True)
    assert _rel(syn, syn0) <= 1e-5
    assert abs(J / J0 - 1) <= 1e-3
    for p in range(3):
        assert _rel(g[:, p], g0[:, p]) <= 2e-3, (p, _rel(g[:, p], g0[:, p]))
    assert _rel(dq0, dq0_o) <= 2e-3
    # the state ends at t_N
    assert abs(s.info()["time"] - n * dt) <= 1e-12 * n * dt


def test_checkpoint_spacing_does_not_change_the_result():
    order, n = 4, 9
    m, mat, q0, rec, src = _case(order, seed=8)
    rho, lam, mu = _rlm(mat)
    data = np.zeros((n + 1, 3, 3))
    out = []
    for every in (1, 4, n):
        s = _gpu(order, m, rho, lam, mu, q0, rec, src, 2e-4)
        out.append(s.misfit_gradient(n, data, every=every))
        s.close()
    for J, g, syn in out[1:]:
        assert J == out[0][0] and np.array_equal(g, out[0][1]) and np.array_equal(syn, out[0][2])


def test_gpu_gradient_against_central_differences_of_the_gpu_misfit():
    """dJ/d(rho, lambda, mu) of the GPU adjoint against central differences of the GPU misfit on
    20 elements (order 4, 108 tets, 8 steps)."""
    order, n = 4, 8
    m, mat, q0, rec, src = _case(order, seed=10)
    rho, lam, mu = _rlm(mat)
    dt = 2e-4
    s = _gpu(order, m, rho, lam, mu, q0, rec, src, dt)
    _, _, syn = s.misfit_gradient(n, np.zeros((n + 1, 3, 3)), every=4)
    data = syn * 1.05
    s = _gpu(order, m, rho, lam, mu, q0, rec, src, dt)
    J, g, _ = s.misfit_gradient(n, data, every=4)
    params = [rho, lam, mu]
    rng = np.random.default_rng(2)
    # 20 elements: the 10 largest |dJ/dmu| and 10 others drawn at random; rho, lambda, mu on each
    top = np.argsort(-np.abs(g[:, 2]))[:10].tolist()
    rest = [k for k in rng.permutation(len(rho)).tolist() if k not in top][:10]
    bad, worst = [], 0.0
    for p in range(3):
        for k in top + rest:
            fd, ok, floor = _central_difference(lambda pp: _gpu(order, m, *pp, q0, rec, src, dt), params, p, k,
                                                lambda t: t.misfit_gradient(n, data, every=n)[0], J, g[k, p], 1e-5)
            if not ok:
                bad.append((p, k, fd, g[k, p]))
            if abs(g[k, p]) > 10 * floor:
                worst = max(worst, abs(fd - g[k, p]) / abs(g[k, p]))
    for r in bad:
        print("FD MISMATCH parameter %d element %d: central difference %.6e adjoint %.6e" % r)
    assert not bad, bad
    print("FD per-element worst relative error (gradients above the rounding floor): %.2e" % worst)


def test_autograd_function():
    torch = pytest.importorskip("torch")
    from paper_2202_10313_gb300.adjoint import MisfitProblem, SeismogramMisfit
    order, n = 3, 6
    m, mat, q0, rec, src = _case(order, seed=12)
    rho, lam, mu = _rlm(mat)
    dt = 2e-4
    data = np.zeros((n + 1, 3, 3))
    prob = MisfitProblem(order, m, q0, rec, data, n, dt, sources=[src], every=2)
    tr, tl, tm = (torch.tensor(x, dtype=torch.float64, requires_grad=True) for x in (rho, lam, mu))
    J = SeismogramMisfit.apply(tr, tl, tm, prob)
    J.backward()
    s = _gpu(order, m, rho, lam, mu, q0, rec, src, dt)
    J2, g, _ = s.misfit_gradient(n, data, every=2)
    assert float(J.detach()) == J2
    assert np.array_equal(tr.grad.numpy(), g[:, 0]) and np.array_equal(tm.grad.numpy(), g[:, 2])


def test_autograd_function_lts():
    """SeismogramMisfit over the clustered LTS loop (three forced clusters): J and the
    gradients handed to the tensors equal lts_misfit_gradient's bitwise."""
    torch = pytest.importorskip("torch")
    from paper_2202_10313_gb300.adjoint import MisfitProblem, SeismogramMisfit
    order, n_macro = 4, 3
    m, mat, q0, rec, src = _case(order, seed=22)
    rho, lam, mu = _rlm(mat)
    cl = _forced_clusters(m)
    assert len(np.unique(cl)) == 3
    dt = 1.5e-4
    s = _gpu_lts(order, m, rho, lam, mu * 1.02, q0, rec, src, cl, dt)
    _, data = s.misfit(4 * n_macro, np.zeros((n_macro + 1, 3, 3)), every=2)
    s.close()
    prob = MisfitProblem(order, m, q0, rec, data, 4 * n_macro, dt, sources=[src], every=2, clusters=cl, n_clusters=3)
    tr, tl, tm = (torch.tensor(x, dtype=torch.float64, requires_grad=True) for x in (rho, lam, mu))
    J = SeismogramMisfit.apply(tr, tl, tm, prob)
    J.backward()
    s = _gpu_lts(order, m, rho, lam, mu, q0, rec, src, cl, dt)
    J2, g, _ = s.misfit_gradient(4 * n_macro, data, every=2)
    s.close()
    assert J2 > 0 and float(J.detach()) == J2
    for t, p in ((tr, 0), (tl, 1), (tm, 2)):
        assert np.array_equal(t.grad.numpy(), g[:, p])


def _forced_clusters(m):
    from oracle import lts as olts
    om = Mesh(m["xyz"], m["tet"], m["face_bc"])
    cx = om.centroid[:, 0]
    return olts.normalise(np.digitize(cx, np.quantile(cx, [0.3, 0.65])), om.nbr)


def _gpu_lts(order, m, rho, lam, mu, q0, rec, src, cl, dt, engine="sparse"):
    s = binding.Solver(order, 0, device=0)
    s.set_contraction(engine)
    s.set_mesh(m["xyz"], m["tet"], m["face_bc"])
    s.set_material(rho, np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho))
    s.add_point_source(*src)
    for x in rec:
        s.add_receiver(x, dt)
    s.force_clusters(cl, 3, 0.5, 1.0)
    s.set_finest_dt(dt)
    s.set_dofs(q0)
    return s


@pytest.mark.parametrize("engine", ["sparse", "fp32"])
@pytest.mark.parametrize("order", [3, 4, 5])
def test_gpu_lts_adjoint_matches_oracle_lts_adjoint(order, engine):
    """Three forced clusters (all buffer relations), samples at the macro-step boundaries;
    both reverse predict kernels."""
    from oracle.adjoint import misfit_gradient_lts
    m, mat, q0, rec, src = _case(order, seed=14)
    rho, lam, mu = _rlm(mat)
    cl = _forced_clusters(m)
    assert len(np.unique(cl)) == 3
    dt, n_macro = 1.5e-4, 3
    om = Mesh(m["xyz"], m["tet"], m["face_bc"])

    def oracle(mu_):
        o = Oracle(order, 0, om, rho, np.sqrt((lam + 2 * mu_) / rho), np.sqrt(mu_ / rho))
        o.add_point_source(*src)
        o.setup_clusters(3, 0.5, lam=1.0, clusters=cl)
        o.delta = dt
        o.Q = q0.copy()
        re = [om.locate(x) for x in rec]
        rp = [o.basis.phi(om.xi_of(k, x)[None, :])[0] for k, x in zip(re, rec)]
        return o, re, rp

    o, re, rp = oracle(mu * 1.02)
    _, _, _, data = misfit_gradient_lts(o, n_macro, re, rp, np.zeros((n_macro + 1, 3, 3)))
    o, re, rp = oracle(mu)
    J0, g0, dq0_o, syn0 = misfit_gradient_lts(o, n_macro, re, rp, data)
    s = _gpu_lts(order, m, rho, lam, mu, q0, rec, src, cl, dt, engine)
    J, g, syn, dq0 = s.misfit_gradient(4 * n_macro, data, every=2, want_dq0=True)
    assert _rel(syn, syn0) <= 1e-5
    assert abs(J / J0 - 1) <= 1e-3
    for p in range(3):
        assert _rel(g[:, p], g0[:, p]) <= 2e-3, (p, _rel(g[:, p], g0[:, p]))
    assert _rel(dq0, dq0_o) <= 2e-3
    assert abs(s.info()["time"] - 4 * n_macro * dt) <= 1e-12


def test_lts_checkpoint_spacing_does_not_change_the_result():
    order, n_macro = 4, 3
    m, mat, q0, rec, src = _case(order, seed=16)
    rho, lam, mu = _rlm(mat)
    cl = _forced_clusters(m)
    data = np.zeros((n_macro + 1, 3, 3))
    out = []
    for every in (1, 2, n_macro):
        s = _gpu_lts(order, m, rho, lam, mu, q0, rec, src, cl, 1.5e-4)
        out.append(s.misfit_gradient(4 * n_macro, data, every=every))
        s.close()
    for J, g, syn in out[1:]:
        assert J == out[0][0] and np.array_equal(g, out[0][1]) and np.array_equal(syn, out[0][2])


@pytest.mark.parametrize("F", [1, 4])
def test_lts_adjoint_memory_budget_does_not_change_the_result(F):
    """A segment replayed once with every phase input kept, and (a 1-byte budget) replayed
    macro step by macro step: the same reverse sweep, bitwise (one and fused simulations)."""
    order, n_macro = 4, 4
    m, mat, q0, rec, src = _case(order, seed=18)
    rho, lam, mu = _rlm(mat)
    cl = _forced_clusters(m)

    def make():
        if F == 1:
            return _gpu_lts(order, m, rho, lam, mu, q0, rec, src, cl, 1.5e-4)
        q0s, srcs = _fused_inputs(m, order, F, seed=60)
        return _fused_lts(order, m, rho, lam, mu, q0s, rec, srcs, cl, 1.5e-4, F)

    shape = (n_macro + 1, 3, 3) if F == 1 else (n_macro + 1, F, 3, 3)
    s = make()
    _, _, syn = s.misfit_gradient(4 * n_macro, np.zeros(shape), every=n_macro)
    s.close()
    data = syn * 1.03
    out = []
    for budget in (0, 1):
        s = make()
        s.set_adjoint_memory(budget)
        out.append(s.misfit_gradient(4 * n_macro, data, every=3, want_dq0=True))
        s.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))


def test_gpu_adjoint_periodic_cube_matches_oracle_adjoint():
    """Periodic faces (every face has a neighbour, some across the box) and a heterogeneous
    material: the GTS adjoint's misfit, gradients and dJ/dQ0 against the oracle's adjoint."""
    order, n = 3, 6
    m = synth.permute_vertex_order(synth.periodic_cube(3, 1000.0), seed=3)
    K = m["tet"].shape[0]
    rng = np.random.default_rng(4)
    rho = 2700.0 * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, K))
    vs = 3464.0 * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, K))
    vp = 6000.0 * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, K))
    mu = rho * vs ** 2
    lam = rho * vp ** 2 - 2 * mu
    nb = order * (order + 1) * (order + 2) // 6
    q0 = synth.random_dofs(K, 9, nb, seed=6)
    rec = [np.array([250.0, 400.0, 600.0]), np.array([700.0, 300.0, 200.0])]
    om = Mesh(m["xyz"], m["tet"], m["face_bc"], m["period"])

    def oracle(mu_):
        o = Oracle(order, 0, om, rho, np.sqrt((lam + 2 * mu_) / rho), np.sqrt(mu_ / rho))
        o.Q = q0.copy()
        return o

    dt = oracle(mu).time_step_gts(0.5)
    re = [om.locate(x) for x in rec]
    o = oracle(mu * 1.02)
    rp = [o.basis.phi(om.xi_of(k, x)[None, :])[0] for k, x in zip(re, rec)]
    _, _, _, data = oracle_misfit_gradient(o, dt, n, re, rp, np.zeros((n + 1, 2, 3)))
    J0, g0, dq0_o, syn0 = oracle_misfit_gradient(oracle(mu), dt, n, re, rp, data)
    s = binding.Solver(order, 0, device=0)
    s.set_mesh(m["xyz"], m["tet"], m["face_bc"], m["period"])
    s.set_material(rho, np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho))
    for x in rec:
        s.add_receiver(x, dt)
    s.setup_clusters(1, 0.5)
    s.set_finest_dt(dt)
    s.set_dofs(q0)
    J, g, syn, dq0 = s.misfit_gradient(n, data, every=2, want_dq0=True)
    assert _rel(syn, syn0) <= 1e-5
    assert abs(J / J0 - 1) <= 1e-3
    for p in range(3):
        assert _rel(g[:, p], g0[:, p]) <= 2e-3, (p, _rel(g[:, p], g0[:, p]))
    assert _rel(dq0, dq0_o) <= 2e-3


def _fused_inputs(m, order, F, seed):
    K = m["tet"].shape[0]
    nb = order * (order + 1) * (order + 2) // 6
    rng = np.random.default_rng(seed)
    q0s = np.stack([synth.random_dofs(K, 9, nb, seed=seed + f) for f in range(F)])
    srcs = [(np.array([200.0, 200.0, -60.0]) + rng.uniform(0.0, 250.0, 3) * np.array([1.0, 1.0, -0.3]),
             rng.normal(size=6), 10.0, 0.02, 1e12) for _ in range(F)]
    return q0s, srcs


def _fused_lts(order, m, rho, lam, mu, q0s, rec, srcs, cl, dt, F, engine="sparse"):
    s = binding.Solver(order, 0, device=0, n_fused=F)
    s.set_contraction(engine)
    s.set_mesh(m["xyz"], m["tet"], m["face_bc"])
    s.set_material(rho, np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho))
    for f, src in enumerate(srcs):
        s.add_point_source(*src, fused_idx=f)
    for x in rec:
        s.add_receiver(x, dt)
    if cl is None:
        s.setup_clusters(1, 0.5)
    else:
        s.force_clusters(cl, 3, 0.5, 1.0)
    s.set_finest_dt(dt)
    s.set_dofs(q0s)
    return s


@pytest.mark.parametrize("engine", ["sparse", "fp32"])
@pytest.mark.parametrize("F,clustered", [(4, True), (8, True), (4, False)])
def test_fused_adjoint_equals_the_sum_of_single_simulation_adjoints(F, clustered, engine):
    """F simulations (own sources, initial states and data; shared material) in one adjoint
    sweep: J and the material gradient are the sums of the single-simulation values, the
    samples and dJ/dQ0 those of each simulation (three forced clusters, or one cluster); the
    fused run with either reverse predict kernel, the single runs with the sparse one."""
    order = 4
    m, mat, _, rec, _ = _case(order, seed=20)
    rho, lam, mu = _rlm(mat)
    cl = _forced_clusters(m) if clustered else None
    dt = 1.5e-4
    n = 8 if clustered else 6
    q0s, srcs = _fused_inputs(m, order, F, seed=40)
    s = _fused_lts(order, m, rho, lam, mu, q0s, rec, srcs, cl, dt, F, engine)
    rows = n // 4 + 1 if clustered else n + 1
    _, syn = s.misfit(n, np.zeros((rows, F, 3, 3)), every=1)
    s.close()
    data = syn * 1.04 + 1e-9
    s = _fused_lts(order, m, rho, lam, mu, q0s, rec, srcs, cl, dt, F, engine)
    J, g, syn_f, dq0 = s.misfit_gradient(n, data, every=1, want_dq0=True)
    gsrc = s.source_gradient()   # source f drives simulation f only
    s.close()
    J1, g1 = 0.0, np.zeros_like(g)
    for f in range(F):
        if clustered:
            t = _gpu_lts(order, m, rho, lam, mu, q0s[f], rec, srcs[f], cl, dt)
        else:
            t = _gpu(order, m, rho, lam, mu, q0s[f], rec, srcs[f], dt)
        Jf, gf, synf, dqf = t.misfit_gradient(n, data[:, f], every=1, want_dq0=True)
        # a source beyond the adjoint's reach in n steps has a zero gradient in both runs
        assert np.allclose(gsrc[f], t.source_gradient()[0], rtol=1e-4, atol=1e-6 * np.abs(gsrc).max()), f
        t.close()
        J1 += Jf
        g1 += gf
        assert _rel(syn_f[:, f], synf) <= 1e-5, f
        assert _rel(dq0[f], dqf) <= 1e-4, (f, _rel(dq0[f], dqf))
    assert abs(J / J1 - 1) <= 1e-5
    for p in range(3):
        assert _rel(g[:, p], g1[:, p]) <= 1e-4, (p, _rel(g[:, p], g1[:, p]))


def test_autograd_function_fused():
    torch = pytest.importorskip("torch")
    from paper_2202_10313_gb300.adjoint import MisfitProblem, SeismogramMisfit
    order, n, F = 3, 6, 4
    m, mat, _, rec, _ = _case(order, seed=22)
    rho, lam, mu = _rlm(mat)
    q0s, srcs = _fused_inputs(m, order, F, seed=50)
    dt = 2e-4
    data = np.full((n + 1, F, 3, 3), 1e-9)
    prob = MisfitProblem(order, m, q0s, rec, data, n, dt, sources=srcs, every=2, n_fused=F)
    tr, tl, tm = (torch.tensor(x, dtype=torch.float64, requires_grad=True) for x in (rho, lam, mu))
    J = SeismogramMisfit.apply(tr, tl, tm, prob)
    J.backward()
    s = _fused_lts(order, m, rho, lam, mu, q0s, rec, srcs, None, dt, F)
    J2, g, _ = s.misfit_gradient(n, data, every=2)
    assert float(J.detach()) == J2
    assert np.array_equal(tl.grad.numpy(), g[:, 1]) and np.array_equal(tm.grad.numpy(), g[:, 2])


@pytest.mark.parametrize("clustered", [True, False])
def test_moment_tensor_gradient_against_central_differences(clustered):
    """dJ/dm6 of two point sources (LTS with three forced clusters, and one cluster): J is
    quadratic in m6, so central differences of the GPU misfit are exact up to FP32 rounding."""
    order, n = 4, 8
    m, mat, q0, rec, src = _case(order, seed=24)
    rho, lam, mu = _rlm(mat)
    cl = _forced_clusters(m)
    src2 = (np.array([420.0, 260.0, -90.0]), np.array([-0.3, 0.5, 0.1, -0.2, 0.7, 0.4]), 12.0, 0.015, 8e11)
    dt = 1.5e-4

    def make(m6a, m6b):
        s = binding.Solver(order, 0, device=0)
        s.set_mesh(m["xyz"], m["tet"], m["face_bc"])
        s.set_material(rho, np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho))
        s.add_point_source(src[0], m6a, *src[2:])
        s.add_point_source(src2[0], m6b, *src2[2:])
        for x in rec:
            s.add_receiver(x, dt)
        if clustered:
            s.force_clusters(cl, 3, 0.5, 1.0)
        else:
            s.setup_clusters(1, 0.5)
        s.set_finest_dt(dt)
        s.set_dofs(np.zeros_like(q0))   # the samples come from the sources alone
        return s

    rows = n // 4 + 1 if clustered else n + 1
    s = make(src[1], src2[1])
    _, syn = s.misfit(n, np.zeros((rows, 3, 3)), every=1)
    s.close()
    data = syn * 0.7 + 1e-10
    s = make(src[1], src2[1])
    s.misfit_gradient(n, data, every=1)
    g = s.source_gradient()
    s.close()
    assert g.shape == (2, 6) and np.abs(g).max() > 0
    for i, (m6, other) in enumerate([(src[1], src2[1]), (src2[1], src[1])]):
        for r in range(6):
            h = 0.5
            vals = []
            for sgn in (1, -1):
                mm = m6.copy()
                mm[r] += sgn * h
                t = make(mm, other) if i == 0 else make(other, mm)
                vals.append(t.misfit(n, data, every=1)[0])
                t.close()
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - g[i, r]) <= 2e-3 * np.abs(g).max(), (i, r, fd, g[i, r])
