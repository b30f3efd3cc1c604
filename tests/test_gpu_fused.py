"""Fused simulations (Sec. IV-A): F simulations share mesh, material and clusters and
differ in sources and initial DOFs. Simulation f of a fused GPU run must match the
oracle run of simulation f alone (relative L2 of the DOFs <= 1e-4 per quantity group,
seismogram misfit <= 1e-8), and the single-simulation GPU run with the same inputs."""
import numpy as np
import pytest

from paper_2202_10313_gb300 import binding, build, synth
from gpu_common import make_pair, rel_l2_groups

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _case(seed=31):
    m = synth.permute_vertex_order(synth.graded_box(4, 4, 3, 250.0, 125.0, seed=seed), seed=4)
    mat = synth.random_layers(m, n_layers=3, seed=9)
    return m, mat


def _fused_solver(order, n_mech, m, mat, F):
    g = binding.Solver(order, n_mech, device=0, n_fused=F)
    g.set_mesh(m["xyz"], m["tet"], m["face_bc"], m.get("period"))
    g.set_material(mat["rho"], mat["vp"], mat["vs"], mat.get("qp"), mat.get("qs"), 0.1, 5.0)
    return g


def _inputs(m, F, nq, nb, seed):
    lo, hi = m["xyz"].min(axis=0), m["xyz"].max(axis=0)
    pos, m6, f0 = synth.random_sources(F, lo + 0.15 * (hi - lo), hi - 0.15 * (hi - lo), f0_range=(4.0, 8.0),
                                       seed=seed)
    K = m["tet"].shape[0]
    # simulation f starts from its own random DOFs; odd simulations start at rest
    d0 = np.stack([synth.random_dofs(K, nq, nb, seed=seed + f, stress_scale=1e3) * (f % 2 == 0)
                   for f in range(F)])
    return pos, m6, f0, d0


@pytest.mark.parametrize("order,n_mech,F", [(4, 3, 8), (5, 3, 8), (5, 0, 4), (3, 3, 12)])
def test_fused_lts_matches_oracle_per_simulation(order, n_mech, F):
    """3 LTS clusters, one moment-tensor source per simulation, two shared receivers,
    two macro steps; simulations in several CTA groups (F > 4) and a single group."""
    m, mat = _case()
    K = m["tet"].shape[0]
    nq, nb = 9 + 6 * n_mech, order * (order + 1) * (order + 2) // 6
    pos, m6, f0, d0 = _inputs(m, F, nq, nb, seed=70 + order)
    g = _fused_solver(order, n_mech, m, mat, F)
    for f in range(F):
        g.add_point_source(pos[f], m6[f], f0[f], 0.1, 1e12, fused_idx=f)
    recs = [np.array([330.0, 410.0, -60.0]), np.array([700.0, 520.0, -150.0])]
    g.setup_clusters(3, 0.5)
    dt_rec = g.info()["finest_dt"] * 1.37
    rid = [g.add_receiver(r, dt_rec) for r in recs]
    cl, lam, _ = g.setup_clusters(3, 0.5)
    assert len(np.unique(cl)) == 3
    g.set_dofs(d0)
    n = 2 * 4
    g.advance_steps(n)
    got = g.get_dofs()
    assert got.shape == (F, K, nq, nb)
    for f in range(F):
        _, ora, _ = make_pair(order, n_mech, m, mat)
        ora.add_point_source(pos[f], m6[f], f0[f], 0.1, 1e12)
        ro = [ora.add_receiver(r, dt_rec) for r in recs]
        ora.setup_clusters(3, 0.5)
        assert np.array_equal(cl, ora.clusters)
        ora.Q = d0[f].copy()
        ora.run_lts(n)
        err = rel_l2_groups(got[f], ora.Q, nq)
        for k, v in err.items():
            assert v <= TOL, (f, err)
        for a, b in zip(rid, ro):
            tg, vg = g.seismogram(a, fused_idx=f)
            to, vo = ora.seismogram(b)
            assert np.array_equal(tg, to)
            for q in range(9):
                den = np.sum(vo[:, q] ** 2)
                if den > 0:
                    assert np.sum((vg[:, q] - vo[:, q]) ** 2) / den <= 1e-8, (f, q)


@pytest.mark.parametrize("engine", ["sparse", "fp32"])
def test_fused_equals_single_simulation_runs_and_energy_sums(engine):
    """The fused run against F single-simulation GPU runs with the same inputs and engine:
    same arithmetic per simulation, so agreement to FP32 rounding (the sparse engine's
    kernels take (element, simulation) slots and are bitwise equal); energies add up."""
    m, mat = _case(seed=33)
    F, order, n_mech = 8, 5, 3
    K = m["tet"].shape[0]
    pos, m6, f0, d0 = _inputs(m, F, 27, 35, seed=90)
    g = _fused_solver(order, n_mech, m, mat, F)
    g.set_contraction(engine)
    for f in range(F):
        g.add_point_source(pos[f], m6[f], f0[f], 0.1, 1e12, fused_idx=f)
    g.setup_clusters(2, 0.5)
    g.set_dofs(d0)
    g.advance_steps(6)
    got = g.get_dofs()
    e_fused = g.energy()
    e_sum = 0.0
    for f in range(F):
        s, _, _ = make_pair(order, n_mech, m, mat)
        s.set_contraction(engine)
        s.add_point_source(pos[f], m6[f], f0[f], 0.1, 1e12)
        s.setup_clusters(2, 0.5)
        s.set_dofs(d0[f])
        s.advance_steps(6)
        one = s.get_dofs()
        e_sum += s.energy()
        den = np.sqrt(np.sum(one ** 2))
        assert np.sqrt(np.sum((got[f] - one) ** 2)) / den <= 1e-6, f
        if engine == "sparse":
            assert np.array_equal(got[f], one), f
        s.close()
    assert abs(e_fused / e_sum - 1.0) < 1e-9


def test_fused_subset_access_and_projection_broadcast():
    """Subset DOF access carries the simulation axis; projection fills every simulation."""
    m, mat = _case(seed=35)
    F = 8
    g = _fused_solver(4, 0, m, mat, F)
    g.setup_clusters(1, 0.5)
    g.project_initial(lambda x: np.tile(np.sin(x[:, :1] / 300.0), (1, 9)))
    d = g.get_dofs()
    for f in range(1, F):
        assert np.array_equal(d[f], d[0])
    elems = np.array([5, 0, 77])
    sub = np.random.default_rng(1).normal(size=(F, 3, 9, 20))
    g.set_dofs_subset(elems, sub)
    back = g.get_dofs_subset(elems)
    assert np.allclose(back, sub.astype(np.float32), rtol=0, atol=0)
    full = g.get_dofs()
    assert np.array_equal(full[:, elems], back)


def test_maximum_fused_count():
    """LTS_MAX_FUSED (64) simulations in one run (16 CTA groups per element): simulations at
    both ends and in the middle match their single-simulation GPU runs."""
    m, mat = _case(seed=37)
    F, order, n_mech = 64, 3, 3
    pos, m6, f0, d0 = _inputs(m, F, 27, 10, seed=91)
    g = _fused_solver(order, n_mech, m, mat, F)
    for f in range(F):
        g.add_point_source(pos[f], m6[f], f0[f], 0.1, 1e12, fused_idx=f)
    g.setup_clusters(2, 0.5)
    g.set_dofs(d0)
    g.advance_steps(4)
    got = g.get_dofs()
    assert np.all(np.isfinite(got))
    for f in (0, 1, 31, 62, 63):
        s, _, _ = make_pair(order, n_mech, m, mat)
        s.add_point_source(pos[f], m6[f], f0[f], 0.1, 1e12)
        s.setup_clusters(2, 0.5)
        s.set_dofs(d0[f])
        s.advance_steps(4)
        one = s.get_dofs()
        s.close()
        assert np.sqrt(np.sum((got[f] - one) ** 2)) / np.sqrt(np.sum(one ** 2)) <= 1e-6, f
