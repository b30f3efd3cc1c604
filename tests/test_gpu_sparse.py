"""The predict kernel with generated sparse products (contraction engine 'sparse': the
nonzero entries of K_c and F~_i as immediate operands, Sec. IV-A "all sparsity") against the
FP64 oracle on the same seeded inputs, per quantity group and elementwise, and against the
dense-block FP32 kernel."""
import numpy as np
import pytest

from paper_2202_10313_gb300 import build, synth
from gpu_common import check_parity, initial_field, make_pair, rel_l2_groups, report_parity

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


@pytest.mark.parametrize("order,n_mech", [(3, 0), (3, 3), (4, 0), (4, 3), (5, 0), (5, 3)])
def test_graded_box_lts_sparse_engine(order, n_mech):
    """Jittered graded box, random layers (free surface + absorbing), 3 clusters from the
    lambda search, two macro steps: the sparse engine against the oracle, and against the
    dense-block FP32 engine started from the same DOFs."""
    m = synth.permute_vertex_order(synth.graded_box(5, 5, 3, 250.0, 125.0, seed=12), seed=2)
    mat = synth.random_layers(m, n_layers=3, seed=5)
    gpu, ora, _ = make_pair(order, n_mech, m, mat)
    ref, _, _ = make_pair(order, n_mech, m, mat)
    gpu.set_contraction("sparse")
    cl, lam, _ = gpu.setup_clusters(3, 0.5)
    ref.setup_clusters(3, 0.5)
    ora.setup_clusters(3, 0.5)
    assert np.array_equal(cl, ora.clusters) and len(np.unique(cl)) == 3
    ora.project(initial_field(ora.nq, [600.0, 700.0, -300.0], 400.0))
    gpu.set_dofs(ora.Q)
    ref.set_dofs(ora.Q)
    n = 2 * 4
    gpu.advance_steps(n)
    ref.advance_steps(n)
    ora.run_lts(n)
    err = check_parity(gpu.get_dofs(), ora.Q, ora.nq, TOL)
    report_parity("sparse engine: graded box, %d tets, O%d, %d mechanisms, 3 clusters, 2 macro steps"
                  % (m["tet"].shape[0], order, n_mech), err)
    agree = rel_l2_groups(gpu.get_dofs(), ref.get_dofs(), ora.nq)
    assert agree["all"] <= 1e-5, agree


def test_forced_clusters_with_all_relations_sparse_engine():
    """Forced 3-cluster split of a periodic cube (B1, B2, B1 - B2 and accumulated B3 reads;
    periodic faces) with 3 mechanisms, order 4 and order 5."""
    from oracle.lts import normalise
    m = synth.permute_vertex_order(synth.periodic_cube(5), seed=3)
    K = m["tet"].shape[0]
    mat = dict(synth.homogeneous(K), qp=np.full(K, 60.0), qs=np.full(K, 30.0))
    for order in (4, 5):
        gpu, ora, om = make_pair(order, 3, m, mat, 1000.0, 50000.0)
        gpu.set_contraction("sparse")
        c = normalise(np.digitize(om.centroid[:, 0], [1 / 3, 2 / 3]), om.nbr).astype(np.int32)
        gpu.force_clusters(c, 3, 0.125)
        ora.setup_clusters(3, 0.125, lam=1.0, clusters=c)
        pw = synth.p_plane_wave(2700.0, 6000.0, 3464.0, 2 * np.pi * np.array([1.0, 1.0, 0.0]))
        ora.project(lambda x: np.concatenate([pw(x, 0.0), np.zeros((len(x), 18))], axis=1))
        gpu.set_dofs(ora.Q)
        gpu.advance_steps(8)
        ora.run_lts(8)
        report_parity("sparse engine: forced clusters, periodic cube, O%d, 3 mechanisms" % order,
                      check_parity(gpu.get_dofs(), ora.Q, ora.nq, TOL))


def test_source_receivers_and_single_element_sparse_engine():
    """Point source and receivers with 3 clusters (DOFs and traces), and a one-element mesh
    (a batch of one, every face absorbing)."""
    m = synth.graded_box(5, 5, 3, 250.0, 125.0, seed=21)
    mat = synth.random_layers(m, n_layers=3, seed=8)
    gpu, ora, _ = make_pair(5, 3, m, mat)
    gpu.set_contraction("sparse")
    xs = np.array([610.0, 640.0, -260.0])
    m6 = np.array([0.2, -0.4, 0.2, 1.0, 0.1, -0.3])
    gpu.add_point_source(xs, m6, 8.0, 0.06, 1e12)
    ora.add_point_source(xs, m6, 8.0, 0.06, 1e12)
    recs = [np.array([300.0 + 170.0 * i, 400.0 + 90.0 * i, -40.0 - 30.0 * i]) for i in range(3)]
    gpu.setup_clusters(3, 0.5)
    dt_rec = gpu.info()["finest_dt"] * 1.37
    rid_g = [gpu.add_receiver(r, dt_rec) for r in recs]
    rid_o = [ora.add_receiver(r, dt_rec) for r in recs]
    cl, _, _ = gpu.setup_clusters(3, 0.5)
    ora.setup_clusters(3, 0.5)
    assert np.array_equal(cl, ora.clusters)
    gpu.advance_steps(16)
    ora.run_lts(16)
    check_parity(gpu.get_dofs(), ora.Q, ora.nq, TOL)
    for a, b in zip(rid_g, rid_o):
        tg, vg = gpu.seismogram(a)
        to, vo = ora.seismogram(b)
        assert np.array_equal(tg, to)
        for q in range(9):
            den = np.sum(vo[:, q] ** 2)
            if den > 0:
                assert np.sum((vg[:, q] - vo[:, q]) ** 2) / den <= 1e-8
    xyz = np.array([[0.0, 0, 0], [100.0, 0, 0], [0, 120.0, 0], [0, 0, 90.0]])
    one = dict(xyz=xyz, tet=np.array([[0, 1, 2, 3]]), face_bc=np.ones((1, 4), dtype=np.int32), period=None)
    mat1 = dict(rho=np.array([2500.0]), vp=np.array([3000.0]), vs=np.array([1700.0]),
                qp=np.array([60.0]), qs=np.array([30.0]))
    gpu, ora, _ = make_pair(5, 3, one, mat1)
    gpu.set_contraction("sparse")
    gpu.setup_clusters(1, 0.5)
    d = synth.random_dofs(1, 27, 35, seed=2)
    gpu.set_dofs(d)
    ora.Q = d.copy()
    gpu.advance_steps(6)
    ora.run_gts(ora.time_step_gts(0.5), 6)
    check_parity(gpu.get_dofs(), ora.Q, ora.nq, TOL)


def test_sparse_engine_repeatable_bitwise():
    m = synth.graded_box(4, 4, 3, 200.0, 100.0, seed=6)
    mat = synth.random_layers(m, n_layers=2, seed=2)
    outs = []
    for _ in range(2):
        gpu, ora, _ = make_pair(5, 3, m, mat)
        gpu.set_contraction("sparse")
        gpu.setup_clusters(2, 0.5)
        ora.project(initial_field(27, [400.0, 400.0, -200.0], 300.0))
        gpu.set_dofs(ora.Q)
        gpu.advance_steps(4)
        outs.append(gpu.get_dofs())
    assert np.array_equal(outs[0], outs[1])


def test_fused_sparse_engine_matches_oracle_per_simulation():
    """Four and eight fused simulations on the sparse engine ((element, simulation) slots),
    each with its own source and initial state, against its own oracle run (3 clusters)."""
    m = synth.graded_box(4, 4, 3, 250.0, 125.0, seed=33)
    mat = synth.random_layers(m, n_layers=3, seed=6)
    K = m["tet"].shape[0]
    from paper_2202_10313_gb300 import binding
    for order, F in ((5, 4), (4, 8)):
        nb = order * (order + 1) * (order + 2) // 6
        d0 = np.stack([synth.random_dofs(K, 27, nb, seed=70 + f) for f in range(F)])
        lo, hi = m["xyz"].min(axis=0), m["xyz"].max(axis=0)
        pos, m6, f0 = synth.random_sources(F, lo + 0.2 * (hi - lo), hi - 0.2 * (hi - lo), f0_range=(4.0, 8.0), seed=5)
        g = binding.Solver(order, 3, device=0, n_fused=F)
        g.set_mesh(m["xyz"], m["tet"], m["face_bc"])
        g.set_material(mat["rho"], mat["vp"], mat["vs"], mat["qp"], mat["qs"], 0.1, 5.0)
        g.set_contraction("sparse")
        for f in range(F):
            g.add_point_source(pos[f], m6[f], f0[f], 0.1, 1e12, fused_idx=f)
        cl, _, _ = g.setup_clusters(3, 0.5)
        g.set_dofs(d0)
        g.advance_steps(8)
        got = g.get_dofs()
        for f in (0, F - 1):
            _, ora, _ = make_pair(order, 3, m, mat)
            ora.add_point_source(pos[f], m6[f], f0[f], 0.1, 1e12)
            ora.setup_clusters(3, 0.5)
            assert np.array_equal(cl, ora.clusters)
            ora.Q = d0[f].copy()
            ora.run_lts(8)
            report_parity("sparse engine, fused %d, O%d, simulation %d" % (F, order, f),
                          check_parity(got[f], ora.Q, 27, TOL))
        g.close()


def test_neighbour_tile_variants_bitwise_equal():
    """The sparse engine's neighbour kernel with 8 and with 4 elements per CTA: the same
    arithmetic per element, so bitwise equal results (order 5 and 4, 3 mechanisms)."""
    m = synth.permute_vertex_order(synth.graded_box(5, 5, 3, 250.0, 125.0, seed=12), seed=2)
    mat = synth.random_layers(m, n_layers=3, seed=5)
    for order in (4, 5):
        outs = []
        for tile in (0, 1):
            gpu, ora, _ = make_pair(order, 3, m, mat)
            gpu.set_contraction("sparse")
            gpu.set_tile(tile)
            gpu.setup_clusters(3, 0.5)
            ora.project(initial_field(ora.nq, [600.0, 700.0, -300.0], 400.0))
            gpu.set_dofs(ora.Q)
            gpu.advance_steps(8)
            outs.append(gpu.get_dofs())
        assert np.array_equal(outs[0], outs[1])


def test_sparse_engine_empty_clusters_and_periodic_gts():
    """Degenerate schedules on the sparse engine: a homogeneous mesh with 4 clusters requested
    (the lambda search leaves some empty, so some phases have no element), and global time
    stepping on a periodic cube (every face has a neighbour, some across the box)."""
    m = synth.graded_box(3, 3, 2, 200.0, 200.0, grade=1.0, jitter=0.0, seed=1)
    K = m["tet"].shape[0]
    gpu, ora, _ = make_pair(4, 3, m, dict(synth.homogeneous(K), qp=np.full(K, 80.0), qs=np.full(K, 40.0)))
    gpu.set_contraction("sparse")
    cl, _, _ = gpu.setup_clusters(4, 0.5)
    ora.setup_clusters(4, 0.5)
    assert np.array_equal(cl, ora.clusters) and len(np.unique(cl)) < 4
    d = synth.random_dofs(K, 27, 20, seed=4)
    gpu.set_dofs(d)
    ora.Q = d.copy()
    gpu.advance_steps(8)
    ora.run_lts(8)
    check_parity(gpu.get_dofs(), ora.Q, 27, TOL)
    m = synth.permute_vertex_order(synth.periodic_cube(4), seed=7)
    K = m["tet"].shape[0]
    gpu, ora, _ = make_pair(5, 3, m, dict(synth.homogeneous(K), qp=np.full(K, 80.0), qs=np.full(K, 40.0)),
                            500.0, 20000.0)
    gpu.set_contraction("sparse")
    gpu.setup_clusters(1, 0.5)
    d = synth.random_dofs(K, 27, 35, seed=3)
    gpu.set_dofs(d)
    ora.Q = d.copy()
    gpu.advance_steps(20)
    ora.run_gts(ora.time_step_gts(0.5), 20)
    report_parity("sparse engine: periodic cube, O5, 3 mechanisms, GTS, 20 steps",
                  check_parity(gpu.get_dofs(), ora.Q, 27, TOL))


def test_dof_copy_wait_runs_out_and_handle_recovers():
    """Failure path of the predict kernel's asynchronous DOF copy, without a GPU fault: with
    the copies suppressed, every bounded wait runs out at a short bound; the next
    synchronising call reports LTS_ERR_TIMEOUT, and after restoring the defaults the same
    handle runs correctly against the oracle."""
    from paper_2202_10313_gb300 import binding
    m = synth.graded_box(3, 3, 2, 200.0, 100.0, seed=7)
    mat = synth.random_layers(m, n_layers=2, seed=3)
    gpu, ora, _ = make_pair(5, 3, m, mat)
    gpu.set_contraction("sparse")
    gpu.setup_clusters(1, 0.5)
    ora.setup_clusters(1, 0.5)
    K = m["tet"].shape[0]
    d0 = synth.random_dofs(K, 27, 35, seed=12)
    gpu.set_wait_limit(200000, suppress_commit=True)
    gpu.set_dofs(d0)
    gpu.advance_steps(2)
    with pytest.raises(binding.LtsError) as ei:
        gpu.get_dofs()
    assert ei.value.code == binding.LTS_ERR_TIMEOUT
    gpu.set_wait_limit()
    gpu.set_dofs(d0)
    ora.Q = d0.copy()
    gpu.advance_steps(2)
    ora.run_gts(ora.time_step_gts(0.5), 2)
    err = rel_l2_groups(gpu.get_dofs(), ora.Q, 9)
    assert err["all"] <= TOL, err
