"""Emulated partitioned run on one GPU (Sec. V-C): cut faces take their neighbour
contribution from face-local messages H = X F-_{j,h} computed on the sending side by a
pack kernel. The arithmetic and its order are those of the unpartitioned run with the same
(gather-and-product) neighbour kernel, so the DOFs must be bitwise equal to it, and within
1e-4 of the oracle. These runs use the FP32 dense-block engine, whose neighbour kernel is the
one partitioned runs use."""
import numpy as np
import pytest

from paper_2202_10313_gb300 import binding, build, synth
from gpu_common import make_pair, rel_l2_groups

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


@pytest.mark.parametrize("order,n_mech,n_parts", [(5, 3, 2), (5, 3, 5), (4, 0, 3)])
def test_partitioned_run_equals_unpartitioned_and_oracle(order, n_mech, n_parts):
    m = synth.permute_vertex_order(synth.graded_box(6, 5, 3, 250.0, 125.0, seed=12), seed=2)
    mat = synth.random_layers(m, n_layers=3, seed=5)
    K = m["tet"].shape[0]
    nq, nb = 9 + 6 * n_mech, order * (order + 1) * (order + 2) // 6
    d0 = synth.random_dofs(K, nq, nb, seed=21)
    xs, m6 = np.array([610.0, 640.0, -260.0]), np.array([0.2, -0.4, 0.2, 1.0, 0.1, -0.3])
    runs = []
    for parted in (False, True):
        gpu, ora, _ = make_pair(order, n_mech, m, mat)
        gpu.set_contraction("fp32")
        gpu.add_point_source(xs, m6, 8.0, 0.06, 1e12)
        cl, _, _ = gpu.setup_clusters(3, 0.5)
        if parted:
            part, st = gpu.partition(n_parts)
            gpu.set_partition(part, n_parts)
        gpu.set_dofs(d0)
        gpu.advance_steps(8)
        runs.append(gpu.get_dofs())
        if parted:
            # 9 x F FP32 values per cut face and update of its receiving element
            F = order * (order + 1) // 2
            assert gpu.exchange_bytes() == 2 * st["msgs_per_macro"] * 9 * F * 4
    assert np.array_equal(runs[0], runs[1])
    ora.add_point_source(xs, m6, 8.0, 0.06, 1e12)
    ora.setup_clusters(3, 0.5)
    ora.Q = d0.copy()
    ora.run_lts(8)
    err = rel_l2_groups(runs[1], ora.Q, nq)
    for k, v in err.items():
        assert v <= 1e-4, err


def test_partition_with_tensor_cores_and_switch_off():
    m = synth.graded_box(5, 5, 3, 250.0, 125.0, seed=12)
    mat = synth.random_layers(m, n_layers=3, seed=5)
    K = m["tet"].shape[0]
    d0 = synth.random_dofs(K, 27, 35, seed=4)
    gpu, ora, _ = make_pair(5, 3, m, mat)
    gpu.set_contraction("tf32x3")
    gpu.setup_clusters(3, 0.5)
    part, _ = gpu.partition(4)
    gpu.set_partition(part, 4)
    gpu.set_dofs(d0)
    gpu.advance_steps(4)
    a = gpu.get_dofs()
    gpu.set_partition(None)
    gpu.set_dofs(d0)
    gpu.advance_steps(4)
    assert np.array_equal(a, gpu.get_dofs())


def test_adjoint_of_a_partitioned_run_equals_the_unpartitioned_adjoint():
    """The partitioned forward run is bitwise the unpartitioned one, and so is its adjoint:
    misfit, gradient, samples and dJ/dQ0 (three clusters, elastic)."""
    order = 4
    m = synth.permute_vertex_order(synth.graded_box(6, 5, 3, 250.0, 125.0, seed=12), seed=2)
    mat = synth.random_layers(m, n_layers=3, seed=5)
    K = m["tet"].shape[0]
    d0 = synth.random_dofs(K, 9, 20, seed=23)
    rec = [np.array([400.0, 500.0, -20.0]), np.array([900.0, 700.0, -60.0])]
    out = []
    for parted in (False, True):
        gpu, _, _ = make_pair(order, 0, m, mat)
        gpu.set_contraction("fp32")
        gpu.add_point_source(np.array([610.0, 640.0, -260.0]), np.array([0.2, -0.4, 0.2, 1.0, 0.1, -0.3]), 8.0, 0.06,
                             1e12)
        for x in rec:
            gpu.add_receiver(x, 1e-3)
        gpu.setup_clusters(3, 0.5)
        if parted:
            part, _ = gpu.partition(3)
            gpu.set_partition(part, 3)
        gpu.set_dofs(d0)
        data = np.full((3, 2, 3), 1e-7)
        out.append(gpu.misfit_gradient(8, data, every=1, want_dq0=True))
        gpu.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))


@pytest.mark.parametrize("F", [4, 8])
def test_fused_partitioned_run_equals_fused_unpartitioned(F):
    """Fused simulations in a partitioned run: one face-local message per simulation and cut
    face; every simulation bitwise equal to the fused unpartitioned run, message bytes F times
    those of one simulation."""
    order, n_mech = 5, 3
    m = synth.permute_vertex_order(synth.graded_box(6, 5, 3, 250.0, 125.0, seed=12), seed=2)
    mat = synth.random_layers(m, n_layers=3, seed=5)
    K = m["tet"].shape[0]
    nq, nb = 27, 35
    d0 = np.stack([synth.random_dofs(K, nq, nb, seed=30 + f) for f in range(F)])
    lo, hi = m["xyz"].min(axis=0), m["xyz"].max(axis=0)
    pos, m6, f0 = synth.random_sources(F, lo + 0.2 * (hi - lo), hi - 0.2 * (hi - lo), f0_range=(4.0, 8.0), seed=3)
    runs, xbytes = [], []
    for parted in (False, True):
        g = binding.Solver(order, n_mech, device=0, n_fused=F)
        g.set_contraction("fp32")
        g.set_mesh(m["xyz"], m["tet"], m["face_bc"])
        g.set_material(mat["rho"], mat["vp"], mat["vs"], mat["qp"], mat["qs"], 0.1, 5.0)
        for f in range(F):
            g.add_point_source(pos[f], m6[f], f0[f], 0.1, 1e12, fused_idx=f)
        g.setup_clusters(3, 0.5)
        if parted:
            part, _ = g.partition(3)
            g.set_partition(part, 3)
        g.set_dofs(d0)
        g.advance_steps(8)
        runs.append(g.get_dofs())
        xbytes.append(g.exchange_bytes())
        g.close()
    assert np.array_equal(runs[0], runs[1])
    assert xbytes[0] == 0 and xbytes[1] > 0
    # one simulation: the same cut, 1/F of the bytes
    s = binding.Solver(order, n_mech, device=0)
    s.set_mesh(m["xyz"], m["tet"], m["face_bc"])
    s.set_material(mat["rho"], mat["vp"], mat["vs"], mat["qp"], mat["qs"], 0.1, 5.0)
    s.setup_clusters(3, 0.5)
    part, _ = s.partition(3)
    s.set_partition(part, 3)
    s.set_dofs(d0[0])
    s.advance_steps(8)
    assert xbytes[1] == F * s.exchange_bytes()
    s.close()
