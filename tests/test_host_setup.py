"""CPU checks of the library's host-side set-up against the oracle.

The library builds its operators by exact polynomial integration and its quadrature
from Gauss-Jacobi nodes; the oracle uses collapsed Gauss-Legendre quadrature. Agreement
to ~1e-12 pins both routes. Clustering runs on a host-only handle (device < 0)."""
import numpy as np
import pytest

from oracle.basis import Basis
from oracle.mesh import Mesh
from oracle import lts as olts
from paper_2202_10313_gb300 import binding, build, synth


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


@pytest.mark.parametrize("order", [3, 4, 5])
def test_reference_operators_match_oracle(order):
    K, Ft, Fb = binding.reference_operators(order)
    b = Basis(order)
    # monomial expansion of degree-2(O-1) products cancels digits: allow 1e-12 relative
    # to the largest entry, times the number of terms
    tol = 1e-12 * b.nb
    for c in range(3):
        assert np.abs(K[c] - b.K[c]).max() < tol * np.abs(b.K[c]).max()
    for i in range(4):
        assert np.abs(Ft[i] - b.Ft[i]).max() < tol * np.abs(b.Ft[i]).max()
    for j in range(4):
        for h in range(3):
            assert np.abs(Fb[j, h] - b.Fb[j][h]).max() < tol * np.abs(b.Fb[j][h]).max()


@pytest.mark.parametrize("order", [3, 5])
def test_basis_values_and_quadrature(order):
    rng = np.random.default_rng(order)
    xi = rng.dirichlet(np.ones(4), size=40)[:, 1:]
    b = Basis(order)
    # monomial evaluation of degree O-1 polynomials loses a few digits to cancellation
    assert np.abs(binding.eval_basis(order, xi) - b.phi(xi)).max() < 1e-10
    qx, qw = binding.quadrature_rule(order)
    assert abs(qw.sum() - 1.0 / 6.0) < 1e-15
    # exact for phi_a phi_b (degree 2(O-1)): the library's rule reproduces the mass matrix
    ph = binding.eval_basis(order, qx)
    assert np.abs((ph * qw[:, None]).T @ ph - np.eye(b.nb)).max() < 1e-10


def _host_handle(order, m, mesh, mat):
    s = binding.Solver(order, m, device=-1)
    s.set_mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"], mesh.get("period"))
    s.set_material(mat["rho"], mat["vp"], mat["vs"], mat.get("qp"), mat.get("qs"))
    return s


@pytest.mark.parametrize("n_clusters", [1, 3, 5])
def test_clusters_match_oracle(n_clusters):
    m = synth.graded_box(8, 8, 6, 250.0, 125.0)
    mat = synth.random_layers(m)
    s = _host_handle(5, 3, m, mat)
    cl, lam, sp = s.setup_clusters(n_clusters, 0.5)
    om = Mesh(m["xyz"], m["tet"], m["face_bc"])
    dt = olts.cfl_time_steps(om.dins, mat["vp"], 5, 0.5)
    lam_o, cl_o, sp_o = olts.search_lambda(dt, om.nbr, n_clusters)
    assert lam == lam_o
    assert np.array_equal(cl, cl_o)
    assert abs(sp / sp_o - 1) < 1e-12
    if n_clusters == 1:
        assert lam == 1.0 and sp == 1.0
    else:
        assert len(np.unique(cl)) > 1 and sp > 1.0


def test_forced_clusters_must_be_normalised():
    m = synth.graded_box(3, 3, 3, 100.0, 50.0)
    mat = synth.homogeneous(m["tet"].shape[0])
    s = _host_handle(3, 0, m, mat)
    om = Mesh(m["xyz"], m["tet"], m["face_bc"])
    bad = np.zeros(om.K, dtype=np.int32)
    k = 0
    bad[k] = 2
    with pytest.raises(binding.LtsError) as ei:
        s.force_clusters(bad, 3, 0.5)
    assert ei.value.code == binding.LTS_ERR_ARG
    s.force_clusters(olts.normalise(bad, om.nbr), 3, 0.5)


def test_mesh_errors():
    m = synth.graded_box(2, 2, 2, 100.0, 50.0)
    s = binding.Solver(3, 0, device=-1)
    tet = m["tet"].copy()
    tet[0, [1, 2]] = tet[0, [2, 1]]           # inverted element
    with pytest.raises(binding.LtsError) as ei:
        s.set_mesh(m["xyz"], tet, m["face_bc"])
    assert ei.value.code == binding.LTS_ERR_MESH
    bc = m["face_bc"].copy()
    k = int(np.nonzero(bc.max(axis=1) == 0)[0][0])
    bc[k, 0] = 0
    tet = m["tet"][1:]                          # drop an element: its neighbours' faces are open
    with pytest.raises(binding.LtsError) as ei:
        s.set_mesh(m["xyz"], tet, m["face_bc"][1:])
    assert ei.value.code == binding.LTS_ERR_MESH
    with pytest.raises(binding.LtsError) as ei:
        s.set_mesh(m["xyz"], m["tet"], np.full_like(m["face_bc"], 7))
    assert ei.value.code == binding.LTS_ERR_ARG
    s.set_mesh(m["xyz"], m["tet"], m["face_bc"])
    with pytest.raises(binding.LtsError) as ei:
        s.advance_steps(1, stream=0)
    assert ei.value.code == binding.LTS_ERR_STATE


def test_periodic_mesh_neighbours_match_oracle():
    m = synth.permute_vertex_order(synth.periodic_cube(3), seed=4)
    s = binding.Solver(3, 0, device=-1)
    s.set_mesh(m["xyz"], m["tet"], m["face_bc"], m["period"])
    mat = synth.homogeneous(m["tet"].shape[0])
    s.set_material(mat["rho"], mat["vp"], mat["vs"])
    cl, lam, sp = s.setup_clusters(1, 0.5)
    assert lam == 1.0 and np.all(cl == 0)


def test_fused_handle_host_checks():
    """A fused handle (16 simulations) sets up like a single one; sources take a
    simulation index in [0, 16)."""
    m = synth.graded_box(2, 2, 2, 100.0, 50.0)
    s = binding.Solver(4, 3, device=-1, n_fused=16)
    s.set_mesh(m["xyz"], m["tet"], m["face_bc"])
    K = m["tet"].shape[0]
    mat = synth.homogeneous(K)
    s.set_material(mat["rho"], mat["vp"], mat["vs"], np.full(K, 80.0), np.full(K, 40.0), 0.1, 5.0)
    x = m["xyz"].mean(axis=0)
    m6 = np.array([1.0, 0, 0, 0, 0, 0])
    s.add_point_source(x, m6, 2.0, 0.5, fused_idx=15)
    for bad in (-1, 16):
        with pytest.raises(binding.LtsError) as ei:
            s.add_point_source(x, m6, 2.0, 0.5, fused_idx=bad)
        assert ei.value.code == binding.LTS_ERR_ARG
    cl, lam, sp = s.setup_clusters(2, 0.5)
    assert cl.shape == (K,)
