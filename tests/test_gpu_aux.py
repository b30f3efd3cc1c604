"""Auxiliary subsystems on the GPU: checkpoint / resume at a macro-step boundary reproduces
the uninterrupted run bitwise (DOFs and seismograms); the energy reduction flags a state
holding NaN or Inf; checkpoints refuse a different set-up."""
import numpy as np
import pytest

from paper_2202_10313_gb300 import binding, build, synth
from gpu_common import initial_field, make_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _solver(m, mat, fused=1):
    g = binding.Solver(4, 3, device=0, n_fused=fused)
    g.set_mesh(m["xyz"], m["tet"], m["face_bc"])
    g.set_material(mat["rho"], mat["vp"], mat["vs"], mat["qp"], mat["qs"], 0.1, 5.0)
    g.add_point_source(np.array([610.0, 640.0, -260.0]), np.array([0.2, -0.4, 0.2, 1.0, 0.1, -0.3]), 8.0, 0.06, 1e12)
    g.add_receiver(np.array([400.0, 500.0, -50.0]), 3e-4)
    g.add_receiver(np.array([700.0, 300.0, -120.0]), 3e-4)
    g.setup_clusters(3, 0.5)
    return g


@pytest.mark.parametrize("fused", [1, 4])
def test_checkpoint_resume_is_bitwise(tmp_path, fused):
    m = synth.graded_box(5, 5, 3, 250.0, 125.0, seed=21)
    mat = synth.random_layers(m, n_layers=3, seed=8)
    a = _solver(m, mat, fused)
    a.project_initial(initial_field(27, [600.0, 700.0, -300.0], 400.0))
    a.advance_steps(8)
    path = tmp_path / "state.ckpt"
    a.checkpoint_save(path)
    a.advance_steps(8)
    b = _solver(m, mat, fused)
    b.checkpoint_load(path)
    assert b.info()["time"] == a.info()["time"] - 8 * a.info()["finest_dt"]
    b.advance_steps(8)
    assert np.array_equal(a.get_dofs(), b.get_dofs())
    for rid in range(2):
        for f in range(fused):
            ta, va = a.seismogram(rid, f)
            tb, vb = b.seismogram(rid, f)
            assert np.array_equal(ta, tb) and np.array_equal(va, vb) and len(ta) > 0
    # a different set-up is refused; mid-macro-step saves are refused
    c = binding.Solver(4, 3, device=0)
    c.set_mesh(m["xyz"], m["tet"], m["face_bc"])
    c.set_material(mat["rho"], mat["vp"], mat["vs"], mat["qp"], mat["qs"], 0.1, 5.0)
    c.setup_clusters(2, 0.5)
    with pytest.raises(binding.LtsError) as ei:
        c.checkpoint_load(path)
    assert ei.value.code == binding.LTS_ERR_ARG


def test_energy_sentinel_flags_non_finite_state():
    m = synth.graded_box(3, 3, 2, 250.0, 125.0, seed=2)
    mat = synth.random_layers(m, n_layers=2, seed=3)
    g, _, _ = make_pair(3, 0, m, mat)
    g.setup_clusters(1, 0.5)
    K = m["tet"].shape[0]
    d = synth.random_dofs(K, 9, 10, seed=1)
    g.set_dofs(d)
    assert np.isfinite(g.energy())
    d[7, 6, 3] = np.nan
    g.set_dofs(d)
    with pytest.raises(binding.LtsError) as ei:
        g.energy()
    assert ei.value.code == binding.LTS_ERR_NONFINITE
