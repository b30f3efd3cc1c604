"""Macro steps replayed from CUDA graphs: the same launches as issued directly, so DOFs and
seismograms are bitwise equal with and without graphs, across even and odd macro steps
(the coarsest cluster's parity) and when the graph must be re-captured (engine change)."""
import numpy as np
import pytest

from paper_2202_10313_gb300 import build, synth
from gpu_common import make_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _run(graphs, switch_engine=False):
    m = synth.graded_box(5, 5, 3, 250.0, 125.0, seed=21)
    mat = synth.random_layers(m, n_layers=3, seed=8)
    gpu, _, _ = make_pair(5, 3, m, mat)
    gpu.set_graphs(graphs)
    gpu.add_point_source(np.array([610.0, 640.0, -260.0]), np.array([0.2, -0.4, 0.2, 1.0, 0.1, -0.3]), 8.0, 0.06,
                         1e12)
    gpu.setup_clusters(3, 0.5)
    dt_rec = gpu.info()["finest_dt"] * 0.73
    rids = [gpu.add_receiver(np.array([300.0 + 170.0 * i, 400.0 + 90.0 * i, -40.0 - 30.0 * i]), dt_rec)
            for i in range(3)]
    gpu.setup_clusters(3, 0.5)
    K = m["tet"].shape[0]
    gpu.set_dofs(synth.random_dofs(K, 27, 35, seed=31))
    for step in range(5):                                 # five macro steps of 4 finest steps
        if switch_engine and step == 2:
            gpu.set_contraction("tf32x3")
        if switch_engine and step == 3:
            gpu.set_contraction("fp32")
        if switch_engine and step == 4:
            gpu.set_contraction("sparse")
            gpu.set_tile(0)
        gpu.advance_steps(4)
    traces = [gpu.seismogram(r) for r in rids]
    return gpu.get_dofs(), traces, gpu.info()["launches"]


@pytest.mark.parametrize("switch_engine", [False, True])
def test_graph_replay_is_bitwise_equal_to_direct_launches(switch_engine):
    q1, t1, n1 = _run(True, switch_engine)
    q0, t0, n0 = _run(False, switch_engine)
    assert np.array_equal(q1, q0)
    assert n1 == n0
    for (ta, va), (tb, vb) in zip(t1, t0):
        assert np.array_equal(ta, tb) and np.array_equal(va, vb) and len(ta) > 0
