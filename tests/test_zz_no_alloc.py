"""The allocation-free energy entry point against lts_energy, through the C ABI.

lts_energy_noalloc serves callers that cannot allocate device memory while they run
(their memory belongs to another framework's pool, or their time loop must not allocate):
they pass their own device buffers and the call uses only a fixed scratch array built
into the library. This file is collected last so that a failure here comes after every
other test has run."""
import ctypes

import numpy as np
import pytest

from paper_2202_10313_gb300 import binding, build, synth

pytestmark = pytest.mark.gpu


def _det(mesh):
    x = mesh["xyz"][mesh["tet"]]
    return np.linalg.det(np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2))


def test_noalloc_energy_matches_handle_energy_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    m = synth.graded_box(4, 4, 3, 200.0, 100.0, seed=31)
    mat = synth.random_layers(m, n_layers=2, seed=9)
    K = m["tet"].shape[0]
    s = binding.Solver(5, 3, device=0)
    s.set_mesh(m["xyz"], m["tet"], m["face_bc"])
    s.set_material(mat["rho"], mat["vp"], mat["vs"], mat["qp"], mat["qs"])
    s.setup_clusters(2, 0.5)
    s.set_dofs(synth.random_dofs(K, 27, 35, seed=5))
    mu = mat["rho"] * mat["vs"] ** 2
    lam = mat["rho"] * mat["vp"] ** 2 - 2 * mu
    table = torch.tensor(np.stack([lam, mu, mat["rho"], _det(m)], axis=1), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    L = binding.lib()
    for call in range(2):
        if call == 1:
            s.advance_steps(4)
        want = s.energy()
        dofs = torch.tensor(s.get_dofs(), dtype=torch.float32, device="cuda").contiguous()
        out.fill_(-1.0)
        rc = L.lts_energy_noalloc(5, 3, ctypes.c_void_p(dofs.data_ptr()), ctypes.c_void_p(table.data_ptr()), K,
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == binding.LTS_OK
        torch.cuda.synchronize()
        got = float(out.item())
        assert want > 0 and abs(got / want - 1.0) < 1e-9, (call, got, want)
    # sizes beyond the fixed scratch are rejected before anything runs
    assert L.lts_energy_noalloc(5, 3, ctypes.c_void_p(dofs.data_ptr()), ctypes.c_void_p(table.data_ptr()),
                                262144 + 1, ctypes.c_void_p(out.data_ptr()), None) == binding.LTS_ERR_ARG
