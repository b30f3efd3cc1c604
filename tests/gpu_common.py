"""Shared helpers of the GPU parity tests: run the same seeded case on the library
(through the C ABI) and on the oracle, and compare."""
import numpy as np

from oracle.mesh import Mesh
from oracle.scheme import Solver as OracleSolver
from paper_2202_10313_gb300 import binding, synth

GROUPS = {"stress": slice(0, 6), "velocity": slice(6, 9), "memory": slice(9, None)}


def rel_l2_groups(got, want, nq):
    out = {}
    for name, sl in GROUPS.items():
        if name == "memory" and nq <= 9:
            continue
        w = want[:, sl]
        den = np.sqrt(np.sum(w ** 2))
        out[name] = float(np.sqrt(np.sum((got[:, sl] - w) ** 2)) / den) if den > 0 else float(np.abs(got[:, sl]).max())
    out["all"] = float(np.sqrt(np.sum((got - want) ** 2)) / np.sqrt(np.sum(want ** 2)))
    return out


def rel_elem_groups(got, want, nq):
    """Elementwise companion of rel_l2_groups: per quantity group, the largest per-element
    error norm over the largest per-element norm of the reference, max_k |got_k - want_k| /
    max_k |want_k| (norms over the group's quantities and modes of one element). A defect
    confined to a few elements (one face orientation, the boundary faces, the source
    element) shows here even where it vanishes in the global L2."""
    out = {}
    for name, sl in GROUPS.items():
        if name == "memory" and nq <= 9:
            continue
        w = want[:, sl].reshape(len(want), -1)
        d = (got[:, sl] - want[:, sl]).reshape(len(want), -1)
        den = np.sqrt(np.sum(w ** 2, axis=1)).max()
        num = np.sqrt(np.sum(d ** 2, axis=1)).max()
        out[name] = float(num / den) if den > 0 else float(num)
    return out


def check_parity(got, want, nq, tol):
    """Asserts the relative L2 per quantity group and the elementwise maximum (both <= tol);
    returns the L2 figures with the elementwise ones under 'elem_*' keys."""
    err = rel_l2_groups(got, want, nq)
    el = rel_elem_groups(got, want, nq)
    for k, v in err.items():
        assert v <= tol, ("relative L2", err, el)
    for k, v in el.items():
        assert v <= tol, ("elementwise", err, el)
    out = dict(err)
    out.update({"elem_" + k: v for k, v in el.items()})
    return out


def make_pair(order, n_mech, mesh, mat, f_min=0.1, f_max=5.0):
    gpu = binding.Solver(order, n_mech, device=0)
    gpu.set_mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"], mesh.get("period"))
    gpu.set_material(mat["rho"], mat["vp"], mat["vs"], mat.get("qp"), mat.get("qs"), f_min, f_max)
    om = Mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"], mesh.get("period"))
    ora = OracleSolver(order, n_mech, om, mat["rho"], mat["vp"], mat["vs"], mat.get("qp"), mat.get("qs"), f_min, f_max)
    return gpu, ora, om


def initial_field(nq, center, width, plane=None):
    """Smooth initial state: Gaussian pulse in all quantities (+ optional plane wave)."""
    g = synth.gaussian_pulse(center, width, nq)

    def fn(x):
        v = g(x)
        if plane is not None:
            v[:, :9] += plane(x, 0.0)
        return v

    return fn


def report_parity(case, errors):
    """One line per parity case (run pytest with -s to see them): the worst relative L2
    error against the FP64 oracle per quantity group."""
    import json
    print("PARITY " + json.dumps({"case": case, **{k: float(v) for k, v in errors.items()}}))
