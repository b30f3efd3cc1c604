"""Pins for the oracle's basis, quadrature and reference operators (Sec. III-A)."""
import json
import os

import numpy as np
import pytest

from oracle.basis import (Basis, closed_form_tet_norm2, closed_form_tri_norm2, n_basis,
                          n_face_basis, tet_modes, tri_modes, REF_VERTS, FACE_VERTS)
from oracle.mesh import Mesh
from paper_2202_10313_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))


@pytest.fixture(scope="module", params=[3, 4, 5])
def basis(request):
    return Basis(request.param)


def test_counts_match_paper():
    assert n_basis(4) == GOLD["n_basis"]["4"]
    assert n_basis(5) == GOLD["n_basis"]["5"]
    assert n_face_basis(5) == GOLD["n_face_basis"]["5"]
    g = GOLD["derivative_values"]
    assert g["order"] * 9 * n_basis(g["order"]) == g["values"]
    for o in (3, 4, 5):
        assert len(tet_modes(o)) == n_basis(o) and len(tri_modes(o)) == n_face_basis(o)
        # hierarchical: degree <= p prefix is a leading block
        degs = [sum(m) for m in tet_modes(o)]
        assert degs == sorted(degs)


def test_orthonormal(basis):
    assert np.abs(basis.mass - np.eye(basis.nb)).max() < 1e-13
    ps = basis.psi(basis.fqp)
    fm = (ps * basis.fqw[:, None]).T @ ps
    assert np.abs(fm - np.eye(basis.nf)).max() < 1e-13


def test_norms_match_textbook_jacobi_closed_form(basis):
    cf = np.array([closed_form_tet_norm2(*m) for m in tet_modes(basis.order)])
    assert np.allclose(basis.norm2, cf, rtol=1e-13, atol=0)
    cft = np.array([closed_form_tri_norm2(*m) for m in tri_modes(basis.order)])
    assert np.allclose(basis.fnorm2, cft, rtol=1e-13, atol=0)
    # phi_000 is the constant 1/sqrt(vol) = sqrt(6)
    assert abs(basis.phi(np.array([[0.1, 0.2, 0.3]]))[0, 0] - np.sqrt(6.0)) < 1e-14


def _face_geometry():
    nrm, area = [], []
    for (a, b, c) in FACE_VERTS:
        cr = np.cross(REF_VERTS[b] - REF_VERTS[a], REF_VERTS[c] - REF_VERTS[a])
        nrm.append(cr / np.linalg.norm(cr))
        area.append(0.5 * np.linalg.norm(cr))
    return nrm, area


def test_divergence_theorem_links_stiffness_and_flux_matrices(basis):
    """int d_c(phi_a phi_b) = sum_faces n_c int phi_a phi_b dS; the face integral is
    2|S_i| sum_f F~_i[a,f] F~_i[b,f] because psi spans the face traces."""
    nrm, area = _face_geometry()
    for c in range(3):
        lhs = basis.K[c] + basis.K[c].T
        rhs = sum(nrm[i][c] * 2.0 * area[i] * basis.Ft[i] @ basis.Ft[i].T for i in range(4))
        assert np.abs(lhs - rhs).max() < 1e-12
    # outward orientation of the face table
    cen = REF_VERTS.mean(axis=0)
    for i, (a, b, c) in enumerate(FACE_VERTS):
        assert np.dot(nrm[i], REF_VERTS[a] - cen) > 0


def test_derivative_exact_on_polynomials(basis):
    """Q K_c^T is the projection of d/dxi_c; exact for degree <= O-1 polynomials."""
    rng = np.random.default_rng(0)
    O = basis.order
    expo = [(a, b, c) for a in range(O) for b in range(O) for c in range(O) if a + b + c <= O - 1]
    coef = rng.normal(size=len(expo))

    def p(x):
        return sum(cf * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c for cf, (a, b, c) in zip(coef, expo))

    def dp(x, d):
        out = np.zeros(len(x))
        for cf, e in zip(coef, expo):
            if e[d] == 0:
                continue
            ee = list(e)
            ee[d] -= 1
            out += cf * e[d] * x[:, 0] ** ee[0] * x[:, 1] ** ee[1] * x[:, 2] ** ee[2]
        return out

    q = basis.project(p(basis.qp))
    pts = rng.dirichlet(np.ones(4), size=50)[:, 1:]
    assert np.abs(basis.phi(pts) @ q - p(pts)).max() < 1e-12
    for c in range(3):
        dq = q @ basis.K[c].T
        assert np.abs(basis.phi(pts) @ dq - dp(pts, c)).max() < 1e-10


def test_neighbour_flux_matrices_trace_consistency():
    """Project one global polynomial on two face-adjacent tets: the face trace seen
    from both sides agrees, T_k F~_i = T_nbr F-_{j,h}, for every (j, h) present."""
    O = 4
    b = Basis(O)
    m = synth.permute_vertex_order(synth.graded_box(3, 3, 3, 100.0, 50.0, jitter=0.15, seed=5), seed=6)
    mesh = Mesh(m["xyz"], m["tet"], m["face_bc"])
    rng = np.random.default_rng(1)
    expo = [(a, bb, c) for a in range(O) for bb in range(O) for c in range(O) if a + bb + c <= O - 1]
    coef = rng.normal(size=len(expo))

    def p(x):
        x = x / 300.0
        return sum(cf * x[:, 0] ** a * x[:, 1] ** bb * x[:, 2] ** c for cf, (a, bb, c) in zip(coef, expo))

    pts = mesh.x0[:, None, :] + np.einsum("kdc,qc->kqd", mesh.J, b.qp)
    vals = p(pts.reshape(-1, 3)).reshape(mesh.K, -1)
    Q = b.project(vals)
    seen = set()
    worst = 0.0
    for k in range(mesh.K):
        for i in range(4):
            nb = mesh.nbr[k, i]
            if nb < 0:
                continue
            j, h = mesh.nbr_face[k, i], mesh.nbr_orient[k, i]
            seen.add((int(j), int(h)))
            worst = max(worst, np.abs(Q[k] @ b.Ft[i] - Q[nb] @ b.Fb[j][h]).max())
    assert worst < 1e-10 * max(1.0, np.abs(Q).max())
    assert len(seen) == 12
