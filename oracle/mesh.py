"""Oracle: element geometry and face neighbours (test infrastructure).

Sec. III-A: conforming unstructured tetrahedral meshes; element k maps the
reference tetrahedron affinely, x = x0 + J xi; the neighbour surface kernel needs,
for each face i of k, the neighbour k_i, the neighbour's local face j_k(i) and the
orientation h_k(i) selecting one of the 12 matrices F-_{j,h}.

Face boundary codes (per element face, face numbering of ``basis.FACE_VERTS``):
0 interior, 1 absorbing, 2 free surface, 3 periodic.
"""
import numpy as np

from .basis import FACE_VERTS

BC_INTERIOR, BC_ABSORBING, BC_FREE, BC_PERIODIC = 0, 1, 2, 3


class MeshError(ValueError):
    pass


class Mesh:
    """Geometry and connectivity of a tetrahedral mesh.

    xyz (nv,3) float, tet (K,4) int, face_bc (K,4) int, period (3,) or None.
    Attributes: J (K,3,3), detJ (K,), Jinv (K,3,3) with Jinv[k][c][d] = dxi_c/dx_d,
    normal (K,4,3) outward unit normals, area (K,4), nbr (K,4) neighbour element or
    -1, nbr_face (K,4) = j, nbr_orient (K,4) = h, insphere diameter dins (K,).
    """

    def __init__(self, xyz, tet, face_bc, period=None):
        self.xyz = np.asarray(xyz, dtype=float)
        self.tet = np.asarray(tet, dtype=np.int64)
        self.face_bc = np.asarray(face_bc, dtype=np.int64).reshape(-1, 4)
        self.period = None if period is None else np.asarray(period, dtype=float)
        self.K = self.tet.shape[0]
        self._geometry()
        self._neighbours()

    def _geometry(self):
        x = self.xyz[self.tet]                        # (K,4,3)
        self.x0 = x[:, 0, :]
        self.J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)
        self.detJ = np.linalg.det(self.J)
        if np.any(self.detJ <= 0.0):
            raise MeshError("tetrahedron with non-positive orientation")
        self.Jinv = np.linalg.inv(self.J)
        self.normal = np.zeros((self.K, 4, 3))
        self.area = np.zeros((self.K, 4))
        for i, (a, b, c) in enumerate(FACE_VERTS):
            cr = np.cross(x[:, b] - x[:, a], x[:, c] - x[:, a])
            ln = np.linalg.norm(cr, axis=1)
            self.area[:, i] = 0.5 * ln
            self.normal[:, i, :] = cr / ln[:, None]
        self.volume = self.detJ / 6.0
        # insphere diameter 6 V / (sum of face areas)
        self.dins = 6.0 * self.volume / self.area.sum(axis=1)
        self.centroid = x.mean(axis=1)

    def _vertex_keys(self):
        """Vertex identity used to match periodic faces: position modulo the box."""
        if self.period is None:
            return None
        canon = np.mod(self.xyz, self.period[None, :])
        canon[np.isclose(canon, self.period[None, :], rtol=0.0, atol=0.0)] = 0.0
        table = {}
        keys = np.empty(len(canon), dtype=np.int64)
        for v, c in enumerate(map(tuple, canon)):
            keys[v] = table.setdefault(c, len(table))
        return keys

    def _neighbours(self):
        """Face matching by sorted vertex keys (lexicographic sort), then (j, h).

        Two faces match when their sorted vertex keys (vertex ids; for periodic faces the
        position modulo the box) and boundary kind agree; every such group must hold
        exactly two faces. h is the position in the neighbour's face of the local face's
        first vertex; the other two must appear in reversed cyclic order."""
        K = self.K
        pkeys = self._vertex_keys()
        self.nbr = -np.ones((K, 4), dtype=np.int64)
        self.nbr_face = -np.ones((K, 4), dtype=np.int64)
        self.nbr_orient = -np.ones((K, 4), dtype=np.int64)
        ids = np.stack([self.tet[:, list(fv)] for fv in FACE_VERTS], axis=1)      # (K, 4, 3)
        bc = self.face_bc
        if np.any(bc == BC_PERIODIC) and pkeys is None:
            raise MeshError("periodic face without a period")
        if pkeys is not None:
            ids = np.where((bc == BC_PERIODIC)[:, :, None], pkeys[ids], ids)
        sel = (bc == BC_INTERIOR) | (bc == BC_PERIODIC)
        elem, face = np.nonzero(sel)
        fids = ids[elem, face]                                                     # (F, 3) in face order
        skey = np.sort(fids, axis=1)
        kind = bc[elem, face]
        order = np.lexsort((skey[:, 2], skey[:, 1], skey[:, 0], kind))
        sk = np.concatenate([kind[order][:, None], skey[order]], axis=1)
        same_next = np.all(sk[1:] == sk[:-1], axis=1)
        if len(order) % 2 or not np.all(same_next[0::2]) or np.any(same_next[1::2]):
            raise MeshError("a face is not shared by exactly two elements")
        a_, b_ = order[0::2], order[1::2]
        for e_, g_ in ((a_, b_), (b_, a_)):
            ide, idg = fids[e_], fids[g_]
            h = np.argmax(idg == ide[:, :1], axis=1)
            r = np.arange(len(h))
            ok = (idg[r, h] == ide[:, 0]) & (idg[r, (h + 2) % 3] == ide[:, 1]) & (idg[r, (h + 1) % 3] == ide[:, 2])
            if not np.all(ok):
                raise MeshError("inconsistent face orientation")
            self.nbr[elem[e_], face[e_]] = elem[g_]
            self.nbr_face[elem[e_], face[e_]] = face[g_]
            self.nbr_orient[elem[e_], face[e_]] = h

    def xi_of(self, k, x):
        """Reference coordinates of physical point x inside element k."""
        return self.Jinv[k] @ (np.asarray(x, dtype=float) - self.x0[k])

    def locate(self, x, tol=1e-12):
        """First element (lowest index) whose closed tetrahedron contains x."""
        x = np.asarray(x, dtype=float)
        xi = np.einsum("kcd,kd->kc", self.Jinv, x[None, :] - self.x0)
        bary = np.concatenate([1.0 - xi.sum(axis=1, keepdims=True), xi], axis=1)
        inside = np.all(bary >= -tol, axis=1)
        idx = np.nonzero(inside)[0]
        if len(idx) == 0:
            raise MeshError("point outside the mesh")
        return int(idx[0])
