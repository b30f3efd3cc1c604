"""Seeded synthetic inputs: tetrahedral meshes, materials, initial fields, sources, receivers.

This module generates inputs only; it holds none of the solver's arithmetic. The
same arrays feed the solver library and any independent checker.

Meshes are hexahedral grids, each hex split into 6 tetrahedra around its main
diagonal (Kuhn/Freudenthal split: conforming, and translation invariant so a grid
can be periodic). Tetrahedra are emitted positively oriented. Per-face boundary
codes follow the library's face numbering (face i = vertex triple FACE_VERTS[i]):
0 interior, 1 absorbing, 2 free surface, 3 periodic.

Default seeds: mesh 2202, material 10313, sources 7, receivers 11.
"""
import itertools

import numpy as np

FACE_VERTS = ((0, 2, 1), (0, 1, 3), (0, 3, 2), (1, 2, 3))
SEED_MESH, SEED_MATERIAL, SEED_SOURCES, SEED_RECEIVERS = 2202, 10313, 7, 11


def _kuhn_tets(nx, ny, nz):
    """Vertex ids of the 6 nx*ny*nz Kuhn tetrahedra (positively oriented for an
    undistorted grid) of a grid with vertex id (k (ny+1) + j)(nx+1) + i."""
    def vid(i, j, k):
        return (k * (ny + 1) + j) * (nx + 1) + i

    I, J, Kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    I, J, Kk = I.ravel(), J.ravel(), Kk.ravel()
    # order hexes k-major so neighbouring hexes are close in memory
    order = np.lexsort((I, J, Kk))
    I, J, Kk = I[order], J[order], Kk[order]
    tets = []
    for perm in itertools.permutations(range(3)):
        parity = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b]) % 2
        off = np.zeros((4, 3), dtype=np.int64)
        for step in range(1, 4):
            off[step] = off[step - 1]
            if step <= 3:
                off[step, perm[step - 1]] += 1
        verts = [vid(I + off[s, 0], J + off[s, 1], Kk + off[s, 2]) for s in range(4)]
        if parity == 1:
            verts[2], verts[3] = verts[3], verts[2]
        tets.append(np.stack(verts, axis=1))
    tet = np.stack(tets, axis=1).reshape(-1, 4)
    return tet


def _grid_vertices(xs, ys, zs):
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def _boundary_codes(tet, nx, ny, nz, code_of_plane):
    """Per tet face: code_of_plane[p] when all 3 face vertices lie on grid plane p
    (p in xmin, xmax, ymin, ymax, zmin, zmax), else 0."""
    nv = (nx + 1) * (ny + 1) * (nz + 1)
    vi = np.arange(nv) % (nx + 1)
    vj = (np.arange(nv) // (nx + 1)) % (ny + 1)
    vk = np.arange(nv) // ((nx + 1) * (ny + 1))
    planes = [vi == 0, vi == nx, vj == 0, vj == ny, vk == 0, vk == nz]
    bc = np.zeros((tet.shape[0], 4), dtype=np.int32)
    for f, fv in enumerate(FACE_VERTS):
        ids = tet[:, list(fv)]
        for p, on in enumerate(planes):
            allon = on[ids].all(axis=1)
            bc[allon, f] = code_of_plane[p]
    return bc


def periodic_cube(n, length=1.0):
    """Periodic cube [0, L]^3 of n^3 hexes x 6 tets; returns dict(xyz, tet, face_bc, period)."""
    xs = length * np.arange(n + 1) / n
    xyz = _grid_vertices(xs, xs, xs)
    tet = _kuhn_tets(n, n, n)
    bc = _boundary_codes(tet, n, n, n, [3] * 6)
    return dict(xyz=xyz, tet=tet, face_bc=bc, period=np.array([length] * 3))


def periodic_slab(n, z_code=2, length=1.0, nxy=None):
    """[0, L]^3 as n hexes along z and nxy (default n) along x and y, 6 tets each, periodic in
    x and y only: its planes z = 0 and z = L carry boundary code z_code (2 free surface,
    1 absorbing)."""
    nxy = n if nxy is None else nxy
    xs = length * np.arange(nxy + 1) / nxy
    zs = length * np.arange(n + 1) / n
    xyz = _grid_vertices(xs, xs, zs)
    tet = _kuhn_tets(nxy, nxy, n)
    bc = _boundary_codes(tet, nxy, nxy, n, [3, 3, 3, 3, z_code, z_code])
    return dict(xyz=xyz, tet=tet, face_bc=bc, period=np.array([length] * 3))


def graded_box(nx, ny, nz, h, hz_min, grade=4.0, jitter=0.15, seed=SEED_MESH):
    """Box [0, nx h] x [0, ny h] x [-D, 0], z-spacing growing geometrically from hz_min
    at the surface z = 0 to grade*hz_min at the bottom; vertices jittered uniformly by
    +-jitter of the smaller adjacent spacing per axis (boundary vertices tangentially
    only). Surface: free (2); other sides absorbing (1)."""
    rng = np.random.default_rng(seed)
    xs = h * np.arange(nx + 1, dtype=float)
    ys = h * np.arange(ny + 1, dtype=float)
    r = grade ** (1.0 / (nz - 1)) if nz > 1 else 1.0
    hz = hz_min * r ** np.arange(nz)                 # from the surface downwards
    depth_lines = np.concatenate([[0.0], np.cumsum(hz)])
    zs = -depth_lines[::-1]                            # bottom ... 0
    xyz = _grid_vertices(xs, ys, zs)
    tet = _kuhn_tets(nx, ny, nz)
    nv = xyz.shape[0]
    vi = np.arange(nv) % (nx + 1)
    vj = (np.arange(nv) // (nx + 1)) % (ny + 1)
    vk = np.arange(nv) // ((nx + 1) * (ny + 1))
    dz_lines = np.diff(zs)                             # cell heights bottom..top
    sx = np.full(nv, h)
    sy = np.full(nv, h)
    sz = np.minimum(dz_lines[np.clip(vk - 1, 0, nz - 1)], dz_lines[np.clip(vk, 0, nz - 1)])
    free = np.stack([(vi > 0) & (vi < nx), (vj > 0) & (vj < ny), (vk > 0) & (vk < nz)], axis=1)
    spacing = np.stack([sx, sy, sz], axis=1)
    amp = jitter * np.ones(nv)
    base = xyz.copy()
    draw = rng.uniform(-1.0, 1.0, size=(nv, 3))
    for _ in range(20):
        xyz = base + draw * (amp[:, None] * spacing) * free
        x = xyz[tet]
        vol = np.einsum("ki,ki->k", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]))
        bad = vol <= 0.0
        if not np.any(bad):
            break
        amp[np.unique(tet[bad].ravel())] *= 0.5
    else:
        raise RuntimeError("could not untangle jittered mesh")
    bc = _boundary_codes(tet, nx, ny, nz, [1, 1, 1, 1, 1, 2])
    return dict(xyz=xyz, tet=tet, face_bc=bc, period=None, depth=float(depth_lines[-1]))


def centroids(mesh):
    return mesh["xyz"][mesh["tet"]].mean(axis=1)


def homogeneous(n_elem, rho=2700.0, vp=6000.0, vs=3464.0):
    return dict(rho=np.full(n_elem, rho), vp=np.full(n_elem, vp), vs=np.full(n_elem, vs))


def layered(mesh, interfaces_depth, vs_layers, rho=2700.0, qs_per_kms=None):
    """Layers by centroid depth; vp = sqrt(3) vs; optional Qs = qs_per_kms * vs[km/s], Qp = 2 Qs."""
    depth = -centroids(mesh)[:, 2]
    layer = np.searchsorted(np.asarray(interfaces_depth), depth, side="right")
    vs = np.asarray(vs_layers, dtype=float)[layer]
    out = dict(rho=np.full(len(vs), rho), vp=np.sqrt(3.0) * vs, vs=vs)
    if qs_per_kms is not None:
        out["qs"] = qs_per_kms * vs / 1000.0
        out["qp"] = 2.0 * out["qs"]
    return out


def random_layers(mesh, n_layers=8, vs_range=(500.0, 4000.0), seed=SEED_MATERIAL, qs_per_kms=50.0):
    """n_layers equally thick layers with vs ~ U(vs_range) from the seed."""
    rng = np.random.default_rng(seed)
    vs_layers = rng.uniform(vs_range[0], vs_range[1], size=n_layers)
    depth = mesh["depth"]
    interfaces = depth * np.arange(1, n_layers) / n_layers
    return layered(mesh, interfaces, vs_layers, qs_per_kms=qs_per_kms)


def p_plane_wave(rho, vp, vs, kvec, amplitude=1.0):
    """Exact P plane wave of homogeneous isotropic elasticity.

    q(x, t) = r sin(k.x - w t), w = |k| vp, n = k/|k|, velocity part r_v = n and
    stress part r_sigma = -(lam I + 2 mu n n^T)/vp (Voigt: xx yy zz xy yz xz).
    Returns fn(x (N,3), t) -> (N, 9).
    """
    k = np.asarray(kvec, dtype=float)
    n = k / np.linalg.norm(k)
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    S = -(lam * np.eye(3) + 2.0 * mu * np.outer(n, n)) / vp
    r = amplitude * np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[1, 2], S[0, 2], n[0], n[1], n[2]])
    w = np.linalg.norm(k) * vp

    def fn(x, t=0.0):
        ph = np.asarray(x) @ k - w * t
        return np.sin(ph)[:, None] * r[None, :]

    return fn


def s_plane_wave(rho, vs, kvec, pol, amplitude=1.0):
    """Exact S plane wave: velocity along unit pol (pol . k = 0), stress
    -mu (n pol^T + pol n^T)/vs, w = |k| vs."""
    k = np.asarray(kvec, dtype=float)
    n = k / np.linalg.norm(k)
    p = np.asarray(pol, dtype=float)
    p = p - (p @ n) * n
    p /= np.linalg.norm(p)
    mu = rho * vs * vs
    S = -mu * (np.outer(n, p) + np.outer(p, n)) / vs
    r = amplitude * np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[1, 2], S[0, 2], p[0], p[1], p[2]])
    w = np.linalg.norm(k) * vs

    def fn(x, t=0.0):
        ph = np.asarray(x) @ k - w * t
        return np.sin(ph)[:, None] * r[None, :]

    return fn


def gaussian_pulse(center, width, nq, amplitude=1.0, seed=3):
    """Smooth random-direction initial field exp(-|x-c|^2/w^2) * a, a ~ N(0,1)^nq."""
    rng = np.random.default_rng(seed)
    a = amplitude * rng.normal(size=nq)
    scale = np.ones(nq)
    scale[:6] = 1e6          # stresses ~ rho c |v|
    a = a * scale
    c = np.asarray(center, dtype=float)

    def fn(x, t=0.0):
        r2 = np.sum((np.asarray(x) - c) ** 2, axis=1)
        return np.exp(-r2 / width ** 2)[:, None] * a[None, :]

    return fn


def random_sources(n, box_lo, box_hi, f0_range=(1.0, 4.0), seed=SEED_SOURCES):
    """n random moment-tensor sources: positions, unit-norm symmetric tensors, f0."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(box_lo, box_hi, size=(n, 3))
    m6 = rng.normal(size=(n, 6))
    m6 /= np.linalg.norm(m6, axis=1, keepdims=True)
    f0 = rng.uniform(f0_range[0], f0_range[1], size=n)
    return pos, m6, f0


def surface_receiver_grid(nx, ny, x_range, y_range, depth=1.0, seed=SEED_RECEIVERS):
    """nx*ny receivers on a surface grid, slightly perturbed, depth metres below z = 0."""
    rng = np.random.default_rng(seed)
    gx = np.linspace(x_range[0], x_range[1], nx + 2)[1:-1]
    gy = np.linspace(y_range[0], y_range[1], ny + 2)[1:-1]
    X, Y = np.meshgrid(gx, gy, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), np.full(X.size, -depth)], axis=1)
    pts[:, :2] += rng.uniform(-1.0, 1.0, size=(X.size, 2)) * 0.01 * (x_range[1] - x_range[0]) / (nx + 1)
    return pts


_EVEN_PERMS = [p for p in itertools.permutations(range(4))
               if sum(1 for a in range(4) for b in range(a + 1, 4) if p[a] > p[b]) % 2 == 0]


def permute_vertex_order(mesh, seed=SEED_MESH):
    """Apply a random even permutation to each tetrahedron's vertex list (keeps the
    orientation positive) and carry the per-face boundary codes along, so the
    face-neighbour relations (j, h) take all their 12 values. Face i is the face
    opposite local vertex 3 - i."""
    rng = np.random.default_rng(seed)
    tet = np.asarray(mesh["tet"])
    bc = np.asarray(mesh["face_bc"])
    choice = rng.integers(0, len(_EVEN_PERMS), size=tet.shape[0])
    perms = np.array(_EVEN_PERMS)[choice]                      # (K, 4): new vertex v = old perms[v]
    new_tet = np.take_along_axis(tet, perms, axis=1)
    old_face = 3 - perms[:, ::-1]                              # new face i opposite new vertex 3-i
    new_bc = np.take_along_axis(bc, old_face, axis=1)
    out = dict(mesh)
    out["tet"] = new_tet
    out["face_bc"] = new_bc.astype(np.int32)
    return out


def random_dofs(n_elem, n_q, n_basis, seed=SEED_MATERIAL, stress_scale=1e6, decay=0.5):
    """Seeded random modal coefficients [n_elem][n_q][n_basis]: N(0,1) scaled by
    decay^(mode index / n_basis * 4) so higher modes are smaller; stress rows (and
    memory-variable rows beyond 9, which are strain-like) scaled as given."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n_elem, n_q, n_basis))
    d *= (decay ** (4.0 * np.arange(n_basis) / n_basis))[None, None, :]
    d[:, :6, :] *= stress_scale
    return d


def polynomial_field(n_q, degree, scale=1.0, seed=SEED_MATERIAL):
    """A random polynomial field of total degree <= degree in x/scale (exactly
    representable by the modal basis of order degree+1)."""
    rng = np.random.default_rng(seed)
    expo = [(a, b, c) for a in range(degree + 1) for b in range(degree + 1) for c in range(degree + 1)
            if a + b + c <= degree]
    coef = rng.normal(size=(len(expo), n_q))

    def fn(x):
        y = np.asarray(x) / scale
        out = np.zeros((len(y), n_q))
        for cf, (a, b, c) in zip(coef, expo):
            out += (y[:, 0] ** a * y[:, 1] ** b * y[:, 2] ** c)[:, None] * cf[None, :]
        return out

    return fn


def layer_over_halfspace(nx, ny, h, layer=1000.0, hz_layer=125.0, nz_below=8, grade=2.0, jitter=0.15,
                         seed=SEED_MESH):
    """Layer-over-half-space box in the spirit of the LOH.3 benchmark: vertical spacing
    hz_layer through the top `layer` metres (so an element face lies on the interface),
    then nz_below cells growing geometrically by `grade` overall; horizontal spacing h.
    Free surface at z = 0, absorbing elsewhere. Returns the mesh dict with 'depth'."""
    n_layer = int(round(layer / hz_layer))
    r = grade ** (1.0 / max(nz_below - 1, 1))
    below = hz_layer * r ** np.arange(1, nz_below + 1)
    hz = np.concatenate([np.full(n_layer, hz_layer), below])
    depth_lines = np.concatenate([[0.0], np.cumsum(hz)])
    zs = -depth_lines[::-1]
    nz = len(hz)
    rng = np.random.default_rng(seed)
    xs = h * np.arange(nx + 1, dtype=float)
    ys = h * np.arange(ny + 1, dtype=float)
    xyz = _grid_vertices(xs, ys, zs)
    tet = _kuhn_tets(nx, ny, nz)
    nv = xyz.shape[0]
    vi = np.arange(nv) % (nx + 1)
    vj = (np.arange(nv) // (nx + 1)) % (ny + 1)
    vk = np.arange(nv) // ((nx + 1) * (ny + 1))
    dz_lines = np.diff(zs)
    sz = np.minimum(dz_lines[np.clip(vk - 1, 0, nz - 1)], dz_lines[np.clip(vk, 0, nz - 1)])
    # the interface plane (and the surface / bottom) keeps its depth: no vertical jitter there
    on_interface = np.isclose(xyz[:, 2], -layer)
    free = np.stack([(vi > 0) & (vi < nx), (vj > 0) & (vj < ny), (vk > 0) & (vk < nz) & ~on_interface], axis=1)
    spacing = np.stack([np.full(nv, h), np.full(nv, h), sz], axis=1)
    amp = jitter * np.ones(nv)
    base = xyz.copy()
    draw = rng.uniform(-1.0, 1.0, size=(nv, 3))
    for _ in range(20):
        xyz = base + draw * (amp[:, None] * spacing) * free
        x = xyz[tet]
        vol = np.einsum("ki,ki->k", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]))
        bad = vol <= 0.0
        if not np.any(bad):
            break
        amp[np.unique(tet[bad].ravel())] *= 0.5
    else:
        raise RuntimeError("could not untangle jittered mesh")
    bc = _boundary_codes(tet, nx, ny, nz, [1, 1, 1, 1, 1, 2])
    return dict(xyz=xyz, tet=tet, face_bc=bc, period=None, depth=float(depth_lines[-1]))


def loh3_materials(mesh, layer=1000.0):
    """LOH.3 model parameters (Sec. VII-B): layer vs 2000, vp 4000, rho 2600, Qs 40, Qp 120;
    half-space vs 3464, vp 6000, rho 2700, Qs 69.3, Qp 155.9 (by element centroid depth)."""
    in_layer = -centroids(mesh)[:, 2] < layer
    return dict(rho=np.where(in_layer, 2600.0, 2700.0), vp=np.where(in_layer, 4000.0, 6000.0),
                vs=np.where(in_layer, 2000.0, 3464.0), qp=np.where(in_layer, 120.0, 155.9),
                qs=np.where(in_layer, 40.0, 69.3))
