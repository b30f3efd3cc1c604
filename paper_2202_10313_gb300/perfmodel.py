"""Algorithmic work of one element update in this library's formulation.

Flops count the arithmetic of the kernels on the blocks that are not structurally zero
(the hierarchical orthonormal basis makes K_c strictly block-triangular by degree and
the face matrices block-triangular; the kernels skip those zero blocks); a fused
multiply-add counts 2. Bytes count every value the kernel must move to or from HBM
once: DOFs read and written, LTS buffers written (predict) or one 9 x B buffer read
(neighbour: each element's buffer is needed once; the other three face neighbours'
re-reads are assumed to hit L2), and the per-element tables.
"""


def nbasis(o):
    return o * (o + 1) * (o + 2) // 6


def nface(o):
    return o * (o + 1) // 2


def _col_degrees(o):
    return [p for p in range(o) for _ in range((p + 1) * (p + 2) // 2)]


def flops_predict(o, m):
    """Flops of k_predict_local per element (time, volume and local surface kernels)."""
    B, F, NQ = nbasis(o), nface(o), 9 + 6 * m
    degs = _col_degrees(o)
    fdeg = [p for p in range(o) for _ in range(p + 1)]
    # time kernel, summed over the derivatives d = 0 .. o-2: column b takes the modes k of
    # degree > deg b of d^d Q; elastic: d^d Q has degree <= o-1-d, so k < nbasis(o-d)
    kend = [nbasis(o - d) if m == 0 else B for d in range(o - 1)]
    ck_gemm = 27 * sum(max(0, ke - nbasis(p + 1)) for ke in kend for p in degs)
    vol_gemm = 27 * sum(nbasis(p) for p in degs)
    star = 2 * 54 + 20                              # W_d combinations + Hooke / momentum
    ck_epi = star + m * 24 + m * 12 + 2 * (NQ + 9)  # coupling, relaxation, Taylor sums
    vol_epi = star + m * 24 + m * 12 + NQ
    surf_g, flux, surf_h = _surface(o, m)
    upd = B * (NQ + 2 * 6 * m)
    return 2 * ck_gemm + (o - 1) * B * ck_epi + 2 * vol_gemm + B * vol_epi + surf_g + flux + surf_h + upd


def _surface(o, m):
    """Face traces (9 rows x F~ or F-), closed-form interface states (v*, t*), their 6-row
    projection through F^ and the flux rows rebuilt per face and column."""
    B, F = nbasis(o), nface(o)
    degs = _col_degrees(o)
    fdeg = [p for p in range(o) for _ in range(p + 1)]
    surf_g = 2 * 9 * 4 * sum(B - nbasis(p) for p in fdeg)
    flux = 4 * F * 50
    rows = 30 + (18 if m else 0)
    surf_h = 2 * 6 * 4 * sum(nface(p + 1) for p in degs) + B * 4 * rows
    return surf_g, flux, surf_h


def flops_neighbour(o, m):
    """Flops of k_neighbour per element (neighbour surface kernel)."""
    B, NQ = nbasis(o), 9 + 6 * m
    surf_g, flux, surf_h = _surface(o, m)
    return surf_g + flux + surf_h + B * (NQ + 2 * 6 * m)


def bytes_predict(o, m, frac_finer=0.0, frac_coarser=0.0, n_fused=1):
    """HBM bytes of k_predict_local per element and simulation; frac_* are the shares of
    elements that also write B2 (a finer neighbour) or B3 (a coarser one); the
    per-element tables are shared by the n_fused simulations."""
    B, NQ = nbasis(o), 9 + 6 * m
    buf = 4 * 9 * B
    return 4 * 2 * NQ * B + buf * (1.0 + frac_finer + 1.5 * frac_coarser) + (4 * 64 + 4) / n_fused


def bytes_neighbour(o, m, n_fused=1):
    """HBM bytes of k_neighbour per element and simulation."""
    B, NQ = nbasis(o), 9 + 6 * m
    return 4 * 2 * NQ * B + 4 * 9 * B + (4 * 48 + 4 * 9) / n_fused


def paper_flops_per_update():
    """Sec. VII-B: 529,110 flops per element update (O=5, m=3, one simulation, block-sparse)."""
    return 529110


def operator_nonzeros(order, rel=1e-9):
    """Nonzeros of the reference operators the kernels contract with (K_c, F~_i, F-_{j,h}),
    counted from the library's own FP64 operators (host-side, no device); entries below
    rel times the largest are the rounding of exact zeros."""
    import numpy as np
    from . import binding
    K, Ft, Fb = binding.reference_operators(order)
    nz = lambda a: int(np.sum(np.abs(a) > rel * np.abs(a).max()))
    return dict(K=[nz(K[c]) for c in range(3)], Ft=[nz(Ft[i]) for i in range(4)],
                Fb=[[nz(Fb[j, h]) for h in range(3)] for j in range(4)])


def sparse_terms(order):
    """Multiply-adds per row of the generated sparse products (the nonzero entries of the
    library's FP64 operators, entries below 1e-7 of the largest being rounding of exact
    zeros): time kernel per derivative variant v (elastic truncation; v = 0 full), volume,
    face traces (= face projection, F^_i = F~_i^T)."""
    import numpy as np
    from . import binding
    K, Ft, _ = binding.reference_operators(order)
    kz = np.abs(K) > 1e-7 * np.abs(K).max()
    fz = np.abs(Ft) > 1e-7 * np.abs(Ft).max()
    time = [int(sum(kz[c][:nbasis(order - 1 - v), :nbasis(order - v)].sum() for c in range(3)))
            for v in range(order - 1)]
    return dict(time=time, vol=int(kz.sum()), face=int(fz.sum()))


def flops_predict_sparse(o, m):
    """Flops of k_predict_sp per element: the generated sparse products (time kernel, volume,
    face traces and face projection: nonzero operator entries only, Sec. IV-A "all
    sparsity"), the star / relaxation / Taylor arithmetic of the column phase, the
    interface states and flux rows, and the update."""
    B, F, NQ = nbasis(o), nface(o), 9 + 6 * m
    t = sparse_terms(o)
    time = sum(2 * 9 * t["time"][d if m == 0 else 0] for d in range(o - 1))
    star = 2 * 54 + 20
    ck_epi = star + m * 24 + m * 12 + 2 * (NQ + 9)
    vol_epi = star + m * 24 + m * 12 + NQ
    rows = 30 + (18 if m else 0)
    return (time + (o - 1) * B * ck_epi + 2 * 9 * t["vol"] + B * vol_epi + 2 * 9 * t["face"] + 4 * F * 50
            + 2 * 6 * t["face"] + B * 4 * rows + B * (NQ + 2 * 6 * m))


def flops_neighbour_sparse(o, m):
    """Flops of k_neighbour_sp per element: the traces X F~_j of the four neighbours' buffers on
    their faces j (nonzero entries; each face of the reference element equally likely, so the
    four faces together cost the nonzeros of all four F~), the orientation maps R_h (degree
    blocks), the interface states, the generated F^ projection, flux rows and update."""
    B, F, NQ = nbasis(o), nface(o), 9 + 6 * m
    t = sparse_terms(o)
    rh = sum((p + 1) ** 2 for p in range(o))          # terms of one R_h per face row
    rows = 30 + (18 if m else 0)
    return (2 * 9 * t["face"] + 2 * 9 * 4 * rh + 4 * F * 50 + 2 * 6 * t["face"] + B * 4 * rows
            + B * (NQ + 2 * 6 * m))


def essential_flops(order, m):
    """Flops of one element update if only the true nonzeros of K_c, F~ and F- were
    multiplied (the kernels multiply whole degree blocks: flops_predict + flops_neighbour);
    the star, flux and Taylor arithmetic is counted as in the block model."""
    import numpy as np
    from . import binding
    nzs = operator_nonzeros(order)
    B, F, NQ = nbasis(order), nface(order), 9 + 6 * m
    K = binding.reference_operators(order)[0]
    nzk = lambda a: int(np.sum(np.abs(a) > 1e-9 * np.abs(K).max()))
    # one derivative: 3 products of 9 rows; elastic: only the modes k < nbasis(order-d) of d^d Q
    ck = sum(2 * 9 * sum(nzk(K[c][:, :(nbasis(order - d) if m == 0 else B)]) for c in range(3))
             for d in range(order - 1))
    vol = 2 * 9 * sum(nzs["K"])
    face_g = 2 * 9 * sum(nzs["Ft"])
    face_h = 2 * 6 * sum(nzs["Ft"])                # F^ = F~^T
    nbr_g = 2 * 9 * sum(nzs["Fb"][0]) / 3.0 * 4    # one F- per face
    degs = _col_degrees(order)
    star = 2 * 54 + 20
    epi = (order - 1) * B * (star + m * 36 + 2 * (NQ + 9)) + B * (star + m * 36 + NQ)
    flux = 2 * 4 * F * 50 + 2 * B * 4 * (30 + (18 if m else 0))
    upd = 2 * B * (NQ + 12 * m)
    return ck + vol + face_g + face_h + nbr_g + face_h + epi + flux + upd
