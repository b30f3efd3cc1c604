"""The generated sparse products of the predict kernel (contraction engine 'sparse') take
exactly the nonzero entries of the stiffness matrices K_c and of the face matrices F~_i
and of their transposes F^_i (Sec. III-A), and so do the products of the adjoint's reverse
predict pass, with values equal to the oracle's independently
built operators to FP32 rounding, and no term the oracle has is dropped. The generator lists every product term
(kind, part, output, k, value) it writes into the kernel."""
import os
import subprocess

import numpy as np
import pytest

from oracle.basis import Basis
from paper_2202_10313_gb300 import build


def _terms(order):
    build.build()
    exe = os.path.join(build.OUT_DIR, "gen_sparse")
    out = subprocess.run([exe, "--list", str(order)], capture_output=True, text=True, check=True).stdout
    rows = [l.split() for l in out.splitlines() if l.strip()]
    return [(r[0], int(r[1]), int(r[2]), int(r[3]), float(r[4])) for r in rows]


@pytest.mark.parametrize("order", [3, 4, 5])
def test_generated_terms_are_the_oracle_operators_nonzeros(order):
    ob = Basis(order)
    B = len(ob.K[0])
    F = ob.Ft[0].shape[1]
    terms = _terms(order)
    kmax = max(np.abs(k).max() for k in ob.K)
    fmax = max(np.abs(f).max() for f in ob.Ft)
    # the dense matrix each kind of product applies: time X K_c^T (out (c, b), sum over k of
    # K_c[b][k]); volume X K_c (K_c[k][b]); face traces X F~_i (F~_i[k][f])
    want = {"t": np.stack([ob.K[c] for c in range(3)]).reshape(3 * B, B),
            "v": np.stack([ob.K[c].T for c in range(3)]).reshape(3 * B, B),
            "g": np.stack([ob.Ft[i].T for i in range(4)]).reshape(4 * F, B)}
    # face projection: out (i, b) from the inputs (i, f), F^_i[f][b] = int psi_f phi_b = F~_i[b][f]
    proj = np.zeros((4 * B, 4 * F))
    for i in range(4):
        proj[i * B:(i + 1) * B, i * F:(i + 1) * F] = ob.Fh[i].T
    want["p"] = proj
    want["n"] = np.stack([ob.Ft[j].T for j in range(4)]).reshape(4 * F, B)
    # adjoint products: the four faces' transposed traces summed, out b from the inputs
    # (i, f), F~_i[b][f]; the reverse time kernel X K_c (as the volume kernel)
    want["s"] = np.concatenate([ob.Ft[i] for i in range(4)], axis=1)
    want["k"] = want["v"]
    scale = {"t": kmax, "v": kmax, "g": fmax, "p": fmax, "n": fmax, "s": fmax, "k": kmax}
    got = {k: np.zeros_like(v) for k, v in want.items()}
    part_of = {}
    for kind, part, o, k, val in terms:
        assert got[kind][o, k] == 0.0, "term listed twice"
        got[kind][o, k] = val
        assert part_of.setdefault((kind, o), part) == part, "output split over parts"
    for kind in want:
        w, g = want[kind], got[kind]
        if kind == "t":       # the kernel's full time variant writes outputs of degree <= O-2
            w = w.copy()
            nb1 = (order - 1) * order * (order + 1) // 6
            for c in range(3):
                assert np.abs(w[c * B + nb1:(c + 1) * B]).max() <= 1e-10 * scale[kind]
        # every nonzero of the oracle's operator is a term, within FP32 rounding of its value
        assert np.abs(g - w).max() <= 1e-6 * scale[kind], kind
        kept = g != 0.0
        assert np.all(np.abs(w[~kept]) <= 1e-10 * scale[kind]), kind
        assert np.all(np.abs(w[kept]) >= 1e-4 * scale[kind]), kind
    # multiply-adds per row, the paper's "all sparsity" count for these operators
    nk = sum(int(np.sum(np.abs(ob.K[c]) > 1e-9 * kmax)) for c in range(3))
    assert sum(1 for t in terms if t[0] == "t") == nk
    assert sum(1 for t in terms if t[0] == "v") == nk
    assert sum(1 for t in terms if t[0] == "k") == nk
