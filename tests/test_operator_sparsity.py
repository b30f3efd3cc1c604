"""The block sparsity the kernels skip is exact: with the hierarchical orthonormal basis
(Sec. III-A, ordered by degree) K_c[i][j] = int phi_i d_c phi_j vanishes unless
deg i < deg j, and the face traces F~_i[k][f], F-_{j,h}[k][f] vanish unless deg f <= deg k.
Checked on the library's operators (host code) and, independently, on the oracle's. The
library builds them by exact monomial integration in FP64, whose cancellation leaves
entries of ~1e-13 of the largest in blocks that are zero in exact arithmetic; the bound
and the nonzero threshold sit well above that and far below any true entry."""
import numpy as np
import pytest

from oracle.basis import Basis
from paper_2202_10313_gb300 import binding, perfmodel


def _deg_vol(o):
    return np.array([p for p in range(o) for _ in range((p + 1) * (p + 2) // 2)])


def _deg_face(o):
    return np.array([p for p in range(o) for _ in range(p + 1)])


@pytest.mark.parametrize("order", [3, 4, 5])
def test_skipped_blocks_are_exact_zeros_and_counts_agree_with_the_oracle(order):
    K, Ft, Fb = binding.reference_operators(order)
    dv, df = _deg_vol(order), _deg_face(order)
    skip_k = dv[:, None] >= dv[None, :]
    skip_f = dv[:, None] < df[None, :]
    for c in range(3):
        assert np.abs(K[c][skip_k]).max() <= 1e-10 * np.abs(K[c]).max()
    for i in range(4):
        assert np.abs(Ft[i][skip_f]).max() <= 1e-10 * np.abs(Ft[i]).max()
    for j in range(4):
        for h in range(3):
            assert np.abs(Fb[j, h][skip_f]).max() <= 1e-10 * np.abs(Fb[j, h]).max()
    ob = Basis(order)
    nz = perfmodel.operator_nonzeros(order)
    onz = lambda a: int(np.sum(np.abs(a) > 1e-9 * np.abs(a).max()))
    assert nz["K"] == [onz(ob.K[c]) for c in range(3)]
    assert nz["Ft"] == [onz(ob.Ft[i]) for i in range(4)]
    # the block model the kernels execute covers every nonzero
    assert sum(nz["K"]) <= 3 * int(np.sum(~skip_k))


def test_essential_flops_below_block_flops():
    for order, m in ((4, 0), (5, 0), (5, 3)):
        ess = perfmodel.essential_flops(order, m)
        blk = perfmodel.flops_predict(order, m) + perfmodel.flops_neighbour(order, m)
        assert 0 < ess < blk
