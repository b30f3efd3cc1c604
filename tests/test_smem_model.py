"""The shared-memory wavefront model behind the kernels' load layouts: its per-load rules
on hand-countable cases, and the orderings the layout choices rest on."""
from paper_2202_10313_gb300 import smem_model as sm


def test_wavefront_rules():
    lanes = range(32)
    # one address for the whole warp: one wavefront per phase
    assert sm.wavefronts([(l, 0) for l in lanes], 1) == 1
    assert sm.wavefronts([(l, 0) for l in lanes], 2) == 2
    assert sm.wavefronts([(l, 0) for l in lanes], 4) == 4
    # 32 consecutive floats: one wavefront; stride 2: two-way conflict; stride 32: 32-way
    assert sm.wavefronts([(l, l) for l in lanes], 1) == 1
    assert sm.wavefronts([(l, 2 * l) for l in lanes], 1) == 2
    assert sm.wavefronts([(l, 32 * l) for l in lanes], 1) == 32
    # 16-byte loads of 32 consecutive chunks: four conflict-free phases; odd chunk stride too
    assert sm.wavefronts([(l, 4 * l) for l in lanes], 4) == 4
    assert sm.wavefronts([(l, 12 * l) for l in lanes], 4) == 4
    # chunk stride 2 (8 floats): two of the 8 lanes of a phase share a bank group
    assert sm.wavefronts([(l, 8 * l) for l in lanes], 4) == 8
    # only the phases with active lanes count
    assert sm.wavefronts([(0, 0)], 4) == 1


def test_layout_choices_lower_the_modelled_wavefronts():
    old = sm.predict_model(5, k_layout="interleaved", surface="single")
    paired = sm.predict_model(5, k_layout="interleaved", surface="pairs")
    now = sm.predict_model(5, k_layout="planes", surface="pairs")
    assert paired["local_surface"] < 0.7 * old["local_surface"]
    assert now["time"] < 0.9 * paired["time"] and now["volume"] < 0.85 * paired["volume"]
    assert now["total"] < paired["total"] < old["total"]
    # the elastic truncation removes most of the time-kernel products
    el = sm.predict_model(5, elastic=True)
    assert el["time"] < 0.5 * now["time"]
    # neighbour rows: 8-byte loads (stride 10) against 4-byte loads (stride 9)
    assert sm.neighbour_product_model(5, xr=10) > 0 and sm.neighbour_product_model(5, xr=9) > 0
