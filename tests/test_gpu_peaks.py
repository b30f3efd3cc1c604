"""Throughput probes behind the measured roofline denominators: FP32 FMA on the CUDA cores and
tcgen05 tf32 MMA on the tensor cores, both within physical limits for a 152-SM part."""
import math

import pytest

from paper_2202_10313_gb300 import binding, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def test_peak_probes():
    s = binding.Solver(3, 0, device=0)
    p = s.measure_peaks()
    s.close()
    assert all(math.isfinite(v) and v > 0 for v in p.values())
    # FP32: at most 152 SMs x 128 lanes x 2 flops at 2.2 GHz
    assert 10.0 < p["fp32_tflops"] < 152 * 128 * 2 * 2.2e9 / 1e12
    assert p["tf32_tflops"] > p["fp32_tflops"]
