"""CPU checks of the C ABI library: it builds, loads and exports every declared symbol."""
import ctypes

import pytest

from paper_2202_10313_gb300 import binding, build


@pytest.fixture(scope="module")
def built():
    return build.build()


def test_library_exports_every_declared_function(built):
    names = binding.header_functions()
    assert len(names) >= 20
    L = ctypes.CDLL(built)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding declares a signature for each of them
    assert sorted(binding._SIGS) == names


def test_argument_errors_without_gpu(built):
    L = binding.lib()
    h = ctypes.c_void_p()
    assert L.lts_create(7, 0, 1, 0, ctypes.byref(h)) == binding.LTS_ERR_ARG
    assert L.lts_create(5, 2, 1, 0, ctypes.byref(h)) == binding.LTS_ERR_ARG
    for bad_fused in (0, 3, 6, 68):
        assert L.lts_create(5, 3, bad_fused, 0, ctypes.byref(h)) == binding.LTS_ERR_ARG
    assert not h
    L.lts_destroy(None)
