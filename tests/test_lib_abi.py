"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every
function that include/morphstore.h declares (no compute calls: no GPU here)."""
import ctypes
import shutil

import pytest

from paper_2004_09350_gb300 import morphstore


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not __import__("os").path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2004_09350_gb300 import _build
    _build.build()
    return ctypes.CDLL(morphstore.library_path())


def test_header_declares_the_operator_set():
    names = morphstore.header_symbols()
    for op in ("ms_compress", "ms_decompress", "ms_select", "ms_project", "ms_calc", "ms_agg_sum",
               "ms_group_sum", "ms_semijoin", "ms_ctx_create", "ms_get_error", "ms_column_import"):
        assert op in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in morphstore.header_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_the_library(lib):
    assert morphstore.load() is not None
