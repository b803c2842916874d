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


def test_entry_points_reject_missing_arguments_before_touching_the_device(lib):
    """Host-detectable errors return MS_ERR_INVALID_ARG at once (the header's
    contract): a NULL context, column, output or buffer.  None of these calls
    reaches CUDA, so they run here without a GPU."""
    L = morphstore.load()
    bad = morphstore.MS_ERR_INVALID_ARG
    out = ctypes.c_void_p()
    po = ctypes.byref(out)
    u64 = ctypes.c_uint64()
    i32 = ctypes.c_int()
    meta = morphstore.ColumnMeta()
    cfg = morphstore.BatchConfig(8, 2, 32, 0, 0, 1)
    fake = ctypes.c_void_p(16)  # a non-NULL device pointer that is never dereferenced
    calls = {
        "ms_ctx_create(out=NULL)": lambda: L.ms_ctx_create(None, 0, 1 << 20, 1 << 20, morphstore._ALLOC_FN(0),
                                                            morphstore._FREE_FN(0), None),
        "ms_ctx_destroy": lambda: L.ms_ctx_destroy(None),
        "ms_get_error": lambda: L.ms_get_error(None, None),
        "ms_arena_usage": lambda: L.ms_arena_usage(None, ctypes.byref(u64), ctypes.byref(u64), None),
        "ms_arena_reset_high_water": lambda: L.ms_arena_reset_high_water(None, None),
        "ms_column_import": lambda: L.ms_column_import(None, morphstore.DYN_BP, 0, 1, fake, 8, po, None),
        "ms_column_export": lambda: L.ms_column_export(None, fake, fake, 8, ctypes.byref(u64), None),
        "ms_column_info": lambda: L.ms_column_info(None, fake, ctypes.byref(meta), None),
        "ms_column_free": lambda: L.ms_column_free(None, fake, None),
        "ms_compress": lambda: L.ms_compress(None, fake, 1, morphstore.DYN_BP, 0, po, None),
        "ms_decompress": lambda: L.ms_decompress(None, fake, fake, 1, None),
        "ms_select": lambda: L.ms_select(None, fake, morphstore.LT, 1, 0, morphstore.DELTA_BP, 0, po, None),
        "ms_project": lambda: L.ms_project(None, fake, fake, morphstore.DYN_BP, 0, po, None),
        "ms_calc": lambda: L.ms_calc(None, morphstore.ADD, fake, None, 1, morphstore.DYN_BP, 0, po, None),
        "ms_agg_sum": lambda: L.ms_agg_sum(None, fake, fake, None),
        "ms_group_sum": lambda: L.ms_group_sum(None, fake, fake, 4, fake, None),
        "ms_semijoin": lambda: L.ms_semijoin(None, fake, fake, 8, morphstore.DELTA_BP, 0, po, None),
        "ms_column_stats": lambda: L.ms_column_stats(None, fake, fake, None),
        "ms_compress_noalloc(out=NULL)": lambda: L.ms_compress_noalloc(fake, 1, morphstore.DYN_BP, 0, None, 64,
                                                                        fake, None),
        "ms_compress_noalloc(static width 0)": lambda: L.ms_compress_noalloc(fake, 1, morphstore.STATIC_BP, 0, fake,
                                                                              64, fake, None),
        "ms_mlp_forward": lambda: L.ms_mlp_forward(None, fake, 1, fake, None),
        "ms_mlp_adam(step 0)": lambda: L.ms_mlp_adam(fake, fake, fake, fake, 0, 1e-3, 0.9, 0.999, 1e-8, None),
        "ms_batch_create": lambda: L.ms_batch_create(None, 1, fake, fake, fake, fake, fake, po, None),
        "ms_batch_info": lambda: L.ms_batch_info(None, ctypes.byref(u64), ctypes.byref(u64), ctypes.byref(u64)),
        "ms_batch_run": lambda: L.ms_batch_run(None, 0, 1, ctypes.byref(cfg), 0, fake, None),
        "ms_batch_graph": lambda: L.ms_batch_graph(None, 0, 1, ctypes.byref(cfg), 0, fake, po),
        "ms_graph_launch": lambda: L.ms_graph_launch(None, None),
        "ms_graph_destroy": lambda: L.ms_graph_destroy(None),
        "ms_batch_destroy": lambda: L.ms_batch_destroy(None),
        "ms_selftest_wait_timeout": lambda: L.ms_selftest_wait_timeout(None, None),
        "ms_profile_enable": lambda: L.ms_profile_enable(None, 1),
        "ms_profile_collect": lambda: L.ms_profile_collect(None, None, 0, ctypes.byref(i32)),
    }
    got = {name: call() for name, call in calls.items()}
    assert all(v == bad for v in got.values()), {k: v for k, v in got.items() if v != bad}


def _header_enum(name_prefix):
    """name -> value of the header's enumerators with the given prefix."""
    import re
    text = open(morphstore._HEADER).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(" + name_prefix + r"[A-Z0-9_]+)\s*=\s*(\d+)", text)}


def test_binding_format_and_kernel_ids_match_the_header():
    fm = _header_enum("MS_")
    for name in ("UNCOMPR", "STATIC_BP", "DYN_BP", "DELTA_BP", "FOR_BP", "RLE", "FOR_STATIC_BP", "DELTA_STATIC_BP"):
        assert getattr(morphstore, name) == fm["MS_" + name], name
        assert morphstore.FORMAT_NAMES[fm["MS_" + name]] == name.lower()
    ks = _header_enum("MS_K_")
    assert ks["MS_K_RLE"] == ks["MS_K_COUNT"] - 1


def test_oracle_and_binding_share_the_format_numbering():
    """The oracle numbers the formats from the same written definitions (it imports
    nothing from the library); both sides must agree so that the parity tests compare
    like with like."""
    import oracle
    for name in ("UNCOMPR", "STATIC_BP", "DYN_BP", "DELTA_BP", "FOR_BP", "RLE", "FOR_STATIC_BP", "DELTA_STATIC_BP"):
        assert getattr(oracle, name) == getattr(morphstore, name), name
