"""Host-side checks of the C ABI (no GPU needed, no compute calls): the
library builds, loads, exports every entry point the public header
declares, the Python binding wraps each of them under the same name, and
argument errors are reported as status codes before any device work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gko_gb300.h")


@pytest.fixture(scope="module")
def gko():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2011_08879_gb300 as g
    return g


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(gko_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("gko_spmv", "gko_convert", "gko_cg", "gko_cg_mixed", "gko_cg_batched", "gko_matrix_create_csr",
                 "gko_features", "gko_mlp_grad", "gko_select_format"):
        assert must in names


def test_every_declared_symbol_is_exported(gko):
    lib = C.CDLL(gko.binding.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_symbol_with_the_same_name(gko):
    missing = [n for n in declared_functions() if not hasattr(gko.binding, n) and n not in
               ("gko_last_error", "gko_status_string")]
    assert not missing, missing
    assert set(declared_functions()) == set(gko.binding._SIGS)


def test_header_macros_match_the_binding(gko):
    text = open(HEADER).read()
    macros = dict(re.findall(r"#define\s+(GKO_[A-Z0-9_]+)\s+(0x[0-9A-Fa-f]+|\d+)", text))
    b = gko.binding
    assert int(macros["GKO_BATCH_SHARED_P"], 0) == b.BATCH_SHARED_P
    assert int(macros["GKO_BATCH_SHARED_PQ"], 0) == b.BATCH_SHARED_PQ
    # the flags sit above every block size
    assert b.BATCH_SHARED_P > 1024 and b.BATCH_SHARED_P & b.BATCH_SHARED_PQ == 0
    assert b.batch_layout(b.BATCH_SHARED_P | 128) == "shared_p/128"
    assert b.batch_layout(b.BATCH_SHARED_PQ | 64) == "shared_pq/64"
    assert b.batch_layout(-256) == "registers/256" and b.batch_layout(64) == "shared_xrpq/64"
    for code in (0, 64, 1024, -128, b.BATCH_SHARED_P | 32, b.BATCH_SHARED_PQ | 256):
        assert b.batch_layout_code(b.batch_layout(code)) == code
    with pytest.raises(ValueError):
        b.batch_layout_code("shared_q/64")


def test_status_strings_and_version(gko):
    assert gko.binding.status_name(0) == "GKO_OK"
    assert gko.binding.status_name(7) == "GKO_ERR_BREAKDOWN"
    assert gko.binding.status_name(99) == "GKO_ERR_UNKNOWN"
    assert "sm_103a" in gko.gko_version()


def test_argument_errors_before_device_work(gko):
    b = gko.binding
    lib = b.lib
    assert lib.gko_matrix_destroy(None) == b.OK
    assert lib.gko_batch_destroy(None) == b.OK
    assert lib.gko_spmv(0, None, None, None, 1.0, 0.0, None) == b.ERR_INVALID_ARG
    assert "NULL" in b.last_error()
    out = C.c_void_p()
    assert lib.gko_matrix_create_csr(-1, 1, 0, None, None, None, 0, None, C.byref(out)) == b.ERR_INVALID_ARG
    assert lib.gko_matrix_create_csr(1, 1, 0, None, None, None, 0, None, None) == b.ERR_INVALID_ARG
    assert lib.gko_mlp_param_count(0) == -1
    assert lib.gko_mlp_param_count(8) == 64 * 12 + 64 + 64 * 64 + 64 + 8 * 64 + 8
    assert lib.gko_cg(None, 0, None, None, 1e-10, 10, None, None) == b.ERR_INVALID_ARG
    assert lib.gko_selector_load(None, 8, None, None, None, None) == b.ERR_INVALID_ARG
    with pytest.raises(b.GkoError) as e:
        b.gko_spmv(0, None, None, None)
    assert e.value.status == b.ERR_INVALID_ARG


def test_product_path_does_not_import_the_oracle():
    """The library package and its binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_2011_08879_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f
