"""CPU checks of the boundary: the C-ABI library builds for sm_103a, loads
without a GPU, and exports every entry point that include/timest.h declares
(no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "timest.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tm_[a-z0-9_]+)\s*\(", text)) - {"tm_alloc_fn", "tm_free_fn"})


@pytest.fixture(scope="module")
def libpath():
    from paper_2507_20441_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tm_create", "tm_graph_load", "tm_preprocess", "tm_set_motif", "tm_weights", "tm_sample",
                     "tm_batch_run", "tm_destroy", "tm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_names_match_the_abi(libpath):
    import paper_2507_20441_gb300 as tg
    for n in declared_functions():
        if n in ("tm_config_default",):
            continue
        assert hasattr(tg, n), f"binding lacks {n}"


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2507_20441_gb300 as tg
    monkeypatch.setattr(tg, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(tg, "_lib", None)
    with pytest.raises(tg.TimestUnavailable):
        tg.lib()


def test_no_oracle_import_in_product():
    pkg = os.path.join(ROOT, "paper_2507_20441_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "timest_oracle" not in text, f
