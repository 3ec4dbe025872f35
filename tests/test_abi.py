"""The C-ABI library builds for sm_103a, loads, and exports every call that
include/pd.h declares (no compute: this runs without a GPU)."""
import ctypes
import os
import re

from paper_2510_23679_gb300 import _build, pd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(pd_[a-z0-9_]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("pd_build_profiles", "pd_best_hits", "pd_bbh", "pd_best_hits_all", "pd_bbh_all",
                 "pd_summin_pairs", "pd_ctx_create", "pd_choose_k"):
        assert core in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_every_declared_symbol():
    assert sorted(pd.EXPORTED) == declared_functions()


def test_choose_k_without_gpu():
    pd.load()
    assert pd.pd_choose_k(348042) == 5       # 20^4 < 348042 <= 20^5
    assert pd.pd_choose_k(50_000_000) == 6
    assert pd.pd_choose_k(20 ** 7) == 7
    assert pd.pd_choose_k(1) == 1


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No fallback: without the compiled library the binding raises."""
    import pytest
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "absent.so"))
    saved = pd._lib
    try:
        pd._lib = None
        with pytest.raises(RuntimeError, match="not found"):
            pd.load(build=False)
    finally:
        pd._lib = saved


def test_product_sources_do_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2510_23679_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "pd_oracle" not in text, f
