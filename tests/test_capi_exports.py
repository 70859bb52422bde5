"""The C-ABI library builds, loads without a GPU, and exports every function
that include/*.h declares (no compute calls: this runs on CPU-only hosts)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(msort_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2211_16479_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("msort_sort", "msort_sort_pairs", "msort_segmented_sort", "msort_ctx_create",
                     "msort_ctx_destroy", "msort_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_the_header(lib_path):
    import paper_2211_16479_gb300 as ms
    assert set(_declared()) <= set(ms.exported_symbols())
    for n in _declared():
        assert callable(getattr(ms, n))


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_2211_16479_gb300 as ms
    saved = ms._lib
    try:
        ms._lib = None
        with pytest.raises(ImportError):
            ms.load_library(str(tmp_path / "missing.so"))
    finally:
        ms._lib = saved
