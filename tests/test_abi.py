"""The C ABI library loads and exports every entry point include/imm.h
declares; the binding refuses to run without it.  No GPU needed."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^\s*(?:int|void|const char\*)\s+(imm_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2411_09473_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("imm_create", "imm_load_graph", "imm_sample", "imm_select", "imm_run", "imm_destroy",
                 "imm_get_set", "imm_get_counts", "imm_reset_sets", "imm_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_null_handles_are_rejected(lib):
    lib.imm_last_error.restype = ctypes.c_char_p
    lib.imm_last_error.argtypes = [ctypes.c_void_p]
    assert lib.imm_last_error(None) == b"null context"
    lib.imm_destroy.argtypes = [ctypes.c_void_p]
    lib.imm_destroy(None)
    lib.imm_sample.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
    assert lib.imm_sample(None, 0, 10, 1) == 1  # IMM_EINVAL
    lib.imm_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.imm_create(None, 0, None, None) == 1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2411_09473_gb300 import _build, imm
    monkeypatch.setattr(_build, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(imm, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        imm._load()


def test_product_package_does_not_import_oracle():
    # the product path never routes through the oracle
    pkg = os.path.join(ROOT, "paper_2411_09473_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "oracle.c" not in text, fn


def test_bounds_checked_variant_exports_every_symbol():
    from paper_2411_09473_gb300 import _build
    plain = ctypes.CDLL(_build.build())
    checked = ctypes.CDLL(_build.build(variant="bounds"))
    missing = [n for n in _declared() if not hasattr(checked, n)]
    assert not missing, missing
    assert plain.imm_build_flags() == 0 and checked.imm_build_flags() == 1
