"""The C-ABI library loads and exports every function include/*.h declares.

No compute call is made: these run without a GPU.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"\b(lnv_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def so():
    from paper_0911_3584_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("lnv_pattern_build", "lnv_plan_product", "lnv_bsr_multiply",
                 "lnv_trace_product", "lnv_system_create", "lnv_energy_grad"):
        assert must in names


def test_library_exports_every_declared_symbol(so):
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing


def test_version_and_error_string_without_gpu(so):
    so.lnv_version.restype = ctypes.c_char_p
    so.lnv_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in so.lnv_version()
    assert isinstance(so.lnv_last_error(), bytes)


def test_null_arguments_are_rejected_without_gpu(so):
    """Argument checks run before any device work and return LNV_ERR_ARG."""
    so.lnv_plan_info.restype = ctypes.c_int
    assert so.lnv_plan_info(None, None, None) == -1
    so.lnv_pattern_info.restype = ctypes.c_int
    assert so.lnv_pattern_info(None, None, None, None, None, None, None) == -1
    so.lnv_system_workspace_size.restype = ctypes.c_int
    assert so.lnv_system_workspace_size(None, 1, None) == -1


def test_binding_fails_loudly_when_library_missing(monkeypatch, tmp_path):
    import paper_0911_3584_gb300.lnv as lnv
    monkeypatch.setattr(lnv._build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(lnv, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        lnv.lib()
