"""The C-ABI library loads and exports every entry point include/fcm.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fcm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fcm_[A-Za-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("fcm_setup", "fcm_precond_build", "fcm_pcg_solve", "fcm_apply_K", "fcm_apply_S", "fcm_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_1809_00828_gb300 import build, fcm
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(fcm.EXPORTED) == set(_declared())


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1809_00828_gb300 import fcm
    saved = fcm._lib
    fcm._lib = None
    try:
        with pytest.raises(RuntimeError):
            fcm.load(str(tmp_path / "missing.so"))
    finally:
        fcm._lib = saved
