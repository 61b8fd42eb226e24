"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/pds.h declares (no GPU needed: no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2109_08815_gb300 import build as pbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pds.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pds_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib_path = pbuild.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2109_08815_gb300 import api
    assert set(_declared()) == set(api.EXPORTS)


def test_status_strings_without_gpu():
    lib = ctypes.CDLL(pbuild.build())
    lib.pds_strerror.restype = ctypes.c_char_p
    assert lib.pds_strerror(0) == b"ok"
    assert lib.pds_strerror(-1) == b"invalid argument"
    assert lib.pds_strerror(-4) == b"non-finite value"
    assert lib.pds_strerror(-5) == b"device wait timed out"


def test_create_rejects_null_without_touching_the_gpu():
    lib = ctypes.CDLL(pbuild.build())
    out = ctypes.c_void_p()
    rc = lib.pds_problem_create(None, ctypes.c_double(0.01), 10, 2, None, 1, None, ctypes.c_double(0.1),
                                ctypes.c_double(0.1), None, None, None, ctypes.c_double(0.0), None,
                                ctypes.byref(out))
    assert rc == -1 and not out.value


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2109_08815_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.replace("the oracle", "").lower() or f == "workloads.py", f


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    """No CPU fallback: a missing libpds.so is an error, not a slower path."""
    from paper_2109_08815_gb300 import api
    monkeypatch.setattr(api, "_lib", None)
    monkeypatch.setattr(api, "LIB_PATH", str(tmp_path / "libpds.so"))
    with pytest.raises(api.PdsError, match="missing"):
        api.lib()
