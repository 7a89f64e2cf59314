"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "fr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:fr_status|const char\*)\s+(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ("fr_residual", "fr_jvp", "fr_vjp", "gmres_solve", "esdirk_stage",
              "spectral_decay_indicator", "p_rebucket", "fr_create", "fr_destroy", "fr_pack", "fr_unpack"):
        assert n in names


def test_library_builds_loads_and_exports_all_symbols():
    from paper_1910_03693_gb300 import build as B
    lib_path = B.build()
    from paper_1910_03693_gb300 import _lib
    lib = _lib.load(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) <= set(_lib.SIGNATURES) | {"fr_last_error"}


def test_missing_library_fails_loudly(tmp_path):
    from paper_1910_03693_gb300 import _lib
    with pytest.raises(ImportError):
        _lib.load(str(tmp_path / "nope.so"))
