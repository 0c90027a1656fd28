"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU
and exports every function declared in include/laph.h."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "laph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|long|char)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_path():
    names = declared_functions()
    for n in ["laph_eigvecs", "laph_make_sources", "dirac_solve_batch", "laph_sinks", "correlate",
              "laph_stout_smear", "laph_ctx_create", "laph_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import ctypes
    from paper_1104_3870_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_reports_version():
    from paper_1104_3870_gb300 import laph
    assert "sm_103a" in laph.version()
    assert laph.laph_launch_count() >= 0
