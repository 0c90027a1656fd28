"""The product path has no CPU fallback: with the CUDA library absent, importing the
binding raises instead of computing anything elsewhere."""
import importlib
import sys

import pytest


def test_binding_refuses_to_import_without_the_library(monkeypatch, tmp_path):
    import paper_1104_3870_gb300.build as build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "liblaph.so"))
    saved = sys.modules.pop("paper_1104_3870_gb300.laph", None)
    try:
        with pytest.raises(ImportError, match="is not built"):
            importlib.import_module("paper_1104_3870_gb300.laph")
    finally:
        sys.modules.pop("paper_1104_3870_gb300.laph", None)
        if saved is not None:
            sys.modules["paper_1104_3870_gb300.laph"] = saved


def test_package_imports_nothing_from_the_oracle():
    """The oracle is test infrastructure: no module of the package imports it."""
    import pathlib
    root = pathlib.Path(__file__).resolve().parents[1] / "paper_1104_3870_gb300"
    for py in root.rglob("*.py"):
        text = py.read_text()
        assert "import oracle" not in text and "from oracle" not in text, py
