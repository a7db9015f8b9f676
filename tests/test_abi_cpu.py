"""Host-side checks of the C ABI (no GPU): the shared library loads and
exports every function include/pressure_projection.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pressure_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_the_boundary():
    assert {"pressure_plan_create", "pressure_solve", "pressure_correct",
            "pressure_solve_adjoint"} <= _declared()


def test_library_exports_every_declared_symbol():
    from paper_2005_11806_gb300 import pressure
    if not os.path.exists(pressure.LIB_PATH):
        from paper_2005_11806_gb300 import build_ext
        build_ext.build()
    L = pressure.lib()
    for name in sorted(_declared()):
        assert hasattr(L, name), name
    assert set(pressure.EXPORTS) >= _declared()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2005_11806_gb300 import pressure
    monkeypatch.setattr(pressure, "_lib", None)
    monkeypatch.setattr(pressure, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        pressure.lib()
