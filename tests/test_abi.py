"""The C-ABI library loads and exports every entry point include/kldi.h declares
(no compute calls; runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names.update(re.findall(r"\b(kldi_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_declared_symbols():
    from paper_2605_10363_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_symbols()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_imports_and_reports_version():
    from paper_2605_10363_gb300 import kldi
    assert "sm_103a" in kldi.version()
