"""The C-ABI library builds, loads without a GPU and exports every entry point of include/xdg.h."""
import ctypes
import os
import re

from paper_2003_02431_gb300 import xdg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(xdg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("xdg_create_hierarchy", "xdg_apply", "xdg_vcycle", "xdg_solve", "xdg_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    xdg.build()
    lib = ctypes.CDLL(xdg.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    bound = {n for n, _, _ in xdg.SIGNATURES}
    assert set(_declared()) <= bound


def test_strerror_without_gpu():
    lib = xdg.load()
    assert lib.xdg_strerror(0) == b"XDG_OK"
    assert lib.xdg_strerror(4) == b"XDG_ENOTCONV"
