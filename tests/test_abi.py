"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point include/grim.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(grim_[a-z0-9_]+)\s*\(", text))
    return names


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("grim_init", "grim_step", "grim_residual", "grim_stage", "grim_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1702_01106_b300 import build, grim
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(grim.EXPORTS) <= declared_symbols()


def test_library_reports_errors_without_gpu_work():
    from paper_1702_01106_b300 import build
    lib = ctypes.CDLL(build.build())
    lib.grim_strerror.restype = ctypes.c_char_p
    assert lib.grim_strerror(-1).decode().startswith("invalid")
    # NULL arguments are rejected before any CUDA call
    lib.grim_init.argtypes = [ctypes.c_void_p] * 6
    assert lib.grim_init(None, None, None, None, None, None) == -1
