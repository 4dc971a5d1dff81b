"""The C-ABI library builds, loads and exports every symbol include/mfs.h
declares (no GPU needed; no compute call is made)."""
import ctypes
import os
import re

from paper_1605_01522_gb300 import build, mfs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mfs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mfs_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert _declared() == sorted(mfs.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings_and_defaults():
    lib = mfs.load()
    for code in range(0, -8, -1):
        assert lib.mfs_strerror(code)
    p = mfs.default_params()
    assert (p.precond, p.bgs_order, p.bgs_sweeps, p.restart, p.cheb_degree) == (0, 0, 1, 50, 2)
    assert abs(p.cheb_ratio - 30.0) < 1e-15 and abs(p.cheb_boost - 1.1) < 1e-15
