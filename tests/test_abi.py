"""The C-ABI library builds, loads and exports every symbol include/mfs.h
declares (no GPU needed; no compute call is made)."""
import ctypes
import os
import re

import pytest

from paper_1605_01522_gb300 import build, inputs, mfs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mfs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mfs_[a-z0-9_]+)\s*\(", src)))


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
    assert p.rows_split == 0  # threads per row of the float64 matvec: timed at setup
    assert (p.layout_tune, p.vcycle_tail, p.pdl) == (0, 0, -1)  # layouts for one solve, stepwise V-cycle, automatic PDL


@pytest.mark.parametrize("split", [3, -1, 8])
def test_bad_rows_split_is_refused(split):
    """Only 0 (timed) and 1, 2, 4 threads per block row exist; parameters are
    checked before anything is built (a host-only setup reaches the check)."""
    s = inputs.thermo_elastic_2d(ne=4)
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(s, setup_only=1, rows_split=split)
    assert e.value.code == mfs.ERR_INVALID


@pytest.mark.parametrize("field,value", [("pdl", -2), ("vcycle_tail", 2), ("layout_tune", -1)])
def test_bad_launch_options_are_refused(field, value):
    """Out-of-range launch options are refused before anything is built."""
    s = inputs.thermo_elastic_2d(ne=4)
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(s, setup_only=1, **{field: value})
    assert e.value.code == mfs.ERR_INVALID
