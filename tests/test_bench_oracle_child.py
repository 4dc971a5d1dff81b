"""The CPU-baseline child of bench.py: it builds the oracle's own hierarchy,
reports "ready", times whole oracle solves on one core and on every core
after the GPU measurements, and saves its first solution, against which the
GPU arm states its error (vs_oracle).  Host logic only: run here on the
3,267-dof thermo-elastic system with a short budget."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import precond  # noqa: E402
from paper_1605_01522_gb300 import inputs  # noqa: E402


class _Args:
    workload, precond, smoother, simple_pred = "te2d", "bgs_amg", "chebyshev", "bgs_amg"
    baseline_s, no_pg = 0.2, False


def test_child_reports_ready_times_solves_and_saves_the_oracle_solution():
    old_ne = bench.NE
    bench.NE = 32
    try:
        child = bench.BaselineChild(_Args())
        child.wait_ready()
        res = child.result()
        x = child.solution()
    finally:
        bench.NE = old_ne
    assert res["single"]["solves"] >= 1 and res["single"]["iters"] == [19]
    assert res["all"]["cores"] == len(os.sched_getaffinity(0)) and res["all"]["solves"] >= res["all"]["cores"]
    s = inputs.thermo_elastic_2d(ne=32, seed=0)
    D = precond.assemble(s.scipy_blocks(), s.nfields)
    assert x is not None and x.shape == (s.ndofs,)
    assert np.linalg.norm(s.rhs - D @ x) <= 1e-8 * np.linalg.norm(s.rhs)
    assert child.solution() is None  # the file is removed once read
