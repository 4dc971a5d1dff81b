"""Admission and accounting logic of the serving loop on the CPU, with a fake
solver in place of libmfs (no GPU): every request finishes, the HBM budget
and the cap on concurrent setups hold, a system whose size estimate exceeds
the budget is still tried when it runs alone, clones reuse resident
hierarchies, and failed setups are counted without breaking the statistics.
"""
import threading
import time

import numpy as np
import pytest

from paper_1605_01522_gb300 import mfs, serving


class _FakeSystem:
    def __init__(self, ndofs):
        self.ndofs = ndofs


class _FakeSolver:
    live = 0
    peak_setups = 0
    setups_now = 0
    lock = threading.Lock()
    fail_keys = set()

    def __init__(self, system, shared=1000, own=500, **kw):
        self.system, self.shared, self.own = system, shared, own
        with _FakeSolver.lock:
            _FakeSolver.setups_now += 1
            _FakeSolver.peak_setups = max(_FakeSolver.peak_setups, _FakeSolver.setups_now)
        time.sleep(0.01)
        with _FakeSolver.lock:
            _FakeSolver.setups_now -= 1
        if system.ndofs in _FakeSolver.fail_keys:
            raise mfs.MfsError(mfs.ERR_OOM, "fake setup failure")

    def clone(self):
        c = _FakeSolver.__new__(_FakeSolver)
        c.system, c.shared, c.own = self.system, self.shared, self.own
        return c

    def solve(self, b, x, tol=1e-8):
        time.sleep(0.005)
        x[:] = 1.0
        return x, {"iters": 1}, mfs.OK

    def device_bytes(self, shared):
        return self.shared if shared else self.own

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    _FakeSolver.peak_setups = 0
    _FakeSolver.fail_keys = set()
    monkeypatch.setattr(serving.mfs, "Solver", _FakeSolver)
    return _FakeSolver


def _run(srv, reqs):
    for key, ndofs, reuse in reqs:
        srv.submit(key, _FakeSystem(ndofs), np.zeros(ndofs), reuse)
    srv.drain(timeout=60)
    return srv.stats()


def test_every_request_finishes_within_budget_and_setup_cap(fake):
    srv = serving.Server(hbm_budget=10 ** 7, workers=8, max_setups=2)
    try:
        reqs = [(k % 5, 100 + k % 5, k % 3 == 0) for k in range(60)]
        st = _run(srv, reqs)
    finally:
        srv.close()
    assert st["requests"] == 60 and st["converged"] == 60 and st["failed"] == 0
    assert st["peak_hbm_bytes"] <= 10 ** 7
    assert fake.peak_setups <= 2
    assert st["setups"] < 60  # resident hierarchies were reused


def test_unknown_system_over_its_estimate_runs_alone(fake):
    # the byte estimate of a 10^5-dof system is far above the budget; its real
    # footprint (1500 bytes) fits, so it runs once nothing else does
    srv = serving.Server(hbm_budget=10 ** 6, workers=4)
    try:
        st = _run(srv, [(0, 100000, False), (1, 10, False)])
    finally:
        srv.close()
    assert st["converged"] == 2


def test_failed_setups_are_counted(fake):
    fake.fail_keys = {77}
    srv = serving.Server(hbm_budget=10 ** 7, workers=4)
    try:
        st = _run(srv, [(0, 77, False), (1, 10, False), (2, 77, True)])
    finally:
        srv.close()
    assert st["requests"] == 3 and st["converged"] == 1 and st["failed"] == 2
    assert "fake setup failure" in next(iter(st["errors"]))


def test_fused_mode_solves_ready_requests_together(fake, monkeypatch):
    """fused=True: workers only admit and set up; ready requests are solved
    by shared batches (here a fake mfs_solve_batch); every request finishes,
    each exactly once, the budget and the setup cap hold, and batches hold
    more than one request."""
    calls = []
    lock = threading.Lock()

    def fake_batch(solvers, rhs, xs, tol=1e-8, nthreads=0, check=True):
        assert nthreads == 0 and len(set(map(id, solvers))) == len(solvers)
        with lock:
            calls.append(len(solvers))
        time.sleep(0.02)
        for x in xs:
            x[:] = 1.0
        return xs, [{"iters": 1}] * len(solvers), [mfs.OK] * len(solvers)

    monkeypatch.setattr(serving.mfs, "solve_batch", fake_batch)
    srv = serving.Server(hbm_budget=10 ** 7, workers=4, max_setups=2, fused=True, max_batch=16)
    try:
        st = _run(srv, [(k % 5, 100 + k % 5, k % 3 == 0) for k in range(80)])
    finally:
        srv.close()
    assert st["requests"] == 80 and st["converged"] == 80 and st["failed"] == 0
    assert sum(calls) == 80 and max(calls) > 1 and max(calls) <= 16
    assert st["fused_batches"] == len(calls) and st["peak_hbm_bytes"] <= 10 ** 7
    assert fake.peak_setups <= 2
