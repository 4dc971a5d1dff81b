"""Serving loop (paper_1605_01522_gb300/serving.py) on the GPU.  Needs a GB300.

Requests of different systems arrive while others run; each is admitted
when a slot and HBM budget are free, gets its own handle (a clone of a
resident hierarchy or a fresh setup), is solved on its own stream or - in
the fused mode - together with the other ready requests by the fused batch
executor, and must return exactly the solution a solo solve gives, at a true
residual <= 1e-8.  A tight budget must cap the device memory held and the
requests in flight.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import precond
from paper_1605_01522_gb300 import inputs, mfs, serving

pytestmark = pytest.mark.gpu

KW = dict(max_levels=4, coarse_max=200, precision="fp32p")


def _pool():
    pool = {}
    for ne in (6, 9):
        for nf in (2, 3):
            pool[(ne, nf)] = inputs.coupled_box_3d(ne=ne, nfields=nf, seed=4)
    return pool


def _requests(pool, n, seed):
    rng = np.random.default_rng(seed)
    keys = list(pool)
    out = []
    for k in range(n):
        key = keys[rng.integers(len(keys))]
        out.append((key, inputs.system_rhs(pool[key], 4000 + k), bool(rng.random() < 0.5)))
    return out


@pytest.mark.parametrize("fused", [False, True])
def test_each_result_same_alone_and_in_the_mix(fused):
    pool = _pool()
    reqs = _requests(pool, 24, 1)
    alone = []
    solvers = {key: mfs.Solver(s, **KW) for key, s in pool.items()}
    for key, b, _ in reqs:
        x, info, rc = solvers[key].solve(b, np.zeros(pool[key].ndofs), tol=1e-8)
        assert rc == mfs.OK
        alone.append(x)
    for sv in solvers.values():
        sv.close()
    srv = serving.Server(hbm_budget=8 << 30, workers=6, fused=fused, **KW)
    try:
        handles = []
        for i, (key, b, reuse) in enumerate(reqs):
            handles.append(srv.submit(key, pool[key], b, reuse))
            if i % 5 == 4:
                srv.drain(timeout=600)  # some requests arrive after others finished (resident reuse)
        srv.drain(timeout=600)
        for (key, b, _), r, xa in zip(reqs, handles, alone):
            assert r.rc == mfs.OK, r.error
            assert np.array_equal(r.x, xa)
            D = precond.assemble(pool[key].scipy_blocks(), pool[key].nfields)
            assert np.linalg.norm(b - D @ r.x) <= 1e-8 * np.linalg.norm(b)
        st = srv.stats()
        assert st["converged"] == len(reqs) and st["peak_in_flight"] >= 2
        assert st["setups"] < len(reqs)  # some requests reused a resident hierarchy
        if fused:  # every request went through a fused batch
            assert st["fused_batches"] >= 1 and round(st["fused_batches"] * st["mean_batch"]) == len(reqs)
    finally:
        srv.close()


def test_budget_limits_memory_and_concurrency():
    pool = _pool()
    reqs = _requests(pool, 10, 2)
    probe = mfs.Solver(pool[(9, 3)], **KW)
    one = probe.device_bytes(True) + probe.device_bytes(False)
    probe.close()
    budget = int(2.5 * one)
    srv = serving.Server(hbm_budget=budget, workers=8, keep_resident=False, **KW)
    try:
        handles = [srv.submit(key, pool[key], b, reuse) for key, b, reuse in reqs]
        srv.drain(timeout=600)
        st = srv.stats()
        bad = [(r.key, r.rc, r.error, r.info) for r in handles if r.rc != mfs.OK]
        assert st["converged"] == len(reqs), (bad, budget, one)
        assert st["peak_hbm_bytes"] <= budget
    finally:
        srv.close()
