"""Concurrent setups and solves on one GPU (the serving loop's situation).
Needs a GB300.

Eight host threads each build a handle for a different coupled system and
solve it while the others are in setup or in their own solves; every result
must equal, bit for bit, the solution of a handle built and solved alone.
This guards the setup's stream ordering (uploads, device-side layout builds
and the GPU AMG setup run on several streams at once).
"""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1605_01522_gb300 import inputs, mfs

pytestmark = pytest.mark.gpu

KW = dict(max_levels=4, coarse_max=200, precision="fp32p")


def _systems():
    out = []
    for k, (ne, nf) in enumerate([(10, 3), (12, 2), (14, 3), (9, 2), (13, 3), (11, 2), (15, 2), (8, 3)]):
        out.append(inputs.coupled_box_3d(ne=ne, nfields=nf, seed=20 + k))
    return out


def _solve(s):
    with mfs.Solver(s, **KW) as lib:
        x, info, rc = lib.solve(s.rhs, np.zeros(s.ndofs), tol=1e-8)
    return x, rc


def test_concurrent_setups_give_the_solo_results():
    systems = _systems()
    alone = [_solve(s) for s in systems]
    assert all(rc == mfs.OK for _, rc in alone)
    for _ in range(3):
        got = [None] * len(systems)
        errors = []

        def work(k):
            try:
                got[k] = _solve(systems[k])
            except Exception as e:  # reported below
                errors.append(repr(e))

        threads = [threading.Thread(target=work, args=(k,)) for k in range(len(systems))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors
        for (xa, _), (xg, rc) in zip(alone, got):
            assert rc == mfs.OK
            assert np.array_equal(xa, xg)
