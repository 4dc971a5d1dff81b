"""Batched solves (mfs_clone + mfs_solve_batch) on the GPU.  Needs a GB300.

Independent systems of different sizes solved together by concurrent host
threads on per-handle streams must give, for every system, exactly the result
of solving it alone (same kernels, same reduction order), reach the 1e-8 true
residual, and leave the shared hierarchy untouched for the next batch.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import precond
from paper_1605_01522_gb300 import inputs, mfs

pytestmark = pytest.mark.gpu


def _work(prec):
    sizes = [6, 9, 13, 9, 6, 13, 11]
    base = {}
    for ne in sorted(set(sizes)):
        s = inputs.coupled_box_3d(ne=ne, nfields=2, seed=3)
        base[ne] = (s, mfs.Solver(s, precision=prec, max_levels=4, coarse_max=200))
    rhs = [inputs.system_rhs(base[ne][0], 3000 + k) for k, ne in enumerate(sizes)]
    return sizes, base, rhs


@pytest.mark.parametrize("prec", ["fp64", "fp32p"])
def test_batch_equals_individual_solves(prec):
    sizes, base, rhs = _work(prec)
    solvers = []
    used = set()
    for ne in sizes:
        solvers.append(base[ne][1] if ne not in used else base[ne][1].clone())
        used.add(ne)
    # alone, one after the other
    alone = []
    for sv, b in zip(solvers, rhs):
        x, info, rc = sv.solve(torch.from_numpy(b).cuda(), tol=1e-8)
        assert rc == mfs.OK
        alone.append((x.cpu().numpy(), info["iters"]))
    # together, twice (the second batch reuses every graph and the shared hierarchy)
    for rep in range(2):
        bs = [torch.from_numpy(b).cuda() for b in rhs]
        xs, infos, status = mfs.solve_batch(solvers, bs, tol=1e-8, nthreads=4)
        assert status == [0] * len(sizes)
        for k, (x, info) in enumerate(zip(xs, infos)):
            xk = x.cpu().numpy()
            assert np.array_equal(xk, alone[k][0]), k
            assert info["iters"] == alone[k][1]
            s = base[sizes[k]][0]
            D = precond.assemble(s.scipy_blocks(), 2)
            assert np.linalg.norm(rhs[k] - D @ xk) <= 1e-8 * np.linalg.norm(rhs[k])
    for sv in solvers:
        sv.close()


def test_batch_rejects_duplicate_handles_and_clone_outlives_source():
    s = inputs.coupled_box_3d(ne=6, nfields=2, seed=3)
    a = mfs.Solver(s, max_levels=3, coarse_max=100)
    b = torch.from_numpy(s.rhs).cuda()
    with pytest.raises(mfs.MfsError):
        mfs.solve_batch([a, a], [b, b])
    c = a.clone()
    xa, _, _ = a.solve(b)
    a.close()  # the clone keeps the shared hierarchy alive
    xc, info, rc = c.solve(b)
    assert rc == mfs.OK and torch.equal(xa, xc)
    c.close()
