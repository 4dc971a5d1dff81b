"""The fused batch executor of mfs_solve_batch (nthreads = 0) on the GPU.

All systems of a batch advance their FGMRES iterations together; each step of
an iteration is one multi-system launch over every system, the steps of one
iteration are one CUDA graph.  Each system still runs its own kernels with
its own arguments in its own order, so its result must be its solo result
bit for bit: same x, same iteration count.  Covered: different sizes (and so
different level counts and sparse layouts) in one batch, 2- and 3-field
systems mixed, BGS(AMG) / AMG(BGS) / SIMPLE, float64 and float32
preconditioners, Gauss-Seidel smoothing, restarts at different iterations, a
system that stops at max_iters, a zero right-hand side, host vectors, graph
reuse by a second call, one group and three concurrent groups, and the full 256-system batch of 2-field 3D boxes
(n_e log-uniform in [12, 48]) against solo solves and the FP64 oracle's
iteration counts.  Needs a GB300.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import amg, krylov, precond
from paper_1605_01522_gb300 import inputs, mfs

pytestmark = pytest.mark.gpu


def _systems(sizes, nfields, seed=3):
    out = {}
    for ne, nf in zip(sizes, nfields):
        if (ne, nf) not in out:
            out[(ne, nf)] = inputs.coupled_box_3d(ne=ne, nfields=nf, seed=seed)
    return out


def _solvers(keys, systems, **kw):
    base, solvers = {}, []
    for key in keys:
        if key not in base:
            base[key] = mfs.Solver(systems[key], **kw)
            solvers.append(base[key])
        else:
            solvers.append(base[key].clone())
    return solvers


def _solo(solvers, rhs, x0=None):
    out = []
    for k, (sv, b) in enumerate(zip(solvers, rhs)):
        x = torch.zeros_like(b) if x0 is None else x0[k].clone()
        x, info, rc = sv.solve(b, x, tol=1e-8)
        out.append((x.cpu().numpy(), info["iters"], rc))
    return out


def _check_fused(solvers, rhs, solo, reps=2, x0=None):
    # one group, then three groups of similar sizes (concurrent chains)
    for rep in range(reps + 1):
        xs = [torch.zeros_like(b) if x0 is None else x0[k].clone() for k, b in enumerate(rhs)]
        xs, infos, status = mfs.solve_batch(solvers, rhs, xs, tol=1e-8, nthreads=-1 if rep < reps else -3,
                                            check=False)
        for k in range(len(solvers)):
            assert status[k] == solo[k][2], k
            assert infos[k]["iters"] == solo[k][1], (k, infos[k]["iters"], solo[k][1])
            assert np.array_equal(xs[k].cpu().numpy(), solo[k][0]), k


@pytest.mark.parametrize("prec", ["fp64", "fp32p"])
@pytest.mark.parametrize("pc", ["bgs_amg", "amg_bgs", "simple"])
def test_fused_batch_equals_solo(prec, pc):
    sizes = [5, 9, 13, 9, 17, 5, 11, 13]
    nfields = [2, 3, 2, 2, 3, 3, 2, 2]
    systems = _systems(sizes, nfields)
    keys = list(zip(sizes, nfields))
    solvers = _solvers(keys, systems, precond=pc, precision=prec, max_levels=4, coarse_max=200)
    rhs = [torch.from_numpy(inputs.system_rhs(systems[key], 5000 + k)).cuda() for k, key in enumerate(keys)]
    solo = _solo(solvers, rhs)
    assert all(rc == mfs.OK for _, _, rc in solo)
    _check_fused(solvers, rhs, solo)
    for sv in solvers:
        sv.close()


def test_fused_restarts_max_iters_zero_rhs_and_nonzero_x0():
    """restart 6: the systems restart at different iterations; one handle
    stops at max_iters (status and x as its solo solve); one right-hand side
    is zero (0 iterations); a nonzero initial guess is honoured."""
    sizes = [6, 10, 14, 8]
    systems = _systems(sizes, [2] * 4)
    keys = [(ne, 2) for ne in sizes]
    solvers = [mfs.Solver(systems[keys[0]], restart=6, max_levels=3, coarse_max=100),
               mfs.Solver(systems[keys[1]], restart=6, max_levels=3, coarse_max=100, max_iters=9),
               mfs.Solver(systems[keys[2]], restart=6, max_levels=3, coarse_max=100),
               mfs.Solver(systems[keys[3]], restart=6, max_levels=3, coarse_max=100, precision="fp32p")]
    rhs = [torch.from_numpy(inputs.system_rhs(systems[key], 70 + k)).cuda() for k, key in enumerate(keys)]
    rhs[2].zero_()
    x0 = [torch.zeros_like(b) for b in rhs]
    x0[3] = torch.from_numpy(np.random.default_rng(1).standard_normal(rhs[3].numel())).cuda()
    solo = _solo(solvers, rhs, x0)
    assert solo[1][2] == mfs.ERR_NOT_CONVERGED and solo[1][1] == 9
    assert solo[2][1] == 0 and solo[0][1] > 6
    _check_fused(solvers, rhs, solo, x0=x0)
    for sv in solvers:
        sv.close()


def test_fused_gauss_seidel_and_host_vectors():
    sizes = [7, 12, 9]
    systems = _systems(sizes, [2] * 3)
    keys = [(ne, 2) for ne in sizes]
    solvers = _solvers(keys, systems, smoother="gs", precision="fp32p", max_levels=3, coarse_max=100)
    rhs = [inputs.system_rhs(systems[key], 90 + k) for k, key in enumerate(keys)]
    solo = _solo(solvers, [torch.from_numpy(b).cuda() for b in rhs])
    xs = [np.zeros(b.shape[0]) for b in rhs]
    xs, infos, status = mfs.solve_batch(solvers, rhs, xs, tol=1e-8, nthreads=0)
    for k in range(len(solvers)):
        assert status[k] == mfs.OK and infos[k]["iters"] == solo[k][1]
        assert np.array_equal(xs[k], solo[k][0])
    for sv in solvers:
        sv.close()


def _oracle_iters(system):
    A = system.scipy_blocks()
    D = precond.assemble(A, system.nfields)
    M = precond.Preconditioner(A, [amg.FieldSpec.of(f) for f in system.fields],
                               precond.Params("bgs_amg", max_levels=5, coarse_max=1000))
    return D, krylov.fgmres(lambda v: D @ v, M, system.rhs, 1e-8, 50).iters


def test_fused_full_batch_of_256_systems():
    """The 256-system batch (2-field boxes, n_e log-uniform in [12, 48], 36
    distinct meshes, 28.2 M dofs), BGS(AMG) in FP32P: every system converges
    to a true residual <= 1e-8 (float64 matvec on the device); the smallest,
    the median and the largest system equal their solo solves bit for bit;
    those three need at most 10 % (+1) more iterations than the FP64 oracle."""
    sizes, mats, rhs = inputs.batch_workload(256, 12, 48, 3)
    keys = [int(ne) for ne in sizes]
    base, solvers = {}, []
    for ne in keys:
        if ne not in base:
            base[ne] = mfs.Solver(mats[ne], precision="fp32p", max_levels=5, coarse_max=1000)
            solvers.append(base[ne])
        else:
            solvers.append(base[ne].clone())
    bs = [torch.from_numpy(b).cuda() for b in rhs]
    xs, infos, status = mfs.solve_batch(solvers, bs, tol=1e-8, nthreads=0)
    assert status == [0] * 256
    for k in range(256):
        r = bs[k] - solvers[k].matvec(xs[k])
        assert float(torch.linalg.norm(r) / torch.linalg.norm(bs[k])) <= 1e-8, k
    order = np.argsort(sizes, kind="stable")
    picks = [int(order[0]), int(order[128]), int(order[-1])]
    for k in picks:
        x, info, rc = solvers[k].solve(bs[k], torch.zeros_like(bs[k]), tol=1e-8)
        assert rc == mfs.OK and info["iters"] == infos[k]["iters"]
        assert torch.equal(x, xs[k]), k
    for k in picks[:2]:  # the largest one takes minutes in the CPU oracle
        s = mats[keys[k]]
        s.rhs = rhs[k]
        _, it_o = _oracle_iters(s)
        assert infos[k]["iters"] <= int(1.10 * it_o) + 1, (k, infos[k]["iters"], it_o)
    for sv in solvers:
        sv.close()
