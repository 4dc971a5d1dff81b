"""CUDA path (through the C ABI) against the FP64 oracle.  Needs a GB300.

* coupled matvec: element-wise against scipy on the same blocks;
* one preconditioner application (BGS(AMG), SIMPLE, AMG(BGS), AMG(SIMPLE)), FP64: within
  1e-12 relative (max-norm) of the oracle applied to the library's own
  exported hierarchy - the float64 kernels and the oracle differ only in
  summation order;
* FGMRES solves: true residual <= 1e-8 recomputed on the host, iterations
  within +-1 of the oracle's FGMRES (FP64) and within +10% (+1) for the FP32
  preconditioner;
* edge cases: zero right-hand side, nonzero initial guess, host and device
  vectors, one field, one level, ragged slice tails (node counts that are
  not multiples of 32).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import amg, krylov, precond
from oracle.cycles import SmootherParams
from paper_1605_01522_gb300 import inputs, mfs
from tests.oracle_from_lib import oracle_preconditioner

pytestmark = pytest.mark.gpu

APPLY_TOL = 1e-12


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _small(name):
    if name == "2d":
        return inputs.thermo_elastic_2d(ne=32), dict(max_levels=3, coarse_max=0)
    if name == "3d":
        return inputs.coupled_box_3d(ne=10, nfields=3), dict(max_levels=4, coarse_max=150)
    if name == "3d2":
        return inputs.coupled_box_3d(ne=13, nfields=2), dict(max_levels=3, coarse_max=100)
    if name == "fsi":
        return inputs.fsi_box(ne=8), dict(max_levels=3, coarse_max=100)
    if name == "cons":
        return inputs.constrained_box(ne=9), dict(max_levels=3, coarse_max=100)
    if name == "oseen":
        return inputs.fsi_box(ne=8, wind=(0.1, 0.05, 0.0)), dict(max_levels=3, coarse_max=100)
    if name == "roll":
        return inputs.roller_box(ne=9), dict(max_levels=3, coarse_max=100)
    if name == "rollu":
        return inputs.roller_box(ne=9, user_nullspace=True), dict(max_levels=3, coarse_max=100)
    raise KeyError(name)


def _oracle_params(pc, kw, extra):
    """Oracle parameters for the library options in `extra`."""
    ex = dict(extra)
    kind = ex.pop("smoother", "chebyshev")
    if kind == "gs":
        spk = dict(omega=ex.pop("gs_omega", 0.79), sweeps=ex.pop("gs_sweeps", 1))
    elif kind == "jacobi":
        spk = dict(omega=ex.pop("jacobi_omega", 2.0 / 3.0), sweeps=ex.pop("jacobi_sweeps", 1))
    else:
        spk = dict(degree=ex.pop("cheb_degree", 2))
    ex = {k: v for k, v in ex.items()
          if k in ("simple_group", "simple_approx", "bgs_order", "bgs_sweeps", "simple_pred")}
    return precond.Params(pc, **kw, **ex, smoother=SmootherParams(kind, **spk))


def _oracle_solve(s, kw, pc, extra):
    A = s.scipy_blocks()
    D = precond.assemble(A, s.nfields)
    prm = _oracle_params(pc, kw, extra)
    M = precond.Preconditioner(A, [amg.FieldSpec.of(f) for f in s.fields], prm)
    return krylov.fgmres(lambda v: D @ v, M, s.rhs, 1e-8, 50, maxiter=600), D


@pytest.mark.parametrize("rows_split", [0, 1, 2, 4])
@pytest.mark.parametrize("name", ["2d", "3d", "3d2"])
def test_matvec_matches_scipy(name, rows_split):
    """Every variant of the merged-row float64 matvec (1, 2 or 4 threads per
    block row, or the one the setup's timing picks)."""
    s, kw = _small(name)
    with mfs.Solver(s, **kw, rows_split=rows_split) as lib:
        D = precond.assemble(s.scipy_blocks(), s.nfields)
        x = np.random.default_rng(1).standard_normal(s.ndofs)
        y = lib.matvec(_cuda(x)).cpu().numpy()
        ref = D @ x
        assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
        # host-pointer path gives the same bits
        assert np.array_equal(lib.matvec(x), y)


CASES = [("2d", "bgs_amg", {}), ("2d", "amg_bgs", {}), ("2d", "simple", {}),
         ("3d", "bgs_amg", {}), ("3d", "amg_bgs", {}), ("3d", "simple", dict(simple_group=[0, 0, 1])),
         ("3d", "simple", dict(simple_group=[0, 1, 1])), ("3d", "bgs_amg", dict(bgs_order="fwd")),
         ("3d", "bgs_amg", dict(bgs_order="sym", bgs_sweeps=2)), ("3d2", "amg_bgs", dict(bgs_order="sym")),
         ("3d2", "simple", dict(simple_approx="diag")), ("3d2", "bgs_amg", dict(smoother="jacobi", jacobi_sweeps=2)),
         ("3d2", "bgs_amg", dict(cheb_degree=3)),
         ("fsi", "simple", dict(simple_group=[0, 0, 0, 1], simple_approx="diag")),
         ("fsi", "simple", dict(simple_group=[0, 0, 0, 1])), ("fsi", "bgs_amg", {})]
FSI = [c for c in CASES if c[0] == "fsi"]
# AMG(SIMPLE): the monolithic V-cycle with the SIMPLE level smoother
AMG_SIMPLE = [("2d", "amg_simple", {}), ("3d", "amg_simple", {}), ("3d", "amg_simple", dict(bgs_order="sym")),
              ("3d", "amg_simple", dict(simple_group=[0, 1, 0], simple_approx="diag")),
              ("3d2", "amg_simple", dict(smoother="jacobi", jacobi_sweeps=2)),
              ("fsi", "amg_simple", dict(simple_group=[0, 0, 0, 1]))]
# SIMPLE(BGS(AMG)) / SIMPLE(AMG(BGS)) (Sec. 6.3), incl. the constrained box whose
# multiplier block is zero and whose Schur group is solved by dense LU
NESTED = [("cons", "simple", {}), ("cons", "simple", dict(simple_pred="amg_bgs")),
          ("cons", "simple", dict(simple_pred="amg_bgs", simple_approx="diag", bgs_order="sym")),
          ("3d", "simple", dict(simple_pred="amg_bgs", simple_group=[0, 0, 1])),
          ("fsi", "simple", dict(simple_group=[0, 0, 0, 1], simple_approx="diag", simple_pred="amg_bgs"))]
# multicolour damped Gauss-Seidel smoothing (the paper's DD(GS(omega)), Sec. 7.1)
# and the single-level BGS(GS)
GS = [("2d", "bgs_amg", dict(smoother="gs")), ("3d", "amg_bgs", dict(smoother="gs")),
      ("3d", "simple", dict(smoother="gs", simple_group=[0, 0, 1])),
      ("3d2", "amg_simple", dict(smoother="gs", gs_sweeps=2, gs_omega=1.0)),
      ("3d", "bgs_gs", dict(smoother="gs")), ("2d", "bgs_gs", dict(smoother="gs", gs_omega=0.69, bgs_order="sym")),
      ("cons", "simple", dict(smoother="gs", simple_pred="amg_bgs"))]
# Petrov-Galerkin transfers on the Oseen velocity field (Sec. 7.2, R != P^T)
PG = [("oseen", "simple", dict(simple_group=[0, 0, 0, 1], simple_approx="diag")),
      ("oseen", "simple", dict(simple_group=[0, 0, 0, 1], simple_approx="diag", simple_pred="amg_bgs")),
      ("oseen", "bgs_amg", {})]


# symmetry conditions flagged per dof (1-3 held components per node), with the
# built-in or a caller-supplied rigid-body nullspace
ROLLER = [("roll", "bgs_amg", {}), ("rollu", "bgs_amg", {}), ("rollu", "amg_bgs", {}), ("roll", "simple", {})]


@pytest.mark.parametrize("name,pc,extra", CASES + AMG_SIMPLE + NESTED + GS + PG + ROLLER)
def test_apply_fp64_matches_oracle_on_same_hierarchy(name, pc, extra):
    s, kw = _small(name)
    with mfs.Solver(s, precond=pc, **kw, **extra) as lib:
        Mo = oracle_preconditioner(lib, s)
        for seed in (2, 3):
            v = np.random.default_rng(seed).standard_normal(s.ndofs)
            z = lib.apply(_cuda(v)).cpu().numpy()
            zr = Mo(v)
            err = np.abs(z - zr).max() / np.abs(zr).max()
            assert err <= APPLY_TOL, err


@pytest.mark.parametrize("name,pc,extra", [c for c in CASES if c[0] != "3d2" or c[1] == "simple"][:8] + FSI
                         + AMG_SIMPLE[:4] + NESTED + GS + PG[:2] + ROLLER)
def test_solve_fp64_iterations_match_oracle(name, pc, extra):
    s, kw = _small(name)
    ro, D = _oracle_solve(s, kw, pc, extra)
    with mfs.Solver(s, precond=pc, **kw, **extra) as lib:
        x, info, rc = lib.solve(_cuda(s.rhs), tol=1e-8)
        x = x.cpu().numpy()
    assert rc == mfs.OK and info["converged"] == 1
    true = np.linalg.norm(s.rhs - D @ x) / np.linalg.norm(s.rhs)
    assert true <= 1e-8
    assert abs(true - info["true_relres"]) <= 1e-3 * true + 1e-15
    # +-1, or +-1 % for long restarted runs (rounding differences accumulate over restarts)
    assert abs(info["iters"] - ro.iters) <= max(1, round(0.01 * ro.iters)), (info["iters"], ro.iters)
    assert np.linalg.norm(x - ro.x) <= 1e-6 * np.linalg.norm(ro.x)


@pytest.mark.parametrize("name,pc,extra", [("2d", "bgs_amg", {}), ("3d", "bgs_amg", {}), ("3d", "amg_bgs", {}),
                                           ("3d", "simple", {}), ("fsi", "bgs_amg", {})] + FSI[:1]
                         + AMG_SIMPLE[1:2] + NESTED[:2] + GS[:2] + GS[4:5] + PG[:1])
def test_solve_fp32_preconditioner(name, pc, extra):
    s, kw = _small(name)
    ro, D = _oracle_solve(s, kw, pc, extra)
    with mfs.Solver(s, precond=pc, precision="fp32p", **kw, **extra) as lib:
        x, info, rc = lib.solve(_cuda(s.rhs), tol=1e-8)
        x = x.cpu().numpy()
    true = np.linalg.norm(s.rhs - D @ x) / np.linalg.norm(s.rhs)
    assert rc == mfs.OK and true <= 1e-8
    assert info["iters"] <= int(np.ceil(1.10 * ro.iters)) + 1, (info["iters"], ro.iters)


def test_solve_edge_cases():
    s, kw = _small("3d2")
    D = precond.assemble(s.scipy_blocks(), s.nfields)
    with mfs.Solver(s, **kw) as lib:
        # zero right-hand side: zero iterations, x = 0
        x, info, rc = lib.solve(np.zeros(s.ndofs), tol=1e-8)
        assert rc == mfs.OK and info["iters"] == 0 and not x.any()
        # host vectors (copies inside the library) and a nonzero initial guess
        x0 = np.random.default_rng(5).standard_normal(s.ndofs)
        xh = x0.copy()
        _, info, rc = lib.solve(s.rhs, xh, tol=1e-8)
        assert rc == mfs.OK
        assert np.linalg.norm(s.rhs - D @ xh) <= 1e-8 * np.linalg.norm(s.rhs - D @ x0)
        # too few iterations: NOT_CONVERGED with the last iterate returned
        lib2 = mfs.Solver(s, max_iters=2, **kw)
        x2, info2, rc2 = lib2.solve(s.rhs, tol=1e-8)
        assert rc2 == mfs.ERR_NOT_CONVERGED and info2["iters"] == 2 and info2["true_relres"] < 1.0
        lib2.close()


def test_single_field_and_single_level():
    s, _ = _small("3d2")
    one = inputs.BlockSystem([s.fields[1]], {(0, 0): s.blocks[(1, 1)]}, s.rhs[s.offsets[1]:])
    A = one.scipy_blocks()[(0, 0)]
    for kw in (dict(max_levels=1), dict(max_levels=3, coarse_max=50)):
        for pc in ("bgs_amg", "amg_bgs"):
            with mfs.Solver(one, precond=pc, **kw) as lib:
                x, info, rc = lib.solve(_cuda(one.rhs), tol=1e-8)
                x = x.cpu().numpy()
                assert rc == mfs.OK
                assert np.linalg.norm(one.rhs - A @ x) <= 1e-8 * np.linalg.norm(one.rhs)
                if kw["max_levels"] == 1:
                    assert info["iters"] == 1


def test_dot_matches_host():
    s, kw = _small("3d2")
    rng = np.random.default_rng(12)
    with mfs.Solver(s, **kw) as lib:
        for _ in range(2):
            x, y = rng.standard_normal(s.ndofs), rng.standard_normal(s.ndofs)
            d = lib.dot(_cuda(x), _cuda(y))
            assert abs(d - float(np.dot(x, y))) <= 1e-13 * np.abs(x).max() * np.abs(y).max() * s.ndofs ** 0.5
        with pytest.raises(mfs.MfsError):
            lib.dot(x, y)  # host vectors are rejected


def test_zero_diagonal_block_is_refused():
    """The constrained box's multiplier block is zero: every preconditioner
    that smooths with D^-1 on that field (BGS(AMG), AMG(BGS), AMG(SIMPLE))
    must be refused by the GPU setup, as the oracle refuses it."""
    s, kw = _small("cons")
    for pc in ("bgs_amg", "amg_bgs", "amg_simple"):
        with pytest.raises(mfs.MfsError) as e:
            mfs.Solver(s, precond=pc, **kw)
        assert e.value.code == mfs.ERR_SINGULAR
    # the handle-free failure leaves the device usable
    with mfs.Solver(s, precond="simple", **kw) as lib:
        _, info, rc = lib.solve(_cuda(s.rhs), tol=1e-8)
        assert rc == mfs.OK


@pytest.mark.parametrize("prec", ["fp64", "fp32p"])
@pytest.mark.parametrize("name,pc", [("3d", "bgs_amg"), ("2d", "bgs_amg"), ("3d", "simple"), ("roll", "bgs_amg")])
def test_vcycle_tail_is_the_stepwise_vcycle_bit_for_bit(name, pc, prec):
    """The one-CTA tail (level above the coarsest + coarse solve, shared-memory
    vectors) reduces every row as the per-step launches do, so applications
    and whole solves equal the step-by-step V-cycle exactly; the profiled
    solve shows that the tail ran."""
    s, kw = _small(name)
    v = _cuda(np.random.default_rng(5).standard_normal(s.ndofs))
    with mfs.Solver(s, precond=pc, precision=prec, vcycle_tail=0, **kw) as a, \
            mfs.Solver(s, precond=pc, precision=prec, vcycle_tail=1, profile=1, **kw) as b:
        assert torch.equal(a.apply(v), b.apply(v))
        xa, ia, _ = a.solve(_cuda(s.rhs), tol=1e-8)
        xb, ib, _ = b.solve(_cuda(s.rhs), tol=1e-8)
        assert ia["iters"] == ib["iters"] and torch.equal(xa, xb)
        assert any(r[0] == "vcycle_tail" for r in b.kernel_detail())


@pytest.mark.parametrize("prec", ["fp64", "fp32p"])
@pytest.mark.parametrize("name,pc", [("3d", "bgs_amg"), ("2d", "bgs_amg"), ("3d", "amg_bgs"), ("3d", "simple"),
                                     ("roll", "bgs_amg")])
def test_programmatic_dependent_launch_same_result_bit_for_bit(name, pc, prec):
    """With programmatic dependent launches every kernel still waits on the
    device for its predecessor's results (and a kernel after a copy, an event
    or a graph launch is launched the ordinary way), so solves - graph replay,
    direct launches, per-launch profiling events, host vectors, only the
    launches of at most 40 CTAs programmatic - equal the ordinary launches
    exactly."""
    s, kw = _small(name)
    with mfs.Solver(s, precond=pc, precision=prec, pdl=0, **kw) as a, \
            mfs.Solver(s, precond=pc, precision=prec, pdl=1, **kw) as b, \
            mfs.Solver(s, precond=pc, precision=prec, pdl=1, no_graphs=1, **kw) as c, \
            mfs.Solver(s, precond=pc, precision=prec, pdl=1, profile=1, **kw) as d, \
            mfs.Solver(s, precond=pc, precision=prec, pdl=40, **kw) as e:
        xa, ia, _ = a.solve(_cuda(s.rhs), tol=1e-8)
        for sv in (b, c, d, e, b, d):
            xb, ib, _ = sv.solve(_cuda(s.rhs), tol=1e-8)
            assert ia["iters"] == ib["iters"] and torch.equal(xa, xb)
        xh, ih, _ = b.solve(s.rhs.copy(), np.zeros(s.ndofs), tol=1e-8)
        assert ih["iters"] == ia["iters"] and np.array_equal(xh, xa.cpu().numpy())
        v = _cuda(np.random.default_rng(6).standard_normal(s.ndofs))
        za = a.apply(v)
        for sv in (b, e):  # preconditioner applications and matvecs take the same launches
            assert torch.equal(za, sv.apply(v)) and torch.equal(a.matvec(v), sv.matvec(v))
