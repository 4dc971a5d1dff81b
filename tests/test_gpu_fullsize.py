"""Full-size workload (3-field 64^3 coupled box, 1,373,125 dofs) on the GPU,
in the configuration bench.py times.  Needs a GB300.

* FP64 solves: iterations within +-1 of the oracle's stored counts
  (tests/golden/oracle_counts.json, written by make_oracle_counts.py from the
  oracle alone) and a true residual <= 1e-8 recomputed on the host by scipy;
* FP32-preconditioner solves: true residual <= 1e-8 and at most 10 % (+1)
  more iterations than the oracle;
* coupled matvec on sampled rows, each recomputed on the host.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import precond
from paper_1605_01522_gb300 import inputs, mfs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
KW = dict(max_levels=5, coarse_max=1000)
_SYS = {}


def _system():
    if "s" not in _SYS:
        s = inputs.coupled_box_3d(ne=64, nfields=3, seed=1)
        _SYS["s"] = s
        _SYS["D"] = precond.assemble(s.scipy_blocks(), 3)
    return _SYS["s"], _SYS["D"]


def _counts():
    with open(os.path.join(HERE, "golden", "oracle_counts.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("pc", ["bgs_amg", "amg_bgs", "simple", "amg_simple"])
def test_fullsize_fp64_matches_oracle_counts(pc):
    s, D = _system()
    ref = _counts()[f"coupled_box_3d_ne64_f3/{pc}"]
    with mfs.Solver(s, precond=pc, **KW) as lib:
        x, info, rc = lib.solve(torch.from_numpy(s.rhs).cuda(), tol=1e-8)
        x = x.cpu().numpy()
    assert rc == mfs.OK
    true = np.linalg.norm(s.rhs - D @ x) / np.linalg.norm(s.rhs)
    assert true <= 1e-8
    assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])


@pytest.mark.parametrize("pc", ["bgs_amg", "amg_bgs", "amg_simple"])
def test_fullsize_fp32_preconditioner(pc):
    s, D = _system()
    ref = _counts()[f"coupled_box_3d_ne64_f3/{pc}"]
    with mfs.Solver(s, precond=pc, precision="fp32p", **KW) as lib:
        x, info, rc = lib.solve(torch.from_numpy(s.rhs).cuda(), tol=1e-8)
        x = x.cpu().numpy()
    assert rc == mfs.OK
    true = np.linalg.norm(s.rhs - D @ x) / np.linalg.norm(s.rhs)
    assert true <= 1e-8
    assert info["iters"] <= int(np.ceil(1.10 * ref["iters"])) + 1, (info["iters"], ref["iters"])


_FSI = {}


def _fsi():
    if "s" not in _FSI:
        s = inputs.fsi_box(ne=48, seed=2)
        _FSI["s"] = s
        _FSI["D"] = precond.assemble(s.scipy_blocks(), 4)
    return _FSI["s"], _FSI["D"]


FSI_SIMPLE = dict(simple_group=[0, 0, 0, 1], simple_approx="diag")


@pytest.mark.parametrize("prec", ["fp64", "fp32p"])
def test_fullsize_split_box_saddle_simple(prec):
    s, D = _fsi()
    ref = _counts()["fsi_box_ne48/simple"]
    with mfs.Solver(s, precond="simple", precision=prec, **KW, **FSI_SIMPLE) as lib:
        x, info, rc = lib.solve(torch.from_numpy(s.rhs).cuda(), tol=1e-8)
        x = x.cpu().numpy()
    assert rc == mfs.OK
    assert np.linalg.norm(s.rhs - D @ x) <= 1e-8 * np.linalg.norm(s.rhs)
    if prec == "fp64":
        assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])
    else:
        assert info["iters"] <= int(np.ceil(1.10 * ref["iters"])) + 1, (info["iters"], ref["iters"])


@pytest.mark.parametrize("pc,extra", [("bgs_amg", {}), ("amg_simple", FSI_SIMPLE)])
def test_fullsize_split_box_fails_like_the_oracle(pc, extra):
    """BGS(AMG) on the saddle system does not reach 1e-8 in 400 iterations in
    the oracle (Sec. 4.1: BGS needs dominant diagonal blocks), nor does
    AMG(SIMPLE) with a diagonal A~_11 on the coarse levels; the GPU must
    report the same failure with a similar residual."""
    s, D = _fsi()
    ref = _counts()[f"fsi_box_ne48/{pc}"]
    assert not ref["converged"]
    with mfs.Solver(s, precond=pc, max_iters=ref["iters"], **KW, **extra) as lib:
        x, info, rc = lib.solve(torch.from_numpy(s.rhs).cuda(), tol=1e-8)
    assert rc == mfs.ERR_NOT_CONVERGED and info["iters"] == ref["iters"]
    assert 0.5 * ref["relres"] <= info["true_relres"] <= 2.0 * ref["relres"]


def test_fullsize_matvec_sampled_rows():
    s, D = _system()
    rng = np.random.default_rng(9)
    xv = rng.standard_normal(s.ndofs)
    with mfs.Solver(s, **KW) as lib:
        y = lib.matvec(torch.from_numpy(xv).cuda()).cpu().numpy()
    rows = rng.choice(s.ndofs, 2000, replace=False)
    rows = np.concatenate([rows, [0, s.ndofs - 1, s.offsets[1], s.offsets[2] - 1]])
    for r in rows:
        lo, hi = D.indptr[r], D.indptr[r + 1]
        ref = float(np.dot(D.data[lo:hi], xv[D.indices[lo:hi]]))
        assert abs(y[r] - ref) <= 1e-12 * (np.abs(D.data[lo:hi]).sum() * np.abs(xv).max())


_CONS = {}


def _cons():
    if "s" not in _CONS:
        s = inputs.constrained_box(ne=64, nfields=3, seed=5)
        _CONS["s"] = s
        _CONS["D"] = precond.assemble(s.scipy_blocks(), 4)
    return _CONS["s"], _CONS["D"]


@pytest.mark.parametrize("pred", ["bgs_amg", "amg_bgs"])
@pytest.mark.parametrize("prec", ["fp64", "fp32p"])
def test_fullsize_constrained_box_nested_simple(pred, prec):
    """Lung-like constrained box (zero multiplier block, Schur group solved by
    dense LU): SIMPLE(BGS(AMG)) and SIMPLE(AMG(BGS)) against the oracle's
    stored counts (39 each)."""
    s, D = _cons()
    key = "constrained_box_ne64_f3_m4/simple" + ("+amg_bgs" if pred == "amg_bgs" else "")
    ref = _counts()[key]
    with mfs.Solver(s, precond="simple", simple_pred=pred, precision=prec, **KW) as lib:
        assert lib.num_levels(1) == 1
        x, info, rc = lib.solve(torch.from_numpy(s.rhs).cuda(), tol=1e-8)
        x = x.cpu().numpy()
    assert rc == mfs.OK
    assert np.linalg.norm(s.rhs - D @ x) <= 1e-8 * np.linalg.norm(s.rhs)
    if prec == "fp64":
        assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])
    else:
        assert info["iters"] <= int(np.ceil(1.10 * ref["iters"])) + 1, (info["iters"], ref["iters"])


@pytest.mark.parametrize("prec", ["fp64", "fp32p"])
def test_fullsize_gauss_seidel_smoother(prec):
    """BGS(AMG) with the multicolour damped Gauss-Seidel smoother (omega 0.79,
    the paper's DD(GS(0.79)) analogue) on the 64^3 box: 48 oracle iterations."""
    s, D = _system()
    ref = _counts()["coupled_box_3d_ne64_f3/bgs_amg+gs"]
    with mfs.Solver(s, precond="bgs_amg", smoother="gs", precision=prec, **KW) as lib:
        x, info, rc = lib.solve(torch.from_numpy(s.rhs).cuda(), tol=1e-8)
        x = x.cpu().numpy()
    assert rc == mfs.OK
    assert np.linalg.norm(s.rhs - D @ x) <= 1e-8 * np.linalg.norm(s.rhs)
    if prec == "fp64":
        assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])
    else:
        assert info["iters"] <= int(np.ceil(1.10 * ref["iters"])) + 1, (info["iters"], ref["iters"])


@pytest.mark.parametrize("prec", ["fp64", "fp32p"])
def test_fullsize_oseen_petrov_galerkin(prec):
    """Split box with an Oseen velocity block (wind (0.2, 0.1, 0)); the velocity
    hierarchy uses Petrov-Galerkin transfers: SIMPLE(diag) against the oracle's
    216 iterations (+-1 %, restarted runs)."""
    s = inputs.fsi_box(ne=48, seed=2, wind=(0.2, 0.1, 0.0))
    D = precond.assemble(s.scipy_blocks(), 4)
    ref = _counts()["oseen_fsi_box_ne48/simple"]
    with mfs.Solver(s, precond="simple", precision=prec, **KW, **FSI_SIMPLE) as lib:
        x, info, rc = lib.solve(torch.from_numpy(s.rhs).cuda(), tol=1e-8)
        x = x.cpu().numpy()
    assert rc == mfs.OK
    assert np.linalg.norm(s.rhs - D @ x) <= 1e-8 * np.linalg.norm(s.rhs)
    if prec == "fp64":
        assert abs(info["iters"] - ref["iters"]) <= max(1, round(0.01 * ref["iters"])), (info["iters"], ref["iters"])
    else:
        assert info["iters"] <= int(np.ceil(1.10 * ref["iters"])) + 1, (info["iters"], ref["iters"])


def test_split_box_64_simple_matches_oracle_count():
    """Config 2 at 64^3 (1,394,250 dofs), SIMPLE(diag) as benchmarked:
    FP64 within 1 % (+1) of the oracle's count (a long restarted run),
    FP32P within 10 % (+1); true residuals <= 1e-8 recomputed on the host."""
    ref = _counts()["fsi_box_ne64/simple"]
    s = inputs.fsi_box(ne=64, seed=2)
    D = precond.assemble(s.scipy_blocks(), 4)
    for prec in ("fp64", "fp32p"):
        with mfs.Solver(s, precond="simple", precision=prec, **KW, **FSI_SIMPLE) as lib:
            x, info, rc = lib.solve(torch.from_numpy(s.rhs).cuda(), tol=1e-8)
            x = x.cpu().numpy()
        assert rc == mfs.OK
        assert np.linalg.norm(s.rhs - D @ x) <= 1e-8 * np.linalg.norm(s.rhs)
        if prec == "fp64":
            assert abs(info["iters"] - ref["iters"]) <= max(1, round(0.01 * ref["iters"])), (info["iters"], ref["iters"])
        else:
            assert info["iters"] <= int(np.ceil(1.10 * ref["iters"])) + 1, (info["iters"], ref["iters"])


@pytest.mark.parametrize("pc", ["bgs_amg", "amg_bgs", "simple"])
def test_thermo_elastic_2d_matches_oracle_count(pc):
    """Config 0 (3,267 dofs, 3 SA-AMG levels) as benchmarked: iterations
    within 1 of the oracle's stored count in FP64."""
    ref = _counts()[f"thermo_elastic_2d_ne32/{pc}"]
    s = inputs.thermo_elastic_2d(ne=32, seed=0)
    D = precond.assemble(s.scipy_blocks(), 2)
    with mfs.Solver(s, precond=pc, max_levels=3, coarse_max=0) as lib:
        x, info, rc = lib.solve(torch.from_numpy(s.rhs).cuda(), tol=1e-8)
        x = x.cpu().numpy()
    assert rc == mfs.OK and np.linalg.norm(s.rhs - D @ x) <= 1e-8 * np.linalg.norm(s.rhs)
    assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])
