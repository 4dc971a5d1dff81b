"""GPU AMG setup (setup_device=1) against the host setup and the oracle.
Needs a GB300.

Aggregation is integer work: the GPU's parallel LFMIS rounds must give
exactly the host's (and the oracle's) greedy aggregates.  Prolongators,
restrictions, Galerkin blocks (diagonal and, for AMG(BGS), off-diagonal),
lambda_max, the SIMPLE diagonal and S~ must agree to float64 rounding
(1e-12 relative), at several sizes including ragged and coarse levels.
"""
import numpy as np
import pytest

pytest.importorskip("torch")

from oracle import amg, precond
from paper_1605_01522_gb300 import inputs, mfs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _rel(a, b):
    a, b = a.toarray(), b.toarray()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


SYSTEMS = {
    "2d": (lambda: inputs.thermo_elastic_2d(ne=20), dict(max_levels=3, coarse_max=0)),
    "3d3": (lambda: inputs.coupled_box_3d(ne=11, nfields=3), dict(max_levels=4, coarse_max=100)),
    "3d2": (lambda: inputs.coupled_box_3d(ne=17, nfields=2), dict(max_levels=4, coarse_max=200)),
    # per-dof Dirichlet flags (symmetry conditions), built-in / caller rigid-body modes
    "roll": (lambda: inputs.roller_box(ne=13), dict(max_levels=4, coarse_max=100)),
    "rollu": (lambda: inputs.roller_box(ne=13, user_nullspace=True), dict(max_levels=4, coarse_max=100)),
}


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("pc", ["bgs_amg", "amg_bgs"])
def test_gpu_setup_matches_host_setup_and_oracle(name, pc):
    gen, kw = SYSTEMS[name]
    s = gen()
    g = mfs.Solver(s, precond=pc, setup_device=1, **kw)
    h = mfs.Solver(s, precond=pc, setup_only=1, **kw)
    M = precond.Preconditioner(s.scipy_blocks(), [amg.FieldSpec.of(f) for f in s.fields],
                               precond.Params(pc, seed=7, **kw))
    lv = M.groups[0].levels
    assert g.num_levels(0) == h.num_levels(0) == len(lv)
    for l in range(len(lv)):
        for i in range(s.nfields):
            assert _rel(g.export_csr("A", 0, l, i, i), h.export_csr("A", 0, l, i, i)) < TOL
            if l < len(lv) - 1:
                ag = g.export_array("agg", 0, l, i)
                assert np.array_equal(ag, h.export_array("agg", 0, l, i))
                assert np.array_equal(ag, lv[l][i].agg)
                assert _rel(g.export_csr("P", 0, l, i), h.export_csr("P", 0, l, i)) < TOL
                assert _rel(g.export_csr("R", 0, l, i), lv[l][i].R) < TOL
                lg, lh = g.export_array("lambda", 0, l, i), h.export_array("lambda", 0, l, i)
                assert abs(lg - lh) <= 1e-13 * lh
    if pc == "amg_bgs":
        for l in range(1, len(lv)):
            for (i, j) in s.blocks:
                if i != j:
                    assert _rel(g.export_csr("A", 0, l, i, j), h.export_csr("A", 0, l, i, j)) < TOL
    g.close()
    h.close()


def test_gpu_setup_simple_objects():
    s = inputs.coupled_box_3d(ne=11, nfields=3)
    kw = dict(max_levels=4, coarse_max=100, simple_group=[0, 0, 1])
    g = mfs.Solver(s, precond="simple", setup_device=1, **kw)
    h = mfs.Solver(s, precond="simple", setup_only=1, **kw)
    for jj in range(2):
        assert np.array_equal(g.export_array("dtilde", 0, 0, jj), h.export_array("dtilde", 0, 0, jj))
    assert _rel(g.export_csr("A", 1, 0, 0, 0), h.export_csr("A", 1, 0, 0, 0)) < TOL
    for l in range(g.num_levels(1) - 1):
        assert np.array_equal(g.export_array("agg", 1, l, 0), h.export_array("agg", 1, l, 0))
        assert _rel(g.export_csr("P", 1, l, 0), h.export_csr("P", 1, l, 0)) < TOL
    g.close()
    h.close()


@pytest.mark.parametrize("approx", ["absrowsum", "diag"])
def test_gpu_setup_amg_simple_level_objects(approx):
    """AMG(SIMPLE): A~_11 and S~^l on every smoothed level, GPU vs host setup,
    and S~^l against the oracle's level Schur complement."""
    s = inputs.coupled_box_3d(ne=11, nfields=3)
    kw = dict(max_levels=4, coarse_max=100, simple_group=[0, 0, 1], simple_approx=approx)
    g = mfs.Solver(s, precond="amg_simple", setup_device=1, **kw)
    h = mfs.Solver(s, precond="amg_simple", setup_only=1, **kw)
    M = precond.Preconditioner(s.scipy_blocks(), [amg.FieldSpec.of(f) for f in s.fields],
                               precond.Params("amg_simple", seed=7, **kw))
    L = g.num_levels(0)
    assert L == h.num_levels(0) == len(M.op.grp.levels) and g.num_levels(1) == L - 1
    for l in range(L - 1):
        for jj in range(2):
            dg, dh = g.export_array("dtilde", 0, l, jj), h.export_array("dtilde", 0, l, jj)
            assert np.abs(dg - dh).max() <= 1e-12 * np.abs(dh).max()
            assert np.abs(dh - M.op.dt[l][jj]).max() <= 1e-12 * np.abs(dh).max()
        Sg, Sh = g.export_csr("A", 1, l, 0, 0), h.export_csr("A", 1, l, 0, 0)
        assert _rel(Sg, Sh) < TOL and _rel(Sh, M.op.S[l].A) < TOL
        lg, lh = g.export_array("lambda", 1, l, 0), h.export_array("lambda", 1, l, 0)
        assert abs(lg - lh) <= 1e-12 * lh and abs(lh - M.op.S[l].lam) <= 1e-12 * lh
    g.close()
    h.close()


def test_gpu_setup_constrained_box_nested_simple():
    """SIMPLE(AMG(BGS)) on the constrained box: the GPU setup's predictor
    hierarchy (with coupling blocks) and one-level Schur group equal the host's."""
    s = inputs.constrained_box(ne=12)
    kw = dict(max_levels=4, coarse_max=100, simple_pred="amg_bgs")
    g = mfs.Solver(s, precond="simple", setup_device=1, **kw)
    h = mfs.Solver(s, precond="simple", setup_only=1, **kw)
    assert g.num_levels(0) == h.num_levels(0) and g.num_levels(1) == h.num_levels(1) == 1
    assert _rel(g.export_csr("A", 1, 0, 0, 0), h.export_csr("A", 1, 0, 0, 0)) < TOL
    for l in range(1, g.num_levels(0)):
        for (i, j) in [(0, 1), (1, 0), (0, 2), (2, 0), (1, 2), (2, 1)]:
            assert _rel(g.export_csr("A", 0, l, i, j), h.export_csr("A", 0, l, i, j)) < TOL
    g.close()
    h.close()


def test_gpu_setup_petrov_galerkin_matches_host():
    s = inputs.fsi_box(ne=10, wind=(0.2, 0.1, 0.0))
    kw = dict(max_levels=3, coarse_max=100, simple_group=[0, 0, 0, 1], simple_approx="diag")
    g = mfs.Solver(s, precond="simple", setup_device=1, **kw)
    h = mfs.Solver(s, precond="simple", setup_only=1, **kw)
    assert g.num_levels(0) == h.num_levels(0)
    for l in range(g.num_levels(0) - 1):
        for i in range(3):
            assert _rel(g.export_csr("P", 0, l, i), h.export_csr("P", 0, l, i)) < TOL
            assert _rel(g.export_csr("R", 0, l, i), h.export_csr("R", 0, l, i)) < TOL
            assert _rel(g.export_csr("A", 0, l + 1, i, i), h.export_csr("A", 0, l + 1, i, i)) < TOL
    g.close()
    h.close()


@pytest.mark.parametrize("pc", ["bgs_amg", "amg_bgs", "simple"])
def test_solve_after_host_setup_matches_gpu_setup(pc):
    """A handle built by the host setup (setup_device=0) solves like one built on
    the GPU: the two hierarchies agree to rounding, so the FP64 solves take the
    same iterations and reach the same solution to 1e-9."""
    s = inputs.coupled_box_3d(ne=11, nfields=3)
    kw = dict(max_levels=4, coarse_max=100, precond=pc)
    out = []
    for dev in (0, 1):
        with mfs.Solver(s, setup_device=dev, **kw) as lib:
            x, info, rc = lib.solve(s.rhs, np.zeros(s.ndofs), tol=1e-8)
        assert rc == mfs.OK
        out.append((x, info["iters"]))
    assert abs(out[0][1] - out[1][1]) <= 1
    assert np.linalg.norm(out[0][0] - out[1][0]) <= 1e-9 * np.linalg.norm(out[1][0])
