"""Host setup of libmfs (no GPU needed: setup_only handles) against the oracle.

The library's C++ smoothed-aggregation setup and the oracle's numpy/scipy one
are independent implementations of the same steps; aggregates must agree
exactly (integer work) and prolongators, Galerkin blocks, lambda_max and the
SIMPLE objects to float64 rounding.
"""
import numpy as np
import pytest

from oracle import amg, precond
from paper_1605_01522_gb300 import inputs, mfs

TOL = 1e-12


def _rel(a, b):
    a = a.toarray() if hasattr(a, "toarray") else np.asarray(a)
    b = b.toarray() if hasattr(b, "toarray") else np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _systems():
    return {
        "2d": (inputs.thermo_elastic_2d(ne=16), dict(max_levels=3, coarse_max=0)),
        "3d": (inputs.coupled_box_3d(ne=8, nfields=3), dict(max_levels=4, coarse_max=200)),
    }


SYS = None


def _get(name):
    global SYS
    if SYS is None:
        SYS = _systems()
    return SYS[name]


@pytest.mark.parametrize("name", ["2d", "3d"])
@pytest.mark.parametrize("pc", ["bgs_amg", "amg_bgs"])
def test_hierarchy_matches_oracle(name, pc):
    s, kw = _get(name)
    lib = mfs.Solver(s, precond=pc, setup_only=1, seed=7, **kw)
    A = s.scipy_blocks()
    specs = [amg.FieldSpec.of(f) for f in s.fields]
    M = precond.Preconditioner(A, specs, precond.Params(pc, seed=7, **kw))
    lv = M.groups[0].levels
    assert lib.num_levels(0) == len(lv)
    for l in range(len(lv)):
        for i in range(s.nfields):
            assert _rel(lib.export_csr("A", 0, l, i, i), lv[l][i].A) < TOL
            if l < len(lv) - 1:
                agg = lib.export_array("agg", 0, l, i)
                assert np.array_equal(agg, lv[l][i].agg)
                assert _rel(lib.export_csr("P", 0, l, i), lv[l][i].P) < TOL
                assert _rel(lib.export_csr("R", 0, l, i), lv[l][i].R) < TOL
                assert abs(lib.export_array("lambda", 0, l, i) - lv[l][i].lam) < 1e-13 * lv[l][i].lam
    if pc == "amg_bgs":
        for l in range(1, len(lv)):
            for (i, j), Mij in M.op.A[l].items():
                if i != j:
                    assert _rel(lib.export_csr("A", 0, l, i, j), Mij) < TOL
    lib.close()


@pytest.mark.parametrize("approx", ["absrowsum", "diag"])
def test_simple_objects_match_oracle(approx):
    s, kw = _get("3d")
    grp = [0, 0, 1]
    lib = mfs.Solver(s, precond="simple", simple_group=grp, simple_approx=approx, setup_only=1, **kw)
    A = s.scipy_blocks()
    specs = [amg.FieldSpec.of(f) for f in s.fields]
    M = precond.Preconditioner(A, specs, precond.Params("simple", simple_group=grp, simple_approx=approx, **kw))
    for jj in range(2):
        assert _rel(lib.export_array("dtilde", 0, 0, jj), M.dtilde[jj]) < 1e-14
    assert _rel(lib.export_csr("A", 1, 0, 0, 0), M.schur_blocks[(0, 0)]) < TOL
    lv1 = M.groups[1].levels
    assert lib.num_levels(1) == len(lv1)
    for l in range(len(lv1) - 1):
        assert np.array_equal(lib.export_array("agg", 1, l, 0), lv1[l][0].agg)
        assert _rel(lib.export_csr("P", 1, l, 0), lv1[l][0].P) < TOL
    lib.close()


@pytest.mark.parametrize("approx", ["absrowsum", "diag"])
@pytest.mark.parametrize("grp", [[0, 0, 1], [1, 0, 0]])
def test_amg_simple_level_objects_match_oracle(approx, grp):
    """AMG(SIMPLE): per smoothed level the A~_11 diagonal of the merged
    predictor rows, the explicit S~^l and its lambda_max."""
    s, kw = _get("3d")
    lib = mfs.Solver(s, precond="amg_simple", simple_group=grp, simple_approx=approx, setup_only=1, seed=7, **kw)
    M = precond.Preconditioner(s.scipy_blocks(), [amg.FieldSpec.of(f) for f in s.fields],
                               precond.Params("amg_simple", simple_group=grp, simple_approx=approx, seed=7, **kw))
    L = len(M.op.grp.levels)
    assert lib.num_levels(0) == L and lib.num_levels(1) == L - 1
    for l in range(L - 1):
        for jj in range(2):
            assert _rel(lib.export_array("dtilde", 0, l, jj), M.op.dt[l][jj]) < 1e-14
        assert _rel(lib.export_csr("A", 1, l, 0, 0), M.op.S[l].A) < TOL
        assert abs(lib.export_array("lambda", 1, l, 0) - M.op.S[l].lam) < 1e-13 * M.op.S[l].lam
    with pytest.raises(mfs.MfsError):
        mfs.Solver(s, precond="amg_simple", simple_group=[0, 1, 1], setup_only=1, **kw)
    lib.close()


@pytest.mark.parametrize("pred", ["bgs_amg", "amg_bgs"])
def test_constrained_box_simple_objects_match_oracle(pred):
    """Lung-like constrained box: S~ (4 x 4, from a zero multiplier block) in a
    one-level Schur group, and for SIMPLE(AMG(BGS)) the predictor group's
    blockwise Galerkin coupling blocks on every coarse level."""
    s = inputs.constrained_box(ne=8)
    kw = dict(max_levels=3, coarse_max=100, simple_pred=pred)
    lib = mfs.Solver(s, precond="simple", setup_only=1, **kw)
    M = precond.Preconditioner(s.scipy_blocks(), [amg.FieldSpec.of(f) for f in s.fields],
                               precond.Params("simple", **kw))
    assert lib.num_levels(1) == len(M.groups[1].levels) == 1
    assert _rel(lib.export_csr("A", 1, 0, 0, 0), M.schur_blocks[(0, 0)]) < TOL
    L = lib.num_levels(0)
    assert L == len(M.groups[0].levels) == 3
    if pred == "amg_bgs":
        for l in range(1, L):
            for (i, j), Mij in M.op.pred.A[l].items():
                if i != j:
                    assert _rel(lib.export_csr("A", 0, l, i, j), Mij) < TOL
    lib.close()
    for pc in ("bgs_amg", "amg_bgs", "amg_simple"):
        with pytest.raises(mfs.MfsError) as e:
            mfs.Solver(s, precond=pc, setup_only=1, **kw)
        assert e.value.code == mfs.ERR_SINGULAR


@pytest.mark.parametrize("pc", ["bgs_amg", "amg_simple", "bgs_gs"])
def test_gauss_seidel_colours_match_oracle(pc):
    """Multicolour Gauss-Seidel: the library's greedy colours of every smoothed
    level equal the oracle's node_colors on the oracle's own level matrices."""
    from oracle.cycles import SmootherParams, node_colors
    s, kw = _get("3d")
    lib = mfs.Solver(s, precond=pc, smoother="gs", setup_only=1, seed=7, **kw)
    M = precond.Preconditioner(s.scipy_blocks(), [amg.FieldSpec.of(f) for f in s.fields],
                               precond.Params(pc, seed=7, smoother=SmootherParams("gs"), **kw))
    if pc == "bgs_gs":
        assert lib.num_levels(0) == 1
        for i, lf in enumerate(M.op.solvers):
            assert np.array_equal(lib.export_array("colors", 0, 0, i), node_colors(lf.fl.A, lf.fl.b))
        lib.close()
        return
    lv = M.groups[0].levels
    n = 0
    for l in range(len(lv) - 1):
        for i in range(s.nfields):
            c = lib.export_array("colors", 0, l, i)
            assert np.array_equal(c, node_colors(lv[l][i].A, lv[l][i].A.shape[0] // len(c)))
            n += 1
    if pc == "amg_simple":
        for l, fl in enumerate(M.op.S):
            c = lib.export_array("colors", 1, l, 0)
            assert np.array_equal(c, node_colors(fl.A, fl.A.shape[0] // len(c)))
    with pytest.raises(mfs.MfsError):
        lib.export_array("colors", 0, len(lv) - 1, 0)
    lib.close()
    assert n >= 6


def test_petrov_galerkin_transfers_match_oracle():
    """Oseen split box: the velocity field (non-symmetric, marked Petrov-Galerkin)
    gets R != P^T equal to the oracle's Sala-Tuminaro transfers on every level;
    the symmetric fields keep R = P^T."""
    s = inputs.fsi_box(ne=8, wind=(0.2, 0.1, 0.0))
    assert s.fields[2].petrov_galerkin
    kw = dict(max_levels=3, coarse_max=100, simple_group=[0, 0, 0, 1], simple_approx="diag")
    lib = mfs.Solver(s, precond="simple", setup_only=1, **kw)
    M = precond.Preconditioner(s.scipy_blocks(), [amg.FieldSpec.of(f) for f in s.fields],
                               precond.Params("simple", **kw))
    lv = M.groups[0].levels
    assert lib.num_levels(0) == len(lv) == 3
    for l in range(len(lv) - 1):
        for i in range(3):
            assert _rel(lib.export_csr("P", 0, l, i), lv[l][i].P) < TOL
            assert _rel(lib.export_csr("R", 0, l, i), lv[l][i].R) < TOL
            assert _rel(lib.export_csr("A", 0, l + 1, i, i), lv[l + 1][i].A) < TOL
            asym = np.abs((lv[l][i].R - lv[l][i].P.T).toarray()).max()
            assert (asym > 1e-3) if i == 2 else (asym == 0.0)
    lib.close()


def test_setup_rejects_bad_input():
    s, kw = _get("2d")
    bad = inputs.BlockSystem(s.fields, {k: v for k, v in s.blocks.items() if k != (1, 1)}, s.rhs)
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(bad, setup_only=1)
    assert e.value.code == mfs.ERR_INVALID
    with pytest.raises(mfs.MfsError):
        mfs.Solver(s, setup_only=1, restart=0)
    with pytest.raises(mfs.MfsError):
        mfs.Solver(s, setup_only=1, precond="simple", simple_pred=2)
    with pytest.raises(mfs.MfsError):
        mfs.Solver(s, setup_only=1, precond="bgs_gs")  # needs the Gauss-Seidel smoother
    with pytest.raises(mfs.MfsError):
        mfs.Solver(s, setup_only=1, smoother="gs", gs_omega=2.0)


@pytest.mark.parametrize("user", [False, True])
@pytest.mark.parametrize("pc", ["bgs_amg", "amg_bgs"])
def test_dirichlet_flags_and_user_nullspace_match_oracle(user, pc):
    """Symmetry conditions (1-3 held components per node) flagged per dof,
    rigid-body modes built in or given by the caller: aggregates, P, R and
    the Galerkin blocks of the host setup equal the oracle's; flagged dofs
    have zero prolongator rows."""
    s = inputs.roller_box(ne=7, user_nullspace=user)
    kw = dict(max_levels=3, coarse_max=100)
    lib = mfs.Solver(s, precond=pc, setup_only=1, seed=7, **kw)
    A = s.scipy_blocks()
    specs = [amg.FieldSpec.of(f) for f in s.fields]
    assert specs[0].dirichlet is not None and (specs[0].kind == "user") == user
    M = precond.Preconditioner(A, specs, precond.Params(pc, seed=7, **kw))
    lv = M.groups[0].levels
    assert lib.num_levels(0) == len(lv) == 3
    for l in range(len(lv)):
        for i in range(s.nfields):
            assert _rel(lib.export_csr("A", 0, l, i, i), lv[l][i].A) < TOL
            if l < len(lv) - 1:
                assert np.array_equal(lib.export_array("agg", 0, l, i), lv[l][i].agg)
                P = lib.export_csr("P", 0, l, i)
                assert _rel(P, lv[l][i].P) < TOL
                if l == 0:
                    assert abs(P[np.nonzero(s.fields[i].dirichlet_dofs)[0]]).max() == 0.0
    # the corner node holds all three components and is left unaggregated
    assert lib.export_array("agg", 0, 0, 0)[0] == -1
    lib.close()


def test_dirichlet_flag_on_a_non_identity_row_is_refused():
    s = inputs.coupled_box_3d(ne=4, nfields=2)
    m = np.zeros(s.fields[0].ndofs, bool)
    m[3 * 31 + 1] = True  # node (1, 1, 1), interior: its row is not an identity row
    s.fields[0].dirichlet_dofs = m
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(s, setup_only=1, max_levels=2, coarse_max=10)
    assert e.value.code == mfs.ERR_INVALID and "identity" in str(e.value)


def test_user_nullspace_shape_is_checked():
    s = inputs.coupled_box_3d(ne=4, nfields=2)
    s.fields[1].nullspace = "user"
    s.fields[1].ns_user = np.ones((s.fields[1].ndofs, 4))  # 4 vectors: no 1x4 block kernels
    with pytest.raises(mfs.MfsError) as e:
        mfs.Solver(s, setup_only=1, max_levels=2, coarse_max=10)
    assert e.value.code == mfs.ERR_INVALID
