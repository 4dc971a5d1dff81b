"""Pins for the oracle's block preconditioners and FGMRES (CPU only).

BGS with exact block solves must equal a dense block-triangular solve
(Sec. 4.1, M_BGS); SIMPLE with A~_11 = A_11 and exact inner solves must
reproduce A^-1 (Sec. 4.2: M_SIMPLE then equals A); AMG(BGS) must reduce to the
single-field V-cycle for one field and to BGS(AMG)'s block-diagonal V-cycles
without coupling, and its coarse blocks must equal dense R_i A_ij P_j
(Sec. 4.3); SIMPLE(AMG(BGS)) must reduce to SIMPLE(BGS(AMG)) for one or
uncoupled predictor fields, and the constraint saddle's Schur group must be
a direct solve (Sec. 6.3); AMG(SIMPLE) must reduce to BGS(AMG) without coupling and its
level smoother, with converged inner solves, must apply M_SIMPLE^-1 (Sec. 4.2
factorisation on the level); FGMRES must reach the dense solution and take
one iteration with an exact preconditioner.
"""
import numpy as np
import scipy.sparse as sp
import pytest

from oracle import amg, precond, krylov
from oracle.cycles import SmootherParams, vcycle
from paper_1605_01522_gb300 import inputs


def _sys2(ne=6, alpha=1e-1, beta=5e-2):
    s = inputs.thermo_elastic_2d(ne=ne, alpha=alpha, beta=beta)
    return s, {k: v.to_scipy() for k, v in s.blocks.items()}


def _sys3(ne=3):
    s = inputs.coupled_box_3d(ne=ne, nfields=3, alpha=0.2, beta=0.1)
    return s, {k: v.to_scipy() for k, v in s.blocks.items()}


def _cons(ne=3):
    s = inputs.constrained_box(ne=ne, nfields=3, alpha=0.2, beta=0.1)
    return s, {k: v.to_scipy() for k, v in s.blocks.items()}


def _dense(blocks, nf):
    return precond.assemble(blocks, nf).toarray()


def _block_tri(blocks, nf, sizes, lower):
    D = _dense(blocks, nf)
    off = np.concatenate([[0], np.cumsum(sizes)])
    M = D.copy()
    for i in range(nf):
        for j in range(nf):
            if (lower and j > i) or (not lower and j < i):
                M[off[i]:off[i + 1], off[j]:off[j + 1]] = 0.0
    return M


@pytest.mark.parametrize("maker", [_sys2, _sys3])
@pytest.mark.parametrize("order", ["fwd", "bwd", "sym"])
def test_bgs_exact_blocks_is_block_triangular_solve(maker, order):
    s, A = maker()
    nf = s.nfields
    sizes = [f.ndofs for f in s.fields]
    solvers = [precond.DirectLeaf(A[(i, i)]) for i in range(nf)]
    bgs = precond.BGS(A, nf, solvers, order, 1)
    b = np.random.default_rng(2).standard_normal(sum(sizes))
    x = np.concatenate(bgs(precond.split(b, sizes)))
    D = _dense(A, nf)
    if order == "fwd":
        ref = np.linalg.solve(_block_tri(A, nf, sizes, True), b)
    elif order == "bwd":
        ref = np.linalg.solve(_block_tri(A, nf, sizes, False), b)
    else:
        x1 = np.linalg.solve(_block_tri(A, nf, sizes, True), b)
        ref = x1 + np.linalg.solve(_block_tri(A, nf, sizes, False), b - D @ x1)
    assert np.allclose(x, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_bgs_exact_blocks_zero_coupling_is_exact():
    s, A = _sys2()
    A0 = {k: v for k, v in A.items() if k[0] == k[1]}
    sizes = [f.ndofs for f in s.fields]
    bgs = precond.BGS(A0, 2, [precond.DirectLeaf(A0[(i, i)]) for i in range(2)], "bwd", 1)
    D = _dense(A0, 2)
    b = np.random.default_rng(3).standard_normal(sum(sizes))
    r = krylov.fgmres(lambda v: D @ v, lambda v: np.concatenate(bgs(precond.split(v, sizes))), b, 1e-10, 10)
    assert r.iters == 1 and r.relres < 1e-12


@pytest.mark.parametrize("maker,groups", [(_sys2, [0, 1]), (_sys3, [0, 0, 1]), (_sys3, [0, 1, 1]),
                                          (_cons, [0, 0, 0, 1])])
def test_simple_with_exact_a11_reproduces_inverse(maker, groups):
    s, A = maker()
    nf = s.nfields
    sizes = [f.ndofs for f in s.fields]
    g1 = [i for i in range(nf) if groups[i] == 0]
    g2 = [i for i in range(nf) if groups[i] == 1]
    D = _dense(A, nf)
    off = np.concatenate([[0], np.cumsum(sizes)])
    idx = lambda g: np.concatenate([np.arange(off[i], off[i + 1]) for i in g])
    i1, i2 = idx(g1), idx(g2)
    A11, A12, A21, A22 = D[np.ix_(i1, i1)], D[np.ix_(i1, i2)], D[np.ix_(i2, i1)], D[np.ix_(i2, i2)]
    S = A22 - A21 @ np.linalg.solve(A11, A12)
    s1 = [sizes[i] for i in g1]
    s2 = [sizes[i] for i in g2]
    pred = lambda b1: precond.split(np.linalg.solve(A11, np.concatenate(b1)), s1)
    schur = lambda b2: precond.split(np.linalg.solve(S, np.concatenate(b2)), s2)
    a11inv = lambda t: precond.split(np.linalg.solve(A11, np.concatenate(t)), s1)
    op = precond.SIMPLE(A, g1, g2, pred, schur, a11inv)
    b = np.random.default_rng(4).standard_normal(sum(sizes))
    x = np.concatenate(op(precond.split(b, sizes)))
    assert np.allclose(D @ x, b, atol=1e-9 * np.abs(b).max())


@pytest.mark.parametrize("approx", ["absrowsum", "diag"])
def test_simple_with_diagonal_a11_matches_factorised_matrix(approx):
    """With exact inner solves the SIMPLE step applies M_SIMPLE^-1, where
    M_SIMPLE = [A11 0; A21 S~][I A~11^-1 A12; 0 I]."""
    s, A = _sys3()
    nf = 3
    sizes = [f.ndofs for f in s.fields]
    g1, g2 = [0, 1], [2]
    dt = precond.simple_dtilde(A, g1, approx)
    St = precond.simple_schur(A, g1, g2, dt)
    D = _dense(A, nf)
    n1 = sizes[0] + sizes[1]
    A11, A12, A21 = D[:n1, :n1], D[:n1, n1:], D[n1:, :n1]
    dtv = np.concatenate(dt)
    if approx == "absrowsum":
        assert np.allclose(dtv, np.abs(A11).sum(1))
    else:
        assert np.allclose(dtv, np.diag(A11))
    Sd = St[(0, 0)].toarray()
    assert np.allclose(Sd, D[n1:, n1:] - A21 @ np.diag(1 / dtv) @ A12, atol=1e-13)
    M = np.block([[A11, np.zeros_like(A12)], [A21, Sd]]) @ np.block(
        [[np.eye(n1), np.diag(1 / dtv) @ A12], [np.zeros_like(A21), np.eye(sizes[2])]])
    pred = lambda b1: precond.split(np.linalg.solve(A11, np.concatenate(b1)), sizes[:2])
    schur = lambda b2: [np.linalg.solve(Sd, b2[0])]
    op = precond.SIMPLE(A, g1, g2, pred, schur, lambda t: [ti / d for ti, d in zip(t, dt)])
    b = np.random.default_rng(5).standard_normal(sum(sizes))
    x = np.concatenate(op(precond.split(b, sizes)))
    assert np.allclose(x, np.linalg.solve(M, b), rtol=1e-9, atol=1e-9)


def test_amg_bgs_single_field_equals_vcycle():
    s, A = _sys2(ne=10)
    specs = [amg.FieldSpec.of(s.fields[0])]
    prm = precond.Params("amg_bgs", max_levels=3, coarse_max=0)
    mono = precond.MonoAMG({(0, 0): A[(0, 0)]}, specs, prm, 1)
    b = np.random.default_rng(6).standard_normal(A[(0, 0)].shape[0])
    lv = mono.grp.levels
    x1 = mono([b])[0]
    x2 = vcycle(lv, 0, amg.DenseLU(lv[-1][0].A), b, prm.smoother)
    assert np.array_equal(x1, x2)


def test_amg_bgs_without_coupling_equals_bgs_amg():
    s, A = _sys2(ne=10)
    A0 = {k: v for k, v in A.items() if k[0] == k[1]}
    specs = [amg.FieldSpec.of(f) for f in s.fields]
    sizes = [f.ndofs for f in s.fields]
    b = np.random.default_rng(7).standard_normal(sum(sizes))
    za = precond.Preconditioner(A0, specs, precond.Params("amg_bgs", max_levels=3, coarse_max=0))(b)
    zb = precond.Preconditioner(A0, specs, precond.Params("bgs_amg", max_levels=3, coarse_max=0))(b)
    assert np.allclose(za, zb, rtol=1e-12, atol=1e-13 * np.abs(zb).max())


def test_amg_bgs_coarse_blocks_are_blockwise_galerkin():
    s, A = _sys3(ne=5)
    specs = [amg.FieldSpec.of(f) for f in s.fields]
    prm = precond.Params("amg_bgs", max_levels=3, coarse_max=0)
    mono = precond.MonoAMG(A, specs, prm, 3)
    lv = mono.grp.levels
    for l in range(len(lv) - 1):
        for (i, j), M in mono.A[l].items():
            ref = lv[l][i].P.toarray().T @ M.toarray() @ lv[l][j].P.toarray()
            assert np.allclose(mono.A[l + 1][(i, j)].toarray(), ref, atol=1e-14 * max(1, np.abs(ref).max()))
    # the coupled coarse operator equals R A P with block-diagonal transfers
    P = sp.block_diag([lv[0][i].P for i in range(3)]).toarray()
    D = _dense(A, 3)
    assert np.allclose(_dense(mono.A[1], 3), P.T @ D @ P, atol=1e-12)


def test_amg_simple_without_coupling_equals_bgs_amg():
    """No coupling: S~^l = A^l_22, the predictor is field 1's smoother and the
    level smoother is the block-diagonal one of BGS(AMG)'s V-cycles."""
    s, A = _sys2(ne=10)
    A0 = {k: v for k, v in A.items() if k[0] == k[1]}
    specs = [amg.FieldSpec.of(f) for f in s.fields]
    sizes = [f.ndofs for f in s.fields]
    b = np.random.default_rng(8).standard_normal(sum(sizes))
    for approx in ("absrowsum", "diag"):
        za = precond.Preconditioner(A0, specs, precond.Params("amg_simple", max_levels=3, coarse_max=0,
                                                             simple_approx=approx))(b)
        zb = precond.Preconditioner(A0, specs, precond.Params("bgs_amg", max_levels=3, coarse_max=0))(b)
        assert np.allclose(za, zb, rtol=1e-12, atol=1e-13 * np.abs(zb).max())


def _chain(n, diag, off):
    return sp.diags([np.full(n - 1, off), np.full(n, diag), np.full(n - 1, off)], [-1, 0, 1]).tocsr()


@pytest.mark.parametrize("approx", ["absrowsum", "diag"])
def test_amg_simple_level_smoother_applies_simple_factorisation(approx):
    """Level smoother of AMG(SIMPLE) with converged single-field solves (60
    Jacobi sweeps on diagonally dominant blocks): d = M_SIMPLE^-1 r with
    M_SIMPLE = [A11 0; A21 S~][I A~11^-1 A12; 0 I], S~ = A22 - A21 A~11^-1 A12.
    A12 and A21 are unrelated (not transposes), so swapped or transposed
    coupling blocks, a wrong sign or a dropped term change the result."""
    n = 40
    rng = np.random.default_rng(9)
    A = {(0, 0): _chain(n, 4.0, -1.0), (1, 1): _chain(n, 5.0, -1.0),
         (0, 1): sp.random(n, n, density=0.08, random_state=np.random.RandomState(1), format="csr") * 0.6,
         (1, 0): sp.random(n, n, density=0.08, random_state=np.random.RandomState(2), format="csr") * -0.5}
    specs = [amg.FieldSpec(1, 1, "const"), amg.FieldSpec(1, 1, "const")]
    prm = precond.Params("amg_simple", max_levels=2, coarse_max=0, simple_approx=approx,
                         smoother=SmootherParams("jacobi", omega=1.0, sweeps=60))
    mono = precond.MonoAMGSimple(A, specs, prm, 2, [0], [1])
    D = _dense(A, 2)
    A11, A12, A21, A22 = D[:n, :n], D[:n, n:], D[n:, :n], D[n:, n:]
    dt = np.abs(A11).sum(1) if approx == "absrowsum" else np.diag(A11)
    St = A22 - A21 @ np.diag(1 / dt) @ A12
    M = np.block([[A11, np.zeros((n, n))], [A21, St]]) @ np.block(
        [[np.eye(n), np.diag(1 / dt) @ A12], [np.zeros((n, n)), np.eye(n)]])
    r = rng.standard_normal(2 * n)
    x = mono.smooth(0, [r[:n], r[n:]], [np.zeros(n), np.zeros(n)])
    assert np.allclose(np.concatenate(x), np.linalg.solve(M, r), rtol=1e-10, atol=1e-10)


def test_constrained_saddle_structure_and_direct_schur():
    """Constraint field of the lung-like box (Sec. 6.3): zero diagonal block,
    A_0C = A_C0^T with unit patch weights; BGS-type setups must refuse the zero
    diagonal; SIMPLE's Schur group (4 dofs <= coarse_max) is one level, so its
    solve is the dense solve with S~ = -A_C0 A~_00^-1 A_0C."""
    s, A = _cons(ne=4)
    specs = [amg.FieldSpec.of(f) for f in s.fields]
    assert A[(3, 3)].nnz == 0 and abs(A[(0, 3)] - A[(3, 0)].T).max() == 0
    assert np.allclose(np.asarray(A[(3, 0)].sum(1)).ravel(), 1.0)
    for pc in ("bgs_amg", "amg_bgs", "amg_simple"):
        with pytest.raises(ValueError):
            precond.Preconditioner(A, specs, precond.Params(pc, max_levels=3, coarse_max=20))
    M = precond.Preconditioner(A, specs, precond.Params("simple", max_levels=3, coarse_max=20))
    assert len(M.groups[1].levels) == 1
    S = M.schur_blocks[(0, 0)].toarray()
    D = _dense(A, 4)
    n1 = sum(f.ndofs for f in s.fields[:3])
    dt = np.abs(D[:n1, :n1]).sum(1)
    assert np.allclose(S, -D[n1:, :n1] @ np.diag(1 / dt) @ D[:n1, n1:], rtol=1e-12, atol=0)
    assert np.all(np.linalg.eigvalsh(0.5 * (S + S.T)) < 0)
    r = np.random.default_rng(10).standard_normal(S.shape[0])
    leaf = M.groups[1].leaf(0)
    assert np.allclose(leaf(r), np.linalg.solve(S, r), rtol=1e-12, atol=1e-12 * np.abs(np.linalg.solve(S, r)).max())


def test_simple_amg_bgs_predictor_reductions():
    """SIMPLE(AMG(BGS)) equals SIMPLE(BGS(AMG)) when the predictor is one field
    (the monolithic V-cycle of one field is the single-field V-cycle) and when
    the predictor fields do not couple (AMG(BGS) without coupling is BGS(AMG))."""
    s, A = _sys3(ne=5)
    specs = [amg.FieldSpec.of(f) for f in s.fields]
    kw = dict(max_levels=3, coarse_max=40)
    b = np.random.default_rng(11).standard_normal(sum(f.ndofs for f in s.fields))
    for groups, blocks in (([0, 1, 1], A),
                           ([0, 0, 1], {k: v for k, v in A.items() if set(k) != {0, 1}})):
        za = precond.Preconditioner(blocks, specs, precond.Params("simple", simple_group=groups,
                                                                  simple_pred="amg_bgs", **kw))(b)
        zb = precond.Preconditioner(blocks, specs, precond.Params("simple", simple_group=groups, **kw))(b)
        assert np.allclose(za, zb, rtol=1e-12, atol=1e-13 * np.abs(zb).max())
    # with coupling inside the predictor group the two differ
    za = precond.Preconditioner(A, specs, precond.Params("simple", simple_group=[0, 0, 1], simple_pred="amg_bgs", **kw))(b)
    zb = precond.Preconditioner(A, specs, precond.Params("simple", simple_group=[0, 0, 1], **kw))(b)
    assert not np.allclose(za, zb, rtol=1e-6)


def test_fgmres_unpreconditioned_reaches_dense_solution():
    rng = np.random.default_rng(8)
    n = 60
    M = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n)
    r = krylov.fgmres(lambda v: M @ v, lambda v: v, b, 1e-10, restart=7, maxiter=500)
    x_ref = np.linalg.solve(M, b)
    assert r.converged and r.restarts > 0
    assert np.linalg.norm(r.x - x_ref) <= 1e-8 * np.linalg.norm(x_ref) * np.linalg.cond(M)
    h = np.array(r.history)
    assert np.all(np.diff(h) <= 1e-12)


def test_fgmres_exact_preconditioner_one_iteration_and_estimate():
    s, A = _sys2(ne=5)
    D = _dense(A, 2)
    b = s.rhs
    r = krylov.fgmres(lambda v: D @ v, lambda v: np.linalg.solve(D, v), b, 1e-8, 50)
    assert r.iters == 1 and r.relres < 1e-12
    Mp = precond.Preconditioner(A, [amg.FieldSpec.of(f) for f in s.fields],
                                precond.Params("bgs_amg", max_levels=2, coarse_max=0))
    r2 = krylov.fgmres(lambda v: D @ v, Mp, b, 1e-8, 50)
    assert r2.converged
    # Givens estimate agrees with the true residual of the final iterate
    assert abs(r2.est - r2.relres) <= 1e-6 * r2.relres + 1e-14


@pytest.mark.parametrize("pc", ["bgs_amg", "amg_bgs", "simple", "amg_simple"])
def test_preconditioned_solve_iterations_grow_mildly(pc):
    """Trend of Sec. 7 (weak-scaling tables): multilevel block preconditioners
    keep the iteration count nearly flat under refinement."""
    its = []
    for ne in (8, 16, 32):
        s = inputs.thermo_elastic_2d(ne=ne)
        A = {k: v.to_scipy() for k, v in s.blocks.items()}
        D = precond.assemble(A, 2)
        Mp = precond.Preconditioner(A, [amg.FieldSpec.of(f) for f in s.fields],
                                    precond.Params(pc, max_levels=4, coarse_max=50))
        r = krylov.fgmres(lambda v: D @ v, Mp, s.rhs, 1e-8, 50, maxiter=400)
        assert r.converged
        its.append(r.iters)
    assert its[-1] <= 2 * its[0] + 2
