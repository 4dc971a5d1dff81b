"""Pins for the oracle's smoothers and V-cycle (Algorithm 1), CPU only.

Multicolour Gauss-Seidel (the GPU analogue of Sec. 7.1's DD(GS(omega))): the
greedy colouring is valid and equals the closed-form parity colouring of
structured Q1 grids; one sweep equals SOR(omega) written as a matrix splitting
in the colour ordering (forward: D/omega + L, backward: D/omega + U); the
V-cycle with forward pre- and backward post-smoothing is symmetric and
contracting; the single-level BGS(GS) preconditioner loses iterations under
refinement while BGS(AMG) does not (Sec. 7.1 tables)."""
import numpy as np
import scipy.sparse as sp
import pytest

from oracle import amg
from oracle import krylov, precond
from oracle.cycles import chebyshev, gauss_seidel, jacobi, node_colors, vcycle, SmootherParams
from paper_1605_01522_gb300 import inputs


def _spd(ne=6):
    s = inputs.thermo_elastic_2d(ne=ne)
    return s, {k: v.to_scipy() for k, v in s.blocks.items()}


def _dense_op(f, n):
    return np.column_stack([f(e) for e in np.eye(n)])


def _cheb_poly(t, lo, hi, degree):
    """Closed form of the Chebyshev error polynomial p(t) = T_k((hi+lo-2t)/(hi-lo)) / T_k((hi+lo)/(hi-lo))."""
    T = lambda k, x: np.cos(k * np.arccos(x)) if abs(x) <= 1 else np.cosh(k * np.arccosh(abs(x))) * (np.sign(x) ** k)
    return np.array([T(degree, (hi + lo - 2 * ti) / (hi - lo)) for ti in t]) / T(degree, (hi + lo) / (hi - lo))


@pytest.mark.parametrize("degree", [1, 2, 3, 4])
def test_chebyshev_error_propagation_is_chebyshev_polynomial(degree):
    s, A = _spd(5)
    M = A[(1, 1)]
    n = M.shape[0]
    dinv = 1.0 / M.diagonal()
    Md = M.toarray()
    Dh = np.diag(np.sqrt(dinv))
    w, U = np.linalg.eigh(Dh @ Md @ Dh)
    lam = w.max()
    # E = error propagation on e = x - x*: smoothing with b = 0 maps x -> E x
    E = _dense_op(lambda e: chebyshev(M, dinv, lam, np.zeros(n), e, degree), n)
    lo, hi = lam / 30.0, 1.1 * lam
    p = _cheb_poly(w, lo, hi, degree)
    # D^-1 A = D^-1/2 (U w U^T) D^1/2, so E = D^-1/2 U p(w) U^T D^1/2
    Dm = np.diag(1.0 / np.sqrt(dinv))
    E_ref = Dh @ U @ np.diag(p) @ U.T @ Dm
    assert np.allclose(E, E_ref, atol=1e-12)
    # on [lo, hi] the polynomial is bounded by its value at the interval end
    inside = (w >= lo) & (w <= hi)
    assert np.all(np.abs(p[inside]) <= abs(_cheb_poly([hi], lo, hi, degree)[0]) + 1e-14)


def test_jacobi_matches_definition():
    s, A = _spd(4)
    M = A[(1, 1)]
    n = M.shape[0]
    dinv = 1.0 / M.diagonal()
    E = _dense_op(lambda e: jacobi(M, dinv, np.zeros(n), e, 0.5, 2), n)
    J = np.eye(n) - 0.5 * np.diag(dinv) @ M.toarray()
    assert np.allclose(E, J @ J, atol=1e-14)


def _hier(A, s, levels, fi=0, coarse_max=0):
    spec = [amg.FieldSpec.of(s.fields[fi])]
    lv = amg.build_group([A[(fi, fi)]], spec, levels, coarse_max, 5)
    return lv, amg.DenseLU(lv[-1][0].A)


def test_vcycle_single_level_is_direct_solve():
    s, A = _spd(6)
    lv, lu = _hier(A, s, 1)
    b = np.random.default_rng(1).standard_normal(A[(0, 0)].shape[0])
    x = vcycle(lv, 0, lu, b, SmootherParams())
    assert np.allclose(A[(0, 0)] @ x, b, atol=1e-10)


@pytest.mark.parametrize("levels,fi", [(2, 0), (3, 0), (2, 1), (3, 1)])
def test_vcycle_is_symmetric_and_convergent(levels, fi):
    s, A = _spd(10)
    lv, lu = _hier(A, s, levels, fi)
    M = A[(fi, fi)]
    n = M.shape[0]
    B = _dense_op(lambda e: vcycle(lv, 0, lu, e, SmootherParams()), n)
    # same polynomial smoother before and after, R = P^T: symmetric operator
    assert np.abs(B - B.T).max() <= 1e-11 * np.abs(B).max()
    # error propagation I - B A contracts in the A-norm
    Md = M.toarray()
    L = np.linalg.cholesky(Md)
    E = np.eye(n) - B @ Md
    rho = np.linalg.norm(L.T @ E @ np.linalg.inv(L.T), 2)
    assert rho < 0.9
    assert len(lv) == levels


def test_vcycle_two_level_matches_textbook_two_grid():
    s, A = _spd(8)
    lv, lu = _hier(A, s, 2)
    M = A[(0, 0)].toarray()
    n = M.shape[0]
    fl = lv[0][0]
    P = fl.P.toarray()
    Ac = P.T @ M @ P
    sp_ = SmootherParams()
    S = _dense_op(lambda e: chebyshev(A[(0, 0)], fl.dinv, fl.lam, np.zeros(n), e, 2), n)
    # two-grid error propagation: S (I - P Ac^-1 P^T A) S
    E_ref = S @ (np.eye(n) - P @ np.linalg.solve(Ac, P.T @ M)) @ S
    B = _dense_op(lambda e: vcycle(lv, 0, lu, e, sp_), n)
    assert np.allclose(np.eye(n) - B @ M, E_ref, atol=1e-10)


def _grid_matrix(ne, dim, b):
    """Neumann Q1 Laplacian + mass on a full structured grid (no Dirichlet
    nodes), b identical components per node."""
    g = inputs._Grid(ne, dim)
    _, Kl, Me, _ = inputs.q1_element_matrices(dim, 1.0 / ne)
    nl = Kl.shape[0]
    Kb = np.zeros((nl * b, nl * b))
    for a in range(nl):
        for c in range(nl):
            Kb[a * b:(a + 1) * b, c * b:(c + 1) * b] = (Kl[a, c] + Me[a, c]) * np.eye(b) + 0.1 * (a == c)
    return g, g.bsr(g.assemble(Kb, b, b), b, b).to_scipy()


@pytest.mark.parametrize("dim,b,ne", [(2, 1, 7), (2, 2, 6), (3, 1, 4), (3, 3, 3)])
def test_node_colors_are_the_parity_colouring_on_grids(dim, b, ne):
    g, A = _grid_matrix(ne, dim, b)
    col = node_colors(A, b)
    parity = sum((g.ijk[:, d] % 2) << d for d in range(dim))
    assert np.array_equal(col, parity)
    assert col.max() + 1 == 2 ** dim


def _random_block_matrix(n, b, seed, density=0.05):
    rng = np.random.default_rng(seed)
    S = sp.random(n, n, density=density, random_state=np.random.RandomState(seed), format="csr")
    S = S + S.T
    A = sp.kron(S, np.ones((b, b))).tocsr()
    A.data = rng.standard_normal(A.data.shape) * 0.3
    rows = np.abs(A).sum(1).A.ravel()
    A = (A + sp.diags(rows + 1.0 + rng.random(n * b))).tocsr()
    return A


@pytest.mark.parametrize("b,seed", [(1, 1), (2, 2), (3, 3)])
def test_node_colors_valid_and_first_fit(b, seed):
    A = _random_block_matrix(60, b, seed)
    col = node_colors(A, b)
    Ab = A.tocoo()
    i, j = Ab.row // b, Ab.col // b
    off = i != j
    assert np.all(col[i[off]] != col[j[off]])
    # first fit: every colour below a node's colour is held by a lower-numbered neighbour
    adj = [set() for _ in range(60)]
    for p, q in zip(i[off], j[off]):
        adj[p].add(q)
        adj[q].add(p)
    for v in range(60):
        assert set(range(col[v])) <= {col[u] for u in adj[v] if u < v}


def _sor_reference(A, b, col, x0, rhs, omega, backward):
    """x0 + (D/omega + T)^-1 (rhs - A x0), T the strict lower (forward) or
    upper (backward) triangle of A in the colour-major ordering."""
    n = A.shape[0] // b
    order = np.lexsort((np.arange(n), col))  # colour, then node
    perm = (order[:, None] * b + np.arange(b)[None, :]).ravel()
    Ap = A.toarray()[np.ix_(perm, perm)]
    T = np.triu(Ap, 1) if backward else np.tril(Ap, -1)
    Mp = np.diag(np.diag(Ap)) / omega + T
    r = (rhs - A @ x0)[perm]
    dx = np.zeros_like(x0)
    dx[perm] = np.linalg.solve(Mp, r)
    return x0 + dx


@pytest.mark.parametrize("b,seed,omega", [(1, 4, 1.0), (2, 5, 0.79), (3, 6, 0.69)])
@pytest.mark.parametrize("backward", [False, True])
def test_gauss_seidel_sweep_is_sor_splitting(b, seed, omega, backward):
    A = _random_block_matrix(50, b, seed)
    fl = amg.FieldLevel(A, b)
    rng = np.random.default_rng(seed)
    x0, rhs = rng.standard_normal(A.shape[0]), rng.standard_normal(A.shape[0])
    x1 = gauss_seidel(fl, rhs, x0, omega, 1, backward=backward)
    ref = _sor_reference(A, b, fl.colors, x0, rhs, omega, backward)
    assert np.allclose(x1, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    x2 = gauss_seidel(fl, rhs, x0, omega, 2, backward=backward)
    ref2 = _sor_reference(A, b, fl.colors, ref, rhs, omega, backward)
    assert np.allclose(x2, ref2, rtol=1e-12, atol=1e-12 * np.abs(ref2).max())


@pytest.mark.parametrize("levels,fi", [(2, 0), (3, 0), (3, 1)])
def test_vcycle_with_gauss_seidel_is_symmetric_and_convergent(levels, fi):
    s, A = _spd(8)
    lv, lu = _hier(A, s, levels, fi)
    M = A[(fi, fi)]
    n = M.shape[0]
    sp_ = SmootherParams("gs", omega=0.79, sweeps=1)
    B = _dense_op(lambda e: vcycle(lv, 0, lu, e, sp_), n)
    assert np.abs(B - B.T).max() <= 1e-11 * np.abs(B).max()
    Md = M.toarray()
    L = np.linalg.cholesky(Md)
    E = np.eye(n) - B @ Md
    assert np.linalg.norm(L.T @ E @ np.linalg.inv(L.T), 2) < 0.9


def test_single_level_bgs_gs_is_not_scalable():
    """Sec. 7.1: the single-level BGS(DD(GS)) needs many more iterations as the
    mesh is refined; BGS(AMG) with the same Gauss-Seidel smoother does not."""
    gs = SmootherParams("gs", omega=0.79, sweeps=1)
    its = {"bgs_gs": [], "bgs_amg": []}
    for ne in (8, 16, 32):
        s = inputs.thermo_elastic_2d(ne=ne)
        A = {k: v.to_scipy() for k, v in s.blocks.items()}
        D = precond.assemble(A, 2)
        specs = [amg.FieldSpec.of(f) for f in s.fields]
        for pc in its:
            Mp = precond.Preconditioner(A, specs, precond.Params(pc, max_levels=4, coarse_max=50, smoother=gs))
            r = krylov.fgmres(lambda v: D @ v, Mp, s.rhs, 1e-8, 50, maxiter=1000)
            assert r.converged
            its[pc].append(r.iters)
    assert its["bgs_gs"][-1] >= 3 * its["bgs_gs"][0]
    assert its["bgs_amg"][-1] <= 2 * its["bgs_amg"][0] + 2
    assert its["bgs_amg"][-1] < its["bgs_gs"][-1]


def test_node_colors_chain_beyond_int32_pairs():
    """A 60,000-node chain (node pairs beyond 2^31): colours alternate 0, 1."""
    n = 60000
    A = sp.diags([np.full(n - 1, -1.0), np.full(n, 4.0), np.full(n - 1, -1.0)], [-1, 0, 1]).tocsr()
    col = node_colors(A, 1)
    assert np.array_equal(col, np.arange(n) % 2)
