"""Pins for the oracle's smoothed-aggregation setup (CPU only).

Each check is fixed by mathematics or a published value, not by re-running the
oracle's own formula: the published SplitMix64 outputs, the characterisation
of the lexicographically-first maximal independent set, exact reproduction of
the near-nullspace by the tentative prolongator, uniqueness of the QR
factorisation with positive diagonal, symmetry of Galerkin products, the
energy decrease of prolongator smoothing and a dense eigenvalue solver.
The strength graph at theta > 0 is recomputed by brute force from dense node
blocks (numpy's Frobenius norm pair by pair, then the union with the
transpose) on Q1 elasticity / diffusion blocks and on non-symmetric random
block matrices; squared norms, a max-norm and a missing symmetrisation each
fail that comparison.
Petrov-Galerkin transfers (Sala & Tuminaro 2008): each column parameter is the
minimiser of its D^-1-norm objective (checked by brute force), row parameters
are the column minimum over the row pattern, P keeps the kernel of a
conservative convection-diffusion operator, R = P^T for a symmetric operator
and not otherwise, and the V-cycle needs fewer iterations than with
P^T-restriction on a convection-dominated-enough problem.
"""
import os

import numpy as np
import scipy.sparse as sp
import pytest

from oracle import amg
from oracle.rng import splitmix64, uniform01
from paper_1605_01522_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _neumann(dim, ne, kind):
    """Q1 matrix without Dirichlet rows (A annihilates its near-nullspace)."""
    g = inputs._Grid(ne, dim)
    Ke, Kl, Me, Ce = inputs.q1_element_matrices(dim, 1.0 / ne)
    if kind == "rbm":
        return g.bsr(g.assemble(Ke, dim, dim), dim, dim).to_scipy(), g
    return g.bsr(g.assemble(Kl, 1, 1), 1, 1).to_scipy(), g


def test_splitmix64_published_vector():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    assert [int(v) for v in splitmix64(1234567, 5)] == vals


def test_uniform01_range():
    u = uniform01(3, 10000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.02


def _dist2(G):
    G2 = (G @ G + G) > 0
    return G2.tolil()


@pytest.mark.parametrize("dim,ne,theta", [(2, 12, 0.0), (3, 5, 0.0), (2, 10, 0.3)])
def test_aggregation_is_lexicographically_first_mis2(dim, ne, theta):
    s = inputs.thermo_elastic_2d(ne=ne) if dim == 2 else inputs.coupled_box_3d(ne=ne, nfields=2)
    A = s.blocks[(0, 0)].to_scipy()
    G = amg.strength_graph(A, s.fields[0].b, theta)
    agg, roots, prio = amg.aggregate(G, 11)
    n = G.shape[0]
    isolated = np.diff(G.indptr) == 0
    # Dirichlet nodes are exactly the isolated ones
    d = np.zeros(n, bool)
    d[s.fields[0].dirichlet_nodes] = True
    if theta == 0.0:
        assert np.array_equal(isolated, d)
    H = ((G @ G + G) > 0).astype(int).tolil()
    H.setdiag(0)
    H = H.tocsr()
    isroot = np.zeros(n, bool)
    isroot[roots] = True
    key = lambda i: (int(prio[i]), -i)
    for v in range(n):
        if isolated[v]:
            assert not isroot[v] and agg[v] == -1
            continue
        nb = H.indices[H.indptr[v]:H.indptr[v + 1]]
        higher_roots = [u for u in nb if isroot[u] and key(u) > key(v)]
        # LFMIS characterisation: v is a root iff no higher-priority root within distance 2
        assert isroot[v] == (len(higher_roots) == 0)
        if isroot[v]:
            assert not any(isroot[u] for u in nb)
        assert agg[v] >= 0
    # every aggregate contains its root, and its members are within distance 2 of it
    for a, r in enumerate(roots):
        assert agg[r] == a
        members = np.nonzero(agg == a)[0]
        nb = set(H.indices[H.indptr[r]:H.indptr[r + 1]]) | {r}
        assert set(members) <= nb
    # phase 2: each neighbour of a root belongs to that root's aggregate
    for a, r in enumerate(roots):
        assert np.all(agg[G.indices[G.indptr[r]:G.indptr[r + 1]]] == a)


def _nullspace_global(coords, b, dim, kind):
    return amg.fine_nullspace_rows(b, dim, kind, coords)


@pytest.mark.parametrize("dim,kind", [(2, "const"), (2, "rbm"), (3, "rbm"), (3, "const")])
def test_tentative_prolongator_reproduces_nullspace(dim, kind):
    ne = 10 if dim == 2 else 5
    s = inputs.thermo_elastic_2d(ne=ne) if dim == 2 else inputs.coupled_box_3d(ne=ne, nfields=2)
    fi = 0 if kind == "rbm" else 1
    f = s.fields[fi]
    A = s.blocks[(fi, fi)].to_scipy()
    G = amg.strength_graph(A, f.b, 0.0)
    agg, roots, _ = amg.aggregate(G, 5)
    k = amg.nullspace_dim(f.b, dim, kind)
    Pt, Bc = amg.tentative_prolongator(agg, len(roots), f.b, k, coords=f.coords, kind=kind, dim=dim)
    # global (uncentred) near-nullspace on aggregated dofs
    Bf = _nullspace_global(f.coords, f.b, dim, kind)
    mask = np.repeat(agg >= 0, f.b)
    # P_tent B_c spans B_f aggregate by aggregate: the uncentred modes differ
    # from the centred ones by translations, which P_tent also reproduces,
    # so project: B_f = P_tent (P_tent^T B_f) exactly on aggregated rows.
    assert np.allclose((Pt @ (Pt.T @ Bf))[mask], Bf[mask], atol=1e-12)
    # P_tent B_c reproduces the centred modes exactly
    for a in range(len(roots)):
        nodes = np.nonzero(agg == a)[0]
        dofs = (nodes[:, None] * f.b + np.arange(f.b)).ravel()
        xyz = f.coords[nodes] - f.coords[nodes].mean(0)
        Ba = amg.fine_nullspace_rows(f.b, dim, kind, xyz)
        got = Pt[dofs][:, a * k:(a + 1) * k].toarray() @ Bc[a * k:(a + 1) * k]
        assert np.allclose(got, Ba, atol=1e-13)
    # orthonormal columns, zero rows on Dirichlet dofs
    PtP = (Pt.T @ Pt).toarray()
    assert np.allclose(PtP, np.eye(PtP.shape[0]), atol=1e-13)
    assert abs(Pt[~mask]).sum() == 0.0


def test_gram_schmidt_qr_matches_unique_qr():
    rng = np.random.default_rng(0)
    for m, k in [(8, 3), (24, 6), (6, 6)]:
        B = rng.standard_normal((m, k))
        Q, R = amg.gram_schmidt_qr(B)
        Q2, R2 = np.linalg.qr(B)
        s = np.sign(np.diag(R2))
        assert np.allclose(Q, Q2 * s, atol=1e-13)
        assert np.allclose(R, s[:, None] * R2, atol=1e-13)
        assert np.allclose(np.tril(R, -1), 0.0)


def test_gram_schmidt_qr_drops_dependent_column():
    B = np.zeros((6, 3))
    B[:, 0] = 1.0
    B[:, 1] = np.arange(6)
    B[:, 2] = 2 * B[:, 0] - B[:, 1]
    Q, R = amg.gram_schmidt_qr(B)
    assert np.allclose(Q[:, 2], 0.0) and R[2, 2] == 0.0
    assert np.allclose(Q @ R, B, atol=1e-13)


@pytest.mark.parametrize("dim,kind", [(2, "rbm"), (2, "const"), (3, "rbm")])
def test_smoothed_prolongator_keeps_kernel_and_lowers_energy(dim, kind):
    ne = 8 if dim == 2 else 4
    A, g = _neumann(dim, ne, kind)
    b = dim if kind == "rbm" else 1
    spec = amg.FieldSpec(b, dim, kind, g.coords, 0.0)
    lv = amg.build_group([A], [spec], 2, 0, 3)
    fl = lv[0][0]
    Bf = amg.fine_nullspace_rows(b, dim, kind, g.coords)
    # A annihilates the near-nullspace, so the smoothed P still reproduces it
    assert np.abs(A @ Bf).max() < 1e-10
    Bc = lv[1][0].B
    # P B_c spans B_f: project with the tentative part
    G = amg.strength_graph(A, b, 0.0)
    agg, roots, _ = amg.aggregate(G, 3)
    k = amg.nullspace_dim(b, dim, kind)
    Pt, Bc2 = amg.tentative_prolongator(agg, len(roots), b, k, coords=g.coords, kind=kind, dim=dim)
    assert np.allclose(Bc, Bc2)
    C = Pt.T @ Bf
    assert np.allclose(fl.P @ C, Bf, atol=1e-10)
    # smoothing lowers the energy of every coarse basis function
    e_t = (Pt.T @ A @ Pt).diagonal()
    e_s = (fl.P.T @ A @ fl.P).diagonal()
    assert np.all(e_s <= e_t + 1e-14) and e_s.sum() < 0.9 * e_t.sum()


def test_galerkin_symmetry_and_power_lambda():
    s = inputs.thermo_elastic_2d(ne=12)
    A = {k: v.to_scipy() for k, v in s.blocks.items()}
    specs = [amg.FieldSpec.of(f) for f in s.fields]
    lv = amg.build_group([A[(0, 0)], A[(1, 1)]], specs, 3, 0, 9)
    for l in range(1, len(lv)):
        for fl in lv[l]:
            M = fl.A
            assert abs(M - M.T).max() <= 1e-14 * abs(M).max()
    for l in range(len(lv) - 1):
        for fl in lv[l]:
            DA = (sp.diags(fl.dinv) @ fl.A).toarray()
            lam_true = np.max(np.abs(np.linalg.eigvals(DA)))
            assert fl.lam <= lam_true * (1 + 1e-12)
            assert fl.lam >= 0.7 * lam_true


def test_group_levels_and_coarse_dofs():
    s = inputs.thermo_elastic_2d(ne=32)
    A = {k: v.to_scipy() for k, v in s.blocks.items()}
    specs = [amg.FieldSpec.of(f) for f in s.fields]
    lv = amg.build_group([A[(0, 0)], A[(1, 1)]], specs, 3, 0, 7)
    assert len(lv) == 3
    # RBM coarse node blocks are 3 x 3 in 2D, scalar stays scalar
    assert lv[1][0].b == 3 and lv[1][1].b == 1
    assert lv[1][0].A.shape[0] % 3 == 0
    lv2 = amg.build_group([A[(0, 0)], A[(1, 1)]], specs, 6, 400, 7)
    assert sum(fl.A.shape[0] for fl in lv2[-1]) <= 400
    assert sum(fl.A.shape[0] for fl in lv2[-2]) > 400


def _conv_diff(ne, nu, wind, dirichlet=True):
    g = inputs._Grid(ne, 3)
    h = 1.0 / ne
    _, Kl, _, _ = inputs.q1_element_matrices(3, h)
    C = inputs.q1_convection_matrix(h, wind)
    blk = {(0, 0): g.bsr(g.assemble(nu * Kl + C, 1, 1), 1, 1)}
    dn = np.nonzero(g.ijk[:, 0] == 0)[0] if dirichlet else np.zeros(0, np.int64)
    if dirichlet:
        inputs._apply_dirichlet(g, blk, 1, dn)
    return blk[(0, 0)].to_scipy(), g, dn


def _pg_parts(A, seed=7, with_bc=False):
    fl = amg.FieldLevel(A, 1)
    agg, roots, _ = amg.aggregate(amg.strength_graph(A, 1, 0.0), seed)
    Pt, Bc = amg.tentative_prolongator(agg, len(roots), 1, 1, kind="const", dim=3)
    return (fl, Pt, Bc) if with_bc else (fl, Pt)


def test_pg_column_parameters_minimise_their_objective():
    A, g, _ = _conv_diff(6, 1e-2, (0.3, 0.1, 0.0))
    fl, Pt = _pg_parts(A)
    Q, wrow, wcol = amg.pg_damping(A, fl.dinv, Pt)
    Ptd, Qd, Ad = Pt.toarray(), Q.toarray(), A.toarray()
    f = lambda j, w: np.sum((Ad @ (Ptd[:, j] - w * Qd[:, j])) ** 2 * fl.dinv)
    checked = 0
    for j in range(Pt.shape[1]):
        if wcol[j] <= 0:
            continue
        grid = wcol[j] * np.linspace(0.5, 1.5, 41)
        vals = np.array([f(j, w) for w in grid])
        assert f(j, wcol[j]) <= vals.min() * (1 + 1e-12)
        checked += 1
    assert checked >= Pt.shape[1] // 2
    # row parameters: the minimum of the column parameters over the row pattern
    thr = amg.PG_PATTERN_REL * np.abs(Q.data).max()
    for i in range(Q.shape[0]):
        cols = np.nonzero(np.abs(Qd[i]) > thr)[0]
        assert wrow[i] == (wcol[cols].min() if len(cols) else 0.0)
    assert np.all(wrow >= 0)


def test_pg_prolongator_keeps_kernel_and_restriction_is_transposed_only_if_symmetric():
    # conservative convection-diffusion without Dirichlet rows: A 1 = 0
    A, g, _ = _conv_diff(6, 1e-2, (0.3, 0.1, 0.0), dirichlet=False)
    assert np.abs(A @ np.ones(A.shape[0])).max() < 1e-14
    fl, Pt, Bc = _pg_parts(A, with_bc=True)
    P, R = amg.pg_transfers(A, fl.dinv, Pt)
    assert np.allclose(Pt @ np.ravel(Bc), 1.0, atol=1e-13)
    assert np.allclose(P @ np.ravel(Bc), 1.0, atol=1e-13)
    assert np.abs((R - P.T).toarray()).max() > 1e-6
    # symmetric operator (no wind): R = P^T
    As, g, _ = _conv_diff(6, 1e-2, (0.0, 0.0, 0.0))
    fl, Pt = _pg_parts(As)
    P, R = amg.pg_transfers(As, fl.dinv, Pt)
    assert np.abs((R - P.T).toarray()).max() <= 1e-15 * np.abs(P.data).max()


def test_pg_vcycle_beats_transposed_restriction_on_convection_diffusion():
    from oracle import krylov
    from oracle.cycles import SmootherParams, vcycle
    A, g, dn = _conv_diff(24, 1e-2, (0.2, 0.1, 0.0))
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    b[dn] = 0.0
    its = []
    for pg in (False, True):
        lv = amg.build_group([A], [amg.FieldSpec(1, 3, "const", None, 0.0, pg)], 4, 50, 7)
        lu = amg.DenseLU(lv[-1][0].A)
        r = krylov.fgmres(lambda v: A @ v, lambda v: vcycle(lv, 0, lu, v, SmootherParams()), b, 1e-8, 50,
                          maxiter=500)
        assert r.converged
        its.append(r.iters)
    assert its[1] < 0.8 * its[0], its


# ---------------------------------------------------------------------------
# Strength of connection at theta > 0, pinned by brute force over node pairs.
# The oracle forms all node-block norms at once by a sparse product
# (E^T (A .* A) E); the check below slices every dense b x b node block,
# takes its Frobenius norm with numpy.linalg.norm, applies the threshold
# ||A_IJ||_F > theta sqrt(||A_II||_F ||A_JJ||_F) pair by pair and then
# takes the union with the transpose (the symmetrised graph of the
# smoothed-aggregation setup, Sec. 3.3 after Vanek, Mandel & Brezina).
# ---------------------------------------------------------------------------

def _strength_brute(A, b, theta):
    D = A.toarray()
    nn = D.shape[0] // b
    blk = lambda I, J: D[I * b:(I + 1) * b, J * b:(J + 1) * b]
    dn = [np.linalg.norm(blk(I, I), "fro") for I in range(nn)]
    S = np.zeros((nn, nn), bool)
    for I in range(nn):
        for J in range(nn):
            if I == J:
                continue
            nij = np.linalg.norm(blk(I, J), "fro")
            if nij > 0.0 and nij > theta * np.sqrt(dn[I] * dn[J]):
                S[I, J] = True
    return S | S.T


def _random_block_matrix(nn, b, seed):
    """Non-symmetric random node-block matrix: about 15 % of the off-diagonal
    node pairs present in one direction only, block magnitudes log-uniform
    over four decades (so the threshold cuts through them), diagonal blocks
    of unit scale."""
    rng = np.random.default_rng(seed)
    D = np.zeros((nn * b, nn * b))
    for I in range(nn):
        D[I * b:(I + 1) * b, I * b:(I + 1) * b] = rng.standard_normal((b, b)) + 3.0 * np.eye(b)
        for J in range(nn):
            if J != I and rng.random() < 0.15:
                scale = 10.0 ** rng.uniform(-3.0, 1.0)
                B = scale * rng.standard_normal((b, b))
                if b > 1 and rng.random() < 0.5:  # one dominant entry: max-norm != Frobenius
                    B = np.zeros((b, b))
                    B[rng.integers(b), rng.integers(b)] = scale
                D[I * b:(I + 1) * b, J * b:(J + 1) * b] = B
    return sp.csr_matrix(D)


def _strength_cases():
    cases = []
    s2 = inputs.thermo_elastic_2d(ne=6)
    s3 = inputs.coupled_box_3d(ne=4, nfields=3, seed=1)
    for theta in (0.02, 0.3):
        cases.append((f"te2d-elast-{theta}", s2.blocks[(0, 0)].to_scipy(), 2, theta))
        cases.append((f"box-elast-{theta}", s3.blocks[(0, 0)].to_scipy(), 3, theta))
        cases.append((f"box-diff-{theta}", s3.blocks[(2, 2)].to_scipy(), 1, theta))
        for b in (1, 2, 3):
            cases.append((f"rand-b{b}-{theta}", _random_block_matrix(40, b, 7 + b), b, theta))
    return cases


@pytest.mark.parametrize("name,A,b,theta", _strength_cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_strength_graph_matches_brute_force_node_blocks(name, A, b, theta):
    G = amg.strength_graph(A, b, theta)
    S = _strength_brute(A, b, theta)
    assert np.array_equal(G.toarray() > 0, S), name
    if name.startswith("rand"):
        # the raw relation is not symmetric here, so the union matters
        D = A.toarray()
        nn = D.shape[0] // b
        raw = np.array([[I != J and np.linalg.norm(D[I*b:(I+1)*b, J*b:(J+1)*b]) > 0 for J in range(nn)]
                        for I in range(nn)])
        assert not np.array_equal(raw, raw.T)


def _mutant(kind):
    """The oracle's strength function with one planted mistake."""
    def f(A, b, theta):
        nn = A.shape[0] // b
        E = amg.node_incidence(nn, b)
        if kind == "maxnorm":
            # per node block the largest |a| instead of the Frobenius norm
            Ab = abs(A).tocoo()
            mx = {}
            for r, c, v in zip(Ab.row // b, Ab.col // b, Ab.data):
                mx[(r, c)] = max(mx.get((r, c), 0.0), v)
            rows = np.array([k[0] for k in mx])
            cols = np.array([k[1] for k in mx])
            norms = np.array(list(mx.values()))
        else:
            A2 = A.multiply(A).tocsr()
            N = (E.T @ A2 @ E).tocoo()
            rows, cols = N.row, N.col
            norms = N.data if kind == "squared" else np.sqrt(N.data)
        dn = np.zeros(nn)
        on = rows == cols
        dn[rows[on]] = norms[on]
        keep = (~on) & (norms > theta * np.sqrt(dn[rows] * dn[cols]))
        G = sp.csr_matrix((np.ones(int(keep.sum())), (rows[keep], cols[keep])), shape=(nn, nn))
        if kind != "nosym":
            G = ((G + G.T) > 0).astype(np.float64).tocsr()
        return G
    return f


@pytest.mark.parametrize("kind", ["squared", "maxnorm", "nosym"])
def test_strength_brute_force_catches_planted_mistakes(kind):
    """Each planted mistake (squared norms, max-norm for Frobenius, no
    symmetrisation) disagrees with the brute force on at least one case,
    while the unmutated form of the mutant agrees on all of them."""
    bad = _mutant(kind)
    good = _mutant("none")
    caught = False
    for name, A, b, theta in _strength_cases():
        S = _strength_brute(A, b, theta)
        assert np.array_equal(good(A, b, theta).toarray() > 0, S), name
        if not np.array_equal(bad(A, b, theta).toarray() > 0, S):
            caught = True
    assert caught, kind


# ---------------------------------------------------------------------------
# Caller-supplied near-nullspace and per-dof Dirichlet flags
# ---------------------------------------------------------------------------

def _rbm_about_origin(coords, dim):
    """Rigid-body modes of every node, rotations about the coordinate origin
    (not the aggregate centroid the built-in kind uses)."""
    m = coords.shape[0]
    if dim == 2:
        B = np.zeros((m, 2, 3))
        B[:, 0, 0] = B[:, 1, 1] = 1.0
        B[:, 0, 2], B[:, 1, 2] = -coords[:, 1], coords[:, 0]
        return B.reshape(2 * m, 3)
    x, y, z = coords[:, 0], coords[:, 1], coords[:, 2]
    B = np.zeros((m, 3, 6))
    B[:, 0, 0] = B[:, 1, 1] = B[:, 2, 2] = 1.0
    B[:, 1, 3], B[:, 2, 3] = -z, y
    B[:, 0, 4], B[:, 2, 4] = z, -x
    B[:, 0, 5], B[:, 1, 5] = -y, x
    return B.reshape(3 * m, 6)


@pytest.mark.parametrize("dim,ne", [(2, 10), (3, 5)])
def test_user_nullspace_spanning_the_rigid_body_modes_gives_the_same_prolongator(dim, ne):
    """The Gram-Schmidt Q of [translations, rotations] does not depend on the
    rotation centre (moving it adds translation components, which the
    projection on the translations removes), so rigid-body modes about the
    origin given as a user nullspace reproduce the built-in hierarchy's
    first prolongator and first coarse operator to rounding (the coarse
    nullspaces R then differ: the built-in one holds per-aggregate centred
    modes, the user one the global modes, so deeper levels differ);
    constants given as a user nullspace reproduce the constant kind exactly."""
    A, g = _neumann(dim, ne, "rbm")
    coords = g.coords
    rbm = amg.FieldSpec(dim, dim, "rbm", coords, 0.0)
    usr = amg.FieldSpec(dim, dim, "user", coords, 0.0, user=_rbm_about_origin(coords, dim))
    L1 = amg.build_group([A], [rbm], 3, 10, 5)
    L2 = amg.build_group([A], [usr], 3, 10, 5)
    assert len(L1) == len(L2) == 3
    d = abs(L1[0][0].P - L2[0][0].P).max()
    assert d <= 1e-11 * abs(L1[0][0].P).max(), d
    d = abs(L1[1][0].A - L2[1][0].A).max()
    assert d <= 1e-10 * abs(L1[1][0].A).max(), d
    # the user hierarchy's coarse nullspace carries the global modes:
    # P_tent B^1 reproduces the fine modes about the origin exactly
    Bf = _rbm_about_origin(coords, dim)
    agg = L2[0][0].agg
    Pt, Bc = amg.tentative_prolongator(agg, int(agg.max()) + 1, dim, Bf.shape[1], kind="user", user=Bf)
    assert np.array_equal(Bc, L2[1][0].B)
    assert np.abs(Pt @ Bc - Bf).max() <= 1e-12 * np.abs(Bf).max()
    S, gs = _neumann(dim, ne, "const")
    c1 = amg.build_group([S], [amg.FieldSpec(1, dim, "const", None, 0.0)], 3, 10, 5)
    c2 = amg.build_group([S], [amg.FieldSpec(1, dim, "user", None, 0.0, user=np.ones((S.shape[0], 1)))], 3, 10, 5)
    assert len(c1) == len(c2) >= 2
    for l in range(len(c1)):
        assert (c1[l][0].A != c2[l][0].A).nnz == 0


def _roller_box(ne):
    """3D elasticity with a roller face: on x = 0 only u_x is fixed (symmetric
    elimination of those dofs alone), the other faces free; returns (A, spec
    without flags, spec with flags, flagged dof mask)."""
    dim = 3
    A, g = _neumann(dim, ne, "rbm")
    A = A.tolil()
    nodes = np.nonzero(np.isclose(g.coords[:, 0], 0.0))[0]
    dofs = nodes * 3
    for d in dofs:
        A[d, :] = 0.0
        A[:, d] = 0.0
        A[d, d] = 1.0
    A = A.tocsr()
    A.eliminate_zeros()
    mask = np.zeros(A.shape[0], bool)
    mask[dofs] = True
    plain = amg.FieldSpec(3, 3, "rbm", g.coords, 0.0)
    flagged = amg.FieldSpec(3, 3, "rbm", g.coords, 0.0, dirichlet=mask)
    return A, plain, flagged, mask


def test_dirichlet_flags_zero_the_nullspace_rows_and_keep_the_dofs_fixed():
    """With per-dof Dirichlet flags the tentative prolongator has zero rows at
    the flagged dofs and reproduces the masked nullspace exactly
    (P_tent B_c = B with those rows zeroed); the smoothed P then also has zero
    rows there (identity rows of A), so a V-cycle started from zero keeps the
    flagged dofs at exactly zero when their right-hand side is zero - which
    the unflagged hierarchy does not."""
    from oracle import cycles
    A, plain, flagged, mask = _roller_box(6)
    L = amg.build_group([A], [flagged], 3, 30, 5)
    P0 = L[0][0].P
    assert abs(P0[np.nonzero(mask)[0]]).max() == 0.0
    # P_tent reproduces the masked nullspace: rebuild it the way the setup does
    agg = L[0][0].agg
    nagg = int(agg.max()) + 1
    Pt, Bc = amg.tentative_prolongator(agg, nagg, 3, 6, coords=flagged.coords, kind="rbm", dim=3, dmask=mask)
    Bm = np.zeros((A.shape[0], 6))
    for a in range(nagg):
        nodes = np.nonzero(agg == a)[0]
        xyz = flagged.coords[nodes] - flagged.coords[nodes].mean(axis=0)
        dofs = (nodes[:, None] * 3 + np.arange(3)).ravel()
        Bm[dofs] = amg.fine_nullspace_rows(3, 3, "rbm", xyz)
    Bm[mask] = 0.0
    for a in range(nagg):
        nodes = np.nonzero(agg == a)[0]
        dofs = (nodes[:, None] * 3 + np.arange(3)).ravel()
        rec = Pt[dofs][:, a * 6:(a + 1) * 6] @ Bc[a * 6:(a + 1) * 6]
        assert np.abs(rec - Bm[dofs]).max() <= 1e-12 * max(1.0, np.abs(Bm[dofs]).max())
    rng = np.random.default_rng(4)
    b = rng.standard_normal(A.shape[0])
    b[mask] = 0.0
    sm = cycles.SmootherParams()
    for spec, exact in ((flagged, True), (plain, False)):
        lv = amg.build_group([A], [spec], 3, 30, 5)
        x = cycles.vcycle(lv, 0, amg.DenseLU(lv[-1][0].A), b, sm)
        if exact:
            assert np.all(x[mask] == 0.0)
        else:
            assert np.abs(x[mask]).max() > 0.0


def test_fully_flagged_nodes_stay_out_of_every_aggregate():
    A, plain, flagged, mask = _roller_box(5)
    all_dofs = np.zeros(A.shape[0], bool)
    nodes = np.arange(0, A.shape[0] // 3, 7)
    for nd in nodes:
        all_dofs[nd * 3:(nd + 1) * 3] = True
    spec = amg.FieldSpec(3, 3, "rbm", flagged.coords, 0.0, dirichlet=all_dofs)
    L = amg.build_group([A], [spec], 2, 30, 5)
    assert np.all(L[0][0].agg[nodes] == -1)
    assert np.all(np.delete(L[0][0].agg, nodes) >= 0)
