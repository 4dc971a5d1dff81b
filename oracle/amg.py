"""Smoothed-aggregation AMG setup, FP64, one field at a time.

TEST INFRASTRUCTURE (oracle).  The paper builds its single-field multigrid
objects P^l, R^l, S^l with standard smoothed aggregation (Sec. 3.3, citing
Vanek, Brezina & Mandel) and forms coarse operators by the Galerkin product
A^{l+1} = R^l A^l P^l (Sec. 3.3; blockwise R_i A_ij P_j for the monolithic
hierarchy, Sec. 4.3).  The paper does not spell out the aggregation, so the
steps below are the readings this project fixes:

1. strength: nodes I != J are strongly connected when the Frobenius norm of
   the node block A_IJ exceeds theta * sqrt(|A_II| |A_JJ|); the graph is
   symmetrised; nodes without strong neighbours (Dirichlet rows after
   symmetric elimination) are isolated and left out of every aggregate.
2. aggregation: roots = the lexicographically-first maximal distance-2
   independent set when nodes are taken in decreasing SplitMix64 priority
   (ties: lower index); every neighbour of a root joins it; every remaining
   node joins, among its neighbours aggregated so far, the aggregate whose
   root has the highest priority.  Aggregates are numbered by root index.
   Nodes whose every dof is flagged as a Dirichlet dof by the caller lose
   all their edges as well.
3. tentative prolongator: per aggregate, QR of the near-nullspace rows (the
   field's constants, rigid-body modes or the caller's vectors; zero rows at
   flagged Dirichlet dofs) by
   column-wise Gram-Schmidt with one re-orthogonalisation, dropping a column
   whose remaining norm is below 1e-10 of its norm before projection; the
   Q columns fill P_tent and R becomes the coarse near-nullspace.
   Rigid-body rotations are taken about the aggregate centroid.
4. lambda_max(D^-1 A): 10 power iterations from a SplitMix64 uniform start
   vector, lambda = ||D^-1 A v|| with ||v|| = 1.
5. P = (I - omega D^-1 A) P_tent, omega = 4 / (3 lambda_max).
6. R = P^T, A_c = R A P.

Fields marked Petrov-Galerkin (the paper's fluid field, Sec. 7.2, citing Sala &
Tuminaro 2008) replace steps 5-6 by pg_transfers: local damping parameters
per coarse dof chosen to minimise ||A p_j|| in the D^-1 norm, moved to the
rows by a minimum so that the near nullspace is kept, R built the same way
from A^T, and A_c = R A P with R != P^T.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.linalg as sla

from .rng import splitmix64, uniform01

RANK_DROP = 1e-10
POWER_ITERS = 10


def node_incidence(n_nodes: int, b: int) -> sp.csr_matrix:
    """E with E[dof, node] = 1 for dof = node * b + c."""
    rows = np.arange(n_nodes * b)
    return sp.csr_matrix((np.ones(n_nodes * b), (rows, rows // b)), shape=(n_nodes * b, n_nodes))


def strength_graph(A: sp.csr_matrix, b: int, theta: float) -> sp.csr_matrix:
    """Symmetric boolean node graph of strong connections (step 1)."""
    nn = A.shape[0] // b
    E = node_incidence(nn, b)
    A2 = A.multiply(A).tocsr()
    N = (E.T @ A2 @ E).tocoo()
    norms = np.sqrt(N.data)
    dn = np.zeros(nn)
    on_diag = N.row == N.col
    dn[N.row[on_diag]] = norms[on_diag]
    keep = (~on_diag) & (norms > theta * np.sqrt(dn[N.row] * dn[N.col]))
    G = sp.csr_matrix((np.ones(int(keep.sum())), (N.row[keep], N.col[keep])), shape=(nn, nn))
    G = ((G + G.T) > 0).astype(np.float64).tocsr()
    G.sort_indices()
    return G


def isolate_nodes(G: sp.csr_matrix, mask: np.ndarray) -> sp.csr_matrix:
    """The strength graph without any edge of a masked node (a node whose
    every dof is a Dirichlet dof stays out of every aggregate)."""
    keep = sp.diags((~mask).astype(np.float64))
    H = (keep @ G @ keep).tocsr()
    H.eliminate_zeros()
    H.sort_indices()
    return H


def aggregate(G: sp.csr_matrix, seed: int):
    """Aggregation of step 2.  Returns (agg, roots, prio): agg[I] is the
    aggregate id of node I or -1 (isolated); roots[a] is the root of a."""
    n = G.shape[0]
    ip, ix = G.indptr, G.indices
    prio = splitmix64(seed, n)
    deg = np.diff(ip)
    isolated = deg == 0
    # decreasing priority, ties by lower index
    order = np.lexsort((np.arange(n), ~prio))
    marked = np.zeros(n, bool)
    roots = []
    for I in order:
        if isolated[I] or marked[I]:
            continue
        roots.append(I)
        nb = ix[ip[I]:ip[I + 1]]
        marked[I] = True
        marked[nb] = True
        for K in nb:
            marked[ix[ip[K]:ip[K + 1]]] = True
    roots = np.sort(np.array(roots, dtype=np.int64))
    agg = np.full(n, -1, np.int64)
    agg[roots] = np.arange(len(roots))
    # phase 2: neighbours of a root (roots are >= 3 apart, so at most one)
    for a, R in enumerate(roots):
        agg[ix[ip[R]:ip[R + 1]]] = a
    # phase 3: the rest join the neighbouring aggregate with the best root
    agg2 = agg.copy()
    rest = np.nonzero((agg2 < 0) & ~isolated)[0]
    for I in rest:
        nb = ix[ip[I]:ip[I + 1]]
        cand = np.unique(agg2[nb][agg2[nb] >= 0])
        if len(cand) == 0:
            raise RuntimeError("aggregation: node not within distance 2 of a root")
        rp = prio[roots[cand]]
        best = np.lexsort((roots[cand], ~rp))[0]
        agg[I] = cand[best]
    return agg, roots, prio


def fine_nullspace_rows(field_b: int, dim: int, kind: str, xyz: np.ndarray) -> np.ndarray:
    """Near-nullspace rows for a set of nodes (|nodes| * b x k), rotations
    about the origin of the given (already centred) coordinates."""
    m = xyz.shape[0]
    if kind == "const":
        return np.tile(np.eye(field_b), (m, 1))
    if kind != "rbm":
        raise ValueError(kind)
    if dim == 2 and field_b == 2:
        B = np.zeros((m, 2, 3))
        B[:, 0, 0] = 1.0
        B[:, 1, 1] = 1.0
        B[:, 0, 2] = -xyz[:, 1]
        B[:, 1, 2] = xyz[:, 0]
        return B.reshape(2 * m, 3)
    if dim == 3 and field_b == 3:
        x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
        B = np.zeros((m, 3, 6))
        B[:, 0, 0] = B[:, 1, 1] = B[:, 2, 2] = 1.0
        B[:, 1, 3], B[:, 2, 3] = -z, y
        B[:, 0, 4], B[:, 2, 4] = z, -x
        B[:, 0, 5], B[:, 1, 5] = -y, x
        return B.reshape(3 * m, 6)
    raise ValueError("rigid-body modes need b == dim")


def nullspace_dim(field_b: int, dim: int, kind: str, user=None) -> int:
    if kind == "const":
        return field_b
    if kind == "user":
        return int(user.shape[1])
    return 3 if dim == 2 else 6


def gram_schmidt_qr(B: np.ndarray):
    """Step 3 QR: column-wise Gram-Schmidt with one re-orthogonalisation.
    Returns Q (m x k, dropped columns zero) and upper-triangular R (k x k)."""
    m, k = B.shape
    Q = np.zeros((m, k))
    R = np.zeros((k, k))
    for c in range(k):
        v = B[:, c].copy()
        n0 = np.linalg.norm(v)
        for _ in range(2):
            h = Q[:, :c].T @ v
            v -= Q[:, :c] @ h
            R[:c, c] += h
        nv = np.linalg.norm(v)
        if nv > RANK_DROP * n0 and nv > 0.0:
            Q[:, c] = v / nv
            R[c, c] = nv
    return Q, R


def tentative_prolongator(agg, nagg, b, k, B=None, coords=None, kind=None, dim=None, user=None, dmask=None):
    """Step 3.  On the fine level B is None and the nullspace is formed from
    node coordinates (centred per aggregate), or taken from the caller's
    vectors (kind "user": `user`, ndofs x k); on coarse levels B is the
    previous level's coarse nullspace (n x k).  On the fine level the rows of
    dofs flagged in dmask (Dirichlet dofs) are zero.  Returns (P_tent, B_coarse)."""
    n = len(agg) * b
    rows, cols, vals = [], [], []
    Bc = np.zeros((nagg * k, k))
    order = np.argsort(agg, kind="stable")
    starts = np.searchsorted(agg[order], np.arange(nagg + 1))
    for a in range(nagg):
        nodes = order[starts[a]:starts[a + 1]]          # ascending node index
        dofs = (nodes[:, None] * b + np.arange(b)[None, :]).ravel()
        if B is None and kind == "const":
            Ba = fine_nullspace_rows(b, dim, kind, np.zeros((len(nodes), 0)))
        elif B is None and kind == "user":
            Ba = np.array(user[dofs], dtype=np.float64)
        elif B is None:
            xyz = coords[nodes]
            xyz = xyz - xyz.mean(axis=0)
            Ba = fine_nullspace_rows(b, dim, kind, xyz)
        else:
            Ba = B[dofs]
        if B is None and dmask is not None:
            Ba = Ba.copy()
            Ba[dmask[dofs]] = 0.0
        Q, R = gram_schmidt_qr(Ba)
        rr, cc = np.nonzero(np.ones_like(Q, bool))
        rows.append(dofs[rr])
        cols.append(a * k + cc)
        vals.append(Q[rr, cc])
        Bc[a * k:(a + 1) * k] = R
    if nagg:
        rows, cols, vals = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    P = sp.csr_matrix((vals, (rows, cols)), shape=(n, nagg * k))
    return P, Bc


def power_lambda(A: sp.csr_matrix, dinv: np.ndarray, seed: int, iters: int = POWER_ITERS) -> float:
    """Step 4: lambda_max(D^-1 A) estimate."""
    v = uniform01(seed, A.shape[0])
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = dinv * (A @ v)
        lam = np.linalg.norm(w)
        v = w / lam
    return float(lam)


class FieldLevel:
    """Multigrid objects of one field on one level."""

    def __init__(self, A, b):
        self.A = A.tocsr()
        self.b = b
        with np.errstate(divide="ignore"):
            self.dinv = 1.0 / self.A.diagonal()
        self.lam = None
        self.agg = None
        self.P = None
        self.R = None
        self.B = None


class FieldSpec:
    """What the setup needs to know about a field (mirrors the C-ABI field
    map): dofs per node, dimension, near-nullspace kind ("const", "rbm" or
    "user" with the caller's vectors `user`, ndofs x k), node coordinates,
    strength threshold, Petrov-Galerkin flag and optional per-dof Dirichlet
    flags (`dirichlet`, bool per dof)."""

    def __init__(self, b, dim, kind, coords=None, theta=0.0, pg=False, user=None, dirichlet=None):
        self.b, self.dim, self.kind, self.coords, self.theta = b, dim, kind, coords, theta
        self.pg = pg
        self.user = user
        self.dirichlet = None if dirichlet is None else np.asarray(dirichlet, bool)

    def node_mask(self):
        """Nodes whose every dof is a flagged Dirichlet dof (or None)."""
        if self.dirichlet is None:
            return None
        return self.dirichlet.reshape(-1, self.b).all(axis=1)

    @classmethod
    def of(cls, f):
        return cls(f.b, f.dim, f.nullspace, f.coords, f.theta, getattr(f, "petrov_galerkin", False),
                   getattr(f, "ns_user", None), getattr(f, "dirichlet_dofs", None))


# a scalar column counts in the row minimum of the damping parameters when its
# entry of D^-1 A P_tent exceeds this fraction of the largest entry (rounding-
# level entries, e.g. inside an aggregate where A annihilates the constant, do not)
PG_PATTERN_REL = 1e-12


def pg_damping(A, dinv, Pt):
    """Row damping parameters of the Petrov-Galerkin prolongator smoothing:
    Q = D^-1 A P_tent; per coarse dof j, omega_j minimises
    f_j(w) = || A (p_j - w q_j) ||^2_{D^-1}  (p_j, q_j: column j of P_tent, Q),
    i.e. omega_j = <A q_j, q_j> / <A q_j, D^-1 A q_j>, set to 0 when not
    positive; row i takes the minimum of omega_j over the columns j with
    |Q_ij| > PG_PATTERN_REL * max |Q| (0 for a row without such columns).
    Returns (Q, row omegas, column omegas)."""
    Q = (sp.diags(dinv) @ (A @ Pt)).tocsr()
    AQ = (A @ Q).tocsr()
    num = np.asarray(AQ.multiply(Q).sum(axis=0)).ravel()
    den = np.asarray(AQ.multiply(AQ).multiply(dinv[:, None]).sum(axis=0)).ravel()
    wcol = np.zeros(Q.shape[1])
    ok = (den > 0) & (num > 0)
    wcol[ok] = num[ok] / den[ok]
    thr = PG_PATTERN_REL * (np.abs(Q.data).max() if Q.nnz else 0.0)
    wrow = np.zeros(Q.shape[0])
    for i in range(Q.shape[0]):
        lo, hi = Q.indptr[i], Q.indptr[i + 1]
        cols = Q.indices[lo:hi][np.abs(Q.data[lo:hi]) > thr]
        if len(cols):
            wrow[i] = wcol[cols].min()
    return Q, wrow, wcol


def pg_transfers(A, dinv, Pt):
    """P = P_tent - diag(omega) D^-1 A P_tent and R = (P_tent - diag(omega')
    D^-1 A^T P_tent)^T with the row parameters of pg_damping for A and A^T."""
    Q, w, _ = pg_damping(A, dinv, Pt)
    P = (Pt - sp.diags(w) @ Q).tocsr()
    At = A.T.tocsr()
    Qt, wt, _ = pg_damping(At, dinv, Pt)
    R = (Pt - sp.diags(wt) @ Qt).T.tocsr()
    return P, R


def build_group(As, specs, max_levels, coarse_max, seed):
    """Single-field SA hierarchies for a group of fields that coarsen together:
    a new level is made while the level count is below max_levels and the
    group's total dof count exceeds coarse_max.  Returns levels[l][i]."""
    levels = [[FieldLevel(A, s.b) for A, s in zip(As, specs)]]
    if not all(np.all(np.isfinite(fl.dinv)) for fl in levels[0]):
        # D^-1 A smoothing (and BGS, Sec. 4.1) needs nonsingular diagonal blocks
        raise ValueError("zero diagonal entry in a diagonal block")
    while len(levels) < max_levels and sum(fl.A.shape[0] for fl in levels[-1]) > coarse_max:
        fine = len(levels) == 1
        nxt = []
        for fl, s in zip(levels[-1], specs):
            fl.lam = power_lambda(fl.A, fl.dinv, seed)
            G = strength_graph(fl.A, fl.b, s.theta)
            if fine and s.node_mask() is not None:
                G = isolate_nodes(G, s.node_mask())
            agg, roots, _ = aggregate(G, seed)
            nagg = len(roots)
            if nagg == 0:
                raise RuntimeError("aggregation produced no aggregate")
            if fine:
                k = nullspace_dim(s.b, s.dim, s.kind, s.user)
                Pt, Bc = tentative_prolongator(agg, nagg, fl.b, k, coords=s.coords, kind=s.kind, dim=s.dim,
                                               user=s.user, dmask=s.dirichlet)
            else:
                k = fl.b
                Pt, Bc = tentative_prolongator(agg, nagg, fl.b, k, B=fl.B)
            if s.pg:
                P, R = pg_transfers(fl.A, fl.dinv, Pt)
            else:
                omega = 4.0 / (3.0 * fl.lam)
                P = (Pt - omega * sp.diags(fl.dinv) @ (fl.A @ Pt)).tocsr()
                R = P.T.tocsr()
            fl.agg, fl.P, fl.R = agg, P, R
            c = FieldLevel(fl.R @ fl.A @ P, k)
            c.B = Bc
            nxt.append(c)
        levels.append(nxt)
    return levels


def coarse_block(Ri, Aij, Pj):
    """Blockwise Galerkin product R_i A_ij P_j (Sec. 4.3)."""
    return (Ri @ Aij @ Pj).tocsr()


class DenseLU:
    """Coarsest-level direct solver: dense LU with partial pivoting (LAPACK
    getrf through scipy), FP64."""

    def __init__(self, M):
        M = M.toarray() if sp.issparse(M) else np.asarray(M)
        self.n = M.shape[0]
        self.lu, self.piv = sla.lu_factor(M)
        d = np.abs(np.diag(self.lu))
        if self.n and (d.min() == 0.0 or not np.isfinite(d).all()):
            raise np.linalg.LinAlgError("singular coarse matrix")

    def solve(self, b):
        return sla.lu_solve((self.lu, self.piv), b)
