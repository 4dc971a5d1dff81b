"""Seeded synthetic coupled block systems (input generation only).

This module builds the N x N block linear systems (Sec. 4, the blocked system
A x = b with blocks A_ij) on which the preconditioned GMRES path is run.  It
holds no solver or preconditioner arithmetic: it assembles bilinear /
trilinear (Q1) finite-element matrices on a uniform structured mesh, applies
Dirichlet conditions by symmetric elimination and draws a seeded N(0,1)
right-hand side.  Both the CUDA path and the CPU oracle consume its output.

The workloads stand in for the paper's thermo-structure interaction (Sec. 6.1,
the monolithic TSI system) and fluid-structure-like (Sec. 6.2) applications,
whose meshes are not available:

* ``thermo_elastic_2d``  - 2 fields on the unit square: plane-strain elasticity
  (2 dof/node) + transient heat (1 dof/node), coupled through
  A_12 = alpha * int B^T m N and A_21 = 1e-3 * int N m^T B.
* ``fsi_box``            - 4 fields on the unit cube split at z = 0.5: elasticity
  above, mesh motion + PSPG Stokes velocity / pressure below, coupled through an
  interface penalty and volume blocks (saddle point: the pressure block is
  negative definite).
* ``coupled_box_3d``     - the 3D analogue on the unit cube with 2 or 3 fields:
  elasticity (3 dof/node), heat (1 dof/node) and an optional scalar diffusion
  field whose diffusivity is log-uniform in [1e-3, 1e3] per element.  The
  heat-diffusion pair is coupled by alpha*M and 1e-3*M.
* ``constrained_box``    - the coupled box plus a field of m Lagrange multipliers
  (stand-in for the lung model's volume constraints, Sec. 6.3): each enforces
  the mean normal displacement over one patch of the free face; the
  multiplier-multiplier block is zero (saddle point with a zero diagonal
  block).

Layout of a block: node-level block-CSR (BSR) with int32 ``rowptr`` / ``colind``
and float64 ``vals`` of shape (nnzb, br, bc), row-major inside a block.
Dofs of a field are interleaved per node (dof = node * b + component).  The
global vector is the field-major concatenation of the field vectors.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import itertools

import numpy as np

__all__ = [
    "BSR", "Field", "BlockSystem", "thermo_elastic_2d", "coupled_box_3d", "constrained_box", "fsi_box", "roller_box",
    "batch_sizes_log_uniform", "batch_workload", "system_rhs",
]


@dataclass
class BSR:
    """Node-level block-CSR matrix: block (I, J) is vals[k] for colind[k] == J."""
    br: int
    bc: int
    nbrows: int
    nbcols: int
    rowptr: np.ndarray  # int32, nbrows + 1
    colind: np.ndarray  # int32, nnzb
    vals: np.ndarray    # float64, (nnzb, br, bc)

    @property
    def nnzb(self) -> int:
        return int(self.colind.shape[0])

    @property
    def shape(self):
        return (self.nbrows * self.br, self.nbcols * self.bc)

    def to_scipy(self):
        """Point CSR copy (scipy), for consumers that work on scalar entries."""
        import scipy.sparse as sp
        m = sp.bsr_matrix((self.vals, self.colind, self.rowptr), shape=self.shape)
        return m.tocsr()


@dataclass
class Field:
    name: str
    b: int                 # dofs per node
    nnodes: int
    dim: int
    coords: np.ndarray     # (nnodes, dim) float64
    nullspace: str         # "const" (per-component constants) or "rbm" (rigid-body modes)
    theta: float = 0.0     # strength-of-connection threshold used for this field
    dirichlet_nodes: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    petrov_galerkin: bool = False  # non-symmetric block: Petrov-Galerkin transfers (R != P^T)
    ns_user: np.ndarray = None     # nullspace "user": caller's near-nullspace vectors (ndofs x k)
    dirichlet_dofs: np.ndarray = None  # optional per-dof flags of eliminated Dirichlet dofs (bool)

    @property
    def ndofs(self) -> int:
        return self.nnodes * self.b


@dataclass
class BlockSystem:
    fields: list
    blocks: dict           # (i, j) -> BSR; absent pairs are zero blocks
    rhs: np.ndarray        # float64, sum of field dofs
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nfields(self) -> int:
        return len(self.fields)

    @property
    def offsets(self):
        off = [0]
        for f in self.fields:
            off.append(off[-1] + f.ndofs)
        return off

    @property
    def ndofs(self) -> int:
        return self.offsets[-1]

    def scipy_blocks(self):
        return {k: v.to_scipy() for k, v in self.blocks.items()}


# ----------------------------------------------------------------------------
# Q1 reference-element matrices on an axis-aligned cell of edge h
# ----------------------------------------------------------------------------

def _local_offsets(dim):
    # local node a <-> offset o_a in {0,1}^dim, x fastest
    return [tuple(reversed(t)) for t in itertools.product((0, 1), repeat=dim)]


def _gauss_2pt():
    g = 0.5 / np.sqrt(3.0)
    return np.array([0.5 - g, 0.5 + g]), np.array([0.5, 0.5])


def _shape_at(dim, xi):
    """Values N_a(xi) and reference gradients dN_a/dxi on [0,1]^dim."""
    offs = _local_offsets(dim)
    n = len(offs)
    N = np.ones(n)
    dN = np.ones((n, dim))
    for a, o in enumerate(offs):
        for d in range(dim):
            f = xi[d] if o[d] else 1.0 - xi[d]
            df = 1.0 if o[d] else -1.0
            N[a] *= f
            for e in range(dim):
                dN[a, e] *= df if e == d else f
    return N, dN


def _strain_matrix(dim, dNdx):
    n = dNdx.shape[0]
    if dim == 2:
        B = np.zeros((3, 2 * n))
        for a in range(n):
            dx, dy = dNdx[a]
            B[0, 2 * a] = dx
            B[1, 2 * a + 1] = dy
            B[2, 2 * a] = dy
            B[2, 2 * a + 1] = dx
        return B
    B = np.zeros((6, 3 * n))
    for a in range(n):
        dx, dy, dz = dNdx[a]
        c = 3 * a
        B[0, c] = dx
        B[1, c + 1] = dy
        B[2, c + 2] = dz
        B[3, c + 1] = dz
        B[3, c + 2] = dy
        B[4, c] = dz
        B[4, c + 2] = dx
        B[5, c] = dy
        B[5, c + 1] = dx
    return B


def _elasticity_D(dim, E, nu):
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    if dim == 2:  # plane strain
        return np.array([[lam + 2 * mu, lam, 0], [lam, lam + 2 * mu, 0], [0, 0, mu]])
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] = lam + 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def q1_element_matrices(dim, h, E=1.0, nu=0.3):
    """Element stiffness (elasticity, Laplacian), mass and thermo-mechanical
    coupling int B^T m N on a cell of edge h with 2^dim Gauss points."""
    pts, wts = _gauss_2pt()
    nloc = 2 ** dim
    D = _elasticity_D(dim, E, nu)
    m = np.array([1.0, 1.0, 0.0]) if dim == 2 else np.array([1.0, 1, 1, 0, 0, 0])
    Ke = np.zeros((dim * nloc, dim * nloc))
    Kl = np.zeros((nloc, nloc))
    Me = np.zeros((nloc, nloc))
    Ce = np.zeros((dim * nloc, nloc))
    detJ = h ** dim
    for idx in itertools.product(range(2), repeat=dim):
        xi = np.array([pts[i] for i in idx])
        w = np.prod([wts[i] for i in idx]) * detJ
        N, dN = _shape_at(dim, xi)
        dNdx = dN / h
        B = _strain_matrix(dim, dNdx)
        Ke += w * B.T @ D @ B
        Kl += w * dNdx @ dNdx.T
        Me += w * np.outer(N, N)
        Ce += w * np.outer(B.T @ m, N)
    return Ke, Kl, Me, Ce


# ----------------------------------------------------------------------------
# Structured-mesh BSR assembly
# ----------------------------------------------------------------------------

class _Grid:
    """Structured node grid of ne cells per direction, or of `shape` cells
    (x, y[, z]) with edge h and the given origin."""

    def __init__(self, ne, dim, shape=None, h=None, origin=None):
        shape = tuple(shape) if shape is not None else (ne,) * dim
        self.ne = ne
        self.dim = dim
        self.shape = shape
        self.h = h if h is not None else 1.0 / ne
        n1 = [c + 1 for c in shape]
        self.n1 = n1[0]
        self.nnodes = int(np.prod(n1))
        ijk = np.indices(tuple(reversed(n1))).reshape(dim, -1)[::-1]  # x fastest
        self.ijk = ijk.T.copy()                                        # (nnodes, dim): (i, j[, k])
        org = np.zeros(dim) if origin is None else np.asarray(origin, float)
        self.coords = self.ijk * self.h + org
        self.stride = np.array([int(np.prod(n1[:d])) for d in range(dim)])
        # neighbour stencil, in increasing node-index order (z slowest)
        self.stencil = [tuple(reversed(t)) for t in itertools.product((-1, 0, 1), repeat=dim)]
        self.sidx = {s: k for k, s in enumerate(self.stencil)}
        ns = len(self.stencil)
        valid = np.ones((self.nnodes, ns), bool)
        for k, s in enumerate(self.stencil):
            for d in range(dim):
                c = self.ijk[:, d] + s[d]
                valid[:, k] &= (c >= 0) & (c <= shape[d])
        self.valid = valid
        counts = valid.sum(1)
        self.rowptr = np.zeros(self.nnodes + 1, np.int64)
        np.cumsum(counts, out=self.rowptr[1:])
        pos = np.full((self.nnodes, ns), -1, np.int64)
        run = np.cumsum(valid, axis=1) - 1 + self.rowptr[:-1, None]
        pos[valid] = run[valid]
        self.pos = pos
        colind = np.zeros(self.rowptr[-1], np.int64)
        for k, s in enumerate(self.stencil):
            off = int(np.dot(s, self.stride))
            v = valid[:, k]
            colind[pos[v, k]] = np.nonzero(v)[0] + off
        self.colind = colind
        # elements: base node index for every cell
        eijk = np.indices(tuple(reversed(shape))).reshape(dim, -1)[::-1].T
        self.nelem = eijk.shape[0]
        self.ebase = eijk @ self.stride
        self.loc = _local_offsets(dim)

    def assemble(self, Kloc, br, bc, scale=None):
        """Sum the element matrix Kloc (nloc*br x nloc*bc, dof = a*b + comp)
        over all cells, optionally scaled per cell; returns BSR vals."""
        vals = np.zeros((self.rowptr[-1], br, bc))
        for a, oa in enumerate(self.loc):
            node_a = self.ebase + int(np.dot(oa, self.stride))
            for b_, ob in enumerate(self.loc):
                s = tuple(ob[d] - oa[d] for d in range(self.dim))
                p = self.pos[node_a, self.sidx[s]]
                blk = Kloc[a * br:(a + 1) * br, b_ * bc:(b_ + 1) * bc]
                if scale is None:
                    vals[p] += blk
                else:
                    vals[p] += scale[:, None, None] * blk
        return vals

    def bsr(self, vals, br, bc):
        return BSR(br, bc, self.nnodes, self.nnodes, self.rowptr.astype(np.int32),
                   self.colind.astype(np.int32), vals)


def _apply_dirichlet(grid, blocks, nfields, dnodes):
    """Symmetric elimination: zero Dirichlet rows/cols in every block and put
    the identity on the diagonal blocks (all fields share the node set)."""
    isd = np.zeros(grid.nnodes, bool)
    isd[dnodes] = True
    rows = np.repeat(np.arange(grid.nnodes), np.diff(grid.rowptr))
    kill = isd[rows] | isd[grid.colind]
    diag = isd[rows] & (rows == grid.colind)
    for (i, j), m in blocks.items():
        m.vals[kill] = 0.0
        if i == j:
            m.vals[diag] = np.eye(m.br)


def _seeded_rhs(fields, seed, dnodes):
    rng = np.random.default_rng(seed)
    n = sum(f.ndofs for f in fields)
    b = rng.standard_normal(n)
    off = 0
    for f in fields:
        d = (dnodes[:, None] * f.b + np.arange(f.b)[None, :]).ravel()
        b[off + d] = 0.0
        off += f.ndofs
    return b


def thermo_elastic_2d(ne=32, alpha=1e-2, beta=1e-3, E=1.0, nu=0.3, k=1.0, dt=0.1, seed=0):
    """2-field thermo-elastic system on the unit square (Sec. 6.1 in 2D):
    field 0 plane-strain elasticity, field 1 transient heat (k*L + M/dt),
    A_01 = alpha*int B^T m N, A_10 = beta*int N m^T B; left edge clamped and
    T = 0 there."""
    g = _Grid(ne, 2)
    h = 1.0 / ne
    Ke, Kl, Me, Ce = q1_element_matrices(2, h, E, nu)
    blocks = {
        (0, 0): g.bsr(g.assemble(Ke, 2, 2), 2, 2),
        (1, 1): g.bsr(g.assemble(k * Kl + Me / dt, 1, 1), 1, 1),
        (0, 1): g.bsr(g.assemble(alpha * Ce, 2, 1), 2, 1),
        (1, 0): g.bsr(g.assemble(beta * Ce.T, 1, 2), 1, 2),
    }
    dnodes = np.nonzero(g.ijk[:, 0] == 0)[0]
    _apply_dirichlet(g, blocks, 2, dnodes)
    fields = [
        Field("elasticity", 2, g.nnodes, 2, g.coords, "rbm", 0.0, dnodes),
        Field("heat", 1, g.nnodes, 2, g.coords, "const", 0.0, dnodes),
    ]
    return BlockSystem(fields, blocks, _seeded_rhs(fields, seed, dnodes),
                       name=f"thermo_elastic_2d_ne{ne}",
                       meta=dict(ne=ne, alpha=alpha, seed=seed))


def coupled_box_3d(ne=64, nfields=3, alpha=1e-2, beta=1e-3, E=1.0, nu=0.3, k=1.0, dt=0.1,
                   diff_theta=0.02, seed=1):
    """3D coupled box on the unit cube: field 0 elasticity (3 dof/node), field 1
    heat (k*L + M/dt), optional field 2 scalar diffusion with per-cell
    diffusivity 10^U(-3,3) (no mass).  Elasticity-scalar pairs use the
    thermo-mechanical coupling (alpha*int B^T m N, beta*int N m^T B); the
    heat-diffusion pair uses alpha*M and beta*M.  The x = 0 face is Dirichlet
    for every field."""
    assert nfields in (2, 3)
    g = _Grid(ne, 3)
    h = 1.0 / ne
    Ke, Kl, Me, Ce = q1_element_matrices(3, h, E, nu)
    rng = np.random.default_rng(seed)
    blocks = {
        (0, 0): g.bsr(g.assemble(Ke, 3, 3), 3, 3),
        (1, 1): g.bsr(g.assemble(k * Kl + Me / dt, 1, 1), 1, 1),
        (0, 1): g.bsr(g.assemble(alpha * Ce, 3, 1), 3, 1),
        (1, 0): g.bsr(g.assemble(beta * Ce.T, 1, 3), 1, 3),
    }
    fields_theta = [0.0, 0.0]
    if nfields == 3:
        kappa = 10.0 ** rng.uniform(-3.0, 3.0, size=g.nelem)
        blocks[(2, 2)] = g.bsr(g.assemble(Kl, 1, 1, scale=kappa), 1, 1)
        blocks[(0, 2)] = g.bsr(g.assemble(alpha * Ce, 3, 1), 3, 1)
        blocks[(2, 0)] = g.bsr(g.assemble(beta * Ce.T, 1, 3), 1, 3)
        blocks[(1, 2)] = g.bsr(g.assemble(alpha * Me, 1, 1), 1, 1)
        blocks[(2, 1)] = g.bsr(g.assemble(beta * Me, 1, 1), 1, 1)
        fields_theta.append(diff_theta)
    dnodes = np.nonzero(g.ijk[:, 0] == 0)[0]
    _apply_dirichlet(g, blocks, nfields, dnodes)
    names = ["elasticity", "heat", "diffusion"]
    fields = []
    for i in range(nfields):
        b = 3 if i == 0 else 1
        fields.append(Field(names[i], b, g.nnodes, 3, g.coords, "rbm" if i == 0 else "const",
                            fields_theta[i], dnodes))
    return BlockSystem(fields, blocks, _seeded_rhs(fields, seed, dnodes),
                       name=f"coupled_box_3d_ne{ne}_f{nfields}",
                       meta=dict(ne=ne, nfields=nfields, alpha=alpha, seed=seed))


def _eliminate_dofs(grid, blocks, masks):
    """Symmetric elimination of single dofs: masks[i] flags the dofs of field
    i (per dof, node-major); their rows and columns are zeroed in every block
    and the diagonal entry of A_ii set to 1."""
    rows = np.repeat(np.arange(grid.nnodes), np.diff(grid.rowptr))
    for (i, j), m in blocks.items():
        ri = masks[i].reshape(grid.nnodes, m.br)[rows]        # (nnzb, br)
        cj = masks[j].reshape(grid.nnodes, m.bc)[grid.colind]  # (nnzb, bc)
        m.vals[ri[:, :, None] | cj[:, None, :]] = 0.0
        if i == j:
            on = rows == grid.colind
            for c in range(m.br):
                sel = on & ri[:, c]
                m.vals[sel, c, c] = 1.0


def roller_box(ne=12, user_nullspace=False, seed=6):
    """2-field 3D box (elasticity + heat, the couplings of coupled_box_3d)
    with symmetry conditions: on each face x_d = 0 only the displacement
    component u_d is held (so edge and corner nodes hold 2 or 3 components),
    T = 0 on x = 0.  The held dofs are eliminated symmetrically and flagged
    per dof (Field.dirichlet_dofs).  user_nullspace: the elasticity field
    gives its rigid-body modes (rotations about the origin) as caller
    vectors (nullspace "user") instead of the built-in kind."""
    g = _Grid(ne, 3)
    h = 1.0 / ne
    Ke, Kl, Me, Ce = q1_element_matrices(3, h)
    blocks = {
        (0, 0): g.bsr(g.assemble(Ke, 3, 3), 3, 3),
        (1, 1): g.bsr(g.assemble(Kl + Me / 0.1, 1, 1), 1, 1),
        (0, 1): g.bsr(g.assemble(1e-2 * Ce, 3, 1), 3, 1),
        (1, 0): g.bsr(g.assemble(1e-3 * Ce.T, 1, 3), 1, 3),
    }
    m0 = np.zeros((g.nnodes, 3), bool)
    for d in range(3):
        m0[g.ijk[:, d] == 0, d] = True
    m1 = g.ijk[:, 0] == 0
    masks = [m0.ravel(), m1.copy()]
    _eliminate_dofs(g, blocks, masks)
    fields = [Field("elasticity", 3, g.nnodes, 3, g.coords, "rbm", 0.0, np.zeros(0, np.int64)),
              Field("heat", 1, g.nnodes, 3, g.coords, "const", 0.0, np.nonzero(m1)[0])]
    fields[0].dirichlet_dofs = masks[0]
    fields[1].dirichlet_dofs = masks[1]
    if user_nullspace:
        x, y, z = g.coords[:, 0], g.coords[:, 1], g.coords[:, 2]
        B = np.zeros((g.nnodes, 3, 6))
        B[:, 0, 0] = B[:, 1, 1] = B[:, 2, 2] = 1.0
        B[:, 1, 3], B[:, 2, 3] = -z, y
        B[:, 0, 4], B[:, 2, 4] = z, -x
        B[:, 0, 5], B[:, 1, 5] = -y, x
        fields[0].nullspace = "user"
        fields[0].ns_user = B.reshape(3 * g.nnodes, 6)
    rng = np.random.default_rng(seed)
    rhs = rng.standard_normal(4 * g.nnodes)
    rhs[:3 * g.nnodes][masks[0]] = 0.0
    rhs[3 * g.nnodes:][masks[1]] = 0.0
    return BlockSystem(fields, blocks, rhs, name=f"roller_box_ne{ne}{'_user' if user_nullspace else ''}",
                       meta=dict(ne=ne, seed=seed))


def constrained_box(ne=64, nfields=3, patches=(2, 2), seed=5, **kw):
    """coupled_box_3d plus a last field C of m = patches[0]*patches[1]
    Lagrange multipliers.  The free face x = 1 is cut into a grid of patches
    over (y, z); multiplier k enforces the mean x-displacement of patch k,
    with weights w_i = (int_{patch} N_i) / |patch| (Q1 face integrals, so the
    weights of a patch sum to 1): A_C0 holds w as 1 x 3 blocks [w_i, 0, 0],
    A_0C = A_C0^T (the multipliers act as uniform pressures on the patches)
    and A_CC is an all-zero (empty) block.  Fields 1.. of the box do not couple
    to C.  The right-hand side is redrawn with this seed over all fields."""
    base = coupled_box_3d(ne=ne, nfields=nfields, seed=seed, **kw)
    g = _Grid(ne, 3)
    py, pz = patches
    m = py * pz
    face = np.nonzero(g.ijk[:, 0] == ne)[0]
    wts = np.zeros((m, g.nnodes))
    # face cells (j, k) in y, z; each adds a quarter of its area to its four nodes
    for cj in range(ne):
        for ck in range(ne):
            k = min(cj * py // ne, py - 1) + py * min(ck * pz // ne, pz - 1)
            for dj in (0, 1):
                for dk in (0, 1):
                    node = ne + (cj + dj) * g.stride[1] + (ck + dk) * g.stride[2]
                    wts[k, node] += 0.25
    wts /= wts.sum(1, keepdims=True)
    rows_c, cols_c, vals_c = [], [], []
    for k in range(m):
        nz = np.nonzero(wts[k])[0]
        rows_c.append(len(nz))
        cols_c.append(nz)
        v = np.zeros((len(nz), 1, 3))
        v[:, 0, 0] = wts[k, nz]
        vals_c.append(v)
    rp = np.zeros(m + 1, np.int64)
    np.cumsum(rows_c, out=rp[1:])
    A_c0 = BSR(1, 3, m, g.nnodes, rp.astype(np.int32), np.concatenate(cols_c).astype(np.int32),
               np.concatenate(vals_c))
    # transpose: row i of A_0C has one block per patch containing node i
    cnt = (wts > 0).sum(0)
    rp2 = np.zeros(g.nnodes + 1, np.int64)
    np.cumsum(cnt, out=rp2[1:])
    col2 = np.zeros(rp2[-1], np.int32)
    val2 = np.zeros((rp2[-1], 3, 1))
    fill = rp2[:-1].copy()
    for k in range(m):
        nz = np.nonzero(wts[k])[0]
        col2[fill[nz]] = k
        val2[fill[nz], 0, 0] = wts[k, nz]
        fill[nz] += 1
    A_0c = BSR(3, 1, g.nnodes, m, rp2.astype(np.int32), col2, val2)
    nf = nfields + 1
    blocks = dict(base.blocks)
    blocks[(0, nf - 1)] = A_0c
    blocks[(nf - 1, 0)] = A_c0
    blocks[(nf - 1, nf - 1)] = BSR(1, 1, m, m, np.zeros(m + 1, np.int32), np.zeros(0, np.int32),
                                   np.zeros((0, 1, 1)))
    centres = np.array([[1.0, (kj + 0.5) / py, (kk + 0.5) / pz] for kk in range(pz) for kj in range(py)])
    fields = list(base.fields) + [Field("constraint", 1, m, 3, centres, "const", 0.0)]
    dnodes = base.fields[0].dirichlet_nodes
    rhs = np.random.default_rng(seed).standard_normal(sum(f.ndofs for f in fields))
    off = 0
    for f in fields[:-1]:
        d = (dnodes[:, None] * f.b + np.arange(f.b)[None, :]).ravel()
        rhs[off + d] = 0.0
        off += f.ndofs
    assert not np.intersect1d(face, dnodes).size
    return BlockSystem(fields, blocks, rhs, name=f"constrained_box_ne{ne}_f{nfields}_m{m}",
                       meta=dict(ne=ne, nfields=nfields, patches=patches, seed=seed))


def q1_flow_matrices(h):
    """3D Q1 cell matrices for the flow blocks: G[a*3+c, b] = -int dN_a/dx_c N_b
    (velocity x pressure, the discrete divergence) and Dz[a, b] = int N_a dN_b/dz."""
    pts, wts = _gauss_2pt()
    G = np.zeros((24, 8))
    Dz = np.zeros((8, 8))
    for idx in itertools.product(range(2), repeat=3):
        xi = np.array([pts[i] for i in idx])
        w = np.prod([wts[i] for i in idx]) * h ** 3
        N, dN = _shape_at(3, xi)
        dNdx = dN / h
        for a in range(8):
            for c in range(3):
                G[a * 3 + c] -= w * dNdx[a, c] * N
        Dz += w * np.outer(N, dNdx[:, 2])
    return G, Dz


def q1_convection_matrix(h, wind):
    """3D Q1 cell convection matrix C[a, b] = int N_a (wind . grad N_b)."""
    pts, wts = _gauss_2pt()
    C = np.zeros((8, 8))
    w3 = np.asarray(wind, float)
    for idx in itertools.product(range(2), repeat=3):
        xi = np.array([pts[i] for i in idx])
        w = np.prod([wts[i] for i in idx]) * h ** 3
        N, dN = _shape_at(3, xi)
        C += w * np.outer(N, (dN / h) @ w3)
    return C


def _vector_cell(K, b):
    """Cell matrix acting componentwise on b-vectors: (K kron I_b) in dof order a*b + c."""
    return np.kron(K, np.eye(b))


def _interface_nodes(grid, k):
    """Node-level interface mass between layer k of `grid` and itself (CSR)."""
    import scipy.sparse as sp
    nx, ny = grid.shape[0], grid.shape[1]
    M2 = q1_element_matrices(2, grid.h)[2]
    loc2 = _local_offsets(2)
    ci, cj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ci, cj = ci.ravel(), cj.ravel()
    rows, cols, vals = [], [], []
    for a, oa in enumerate(loc2):
        for b, ob in enumerate(loc2):
            rows.append((ci + oa[0]) + grid.stride[1] * (cj + oa[1]) + grid.stride[2] * k)
            cols.append((ci + ob[0]) + grid.stride[1] * (cj + ob[1]) + grid.stride[2] * k)
            vals.append(np.full(ci.shape, M2[a, b]))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(grid.nnodes, grid.nnodes))


def _add_to_grid_block(grid, vals, Nm, scale, b):
    """vals (grid BSR of b x b blocks) += scale * Nm (node-level, inside the stencil) kron I_b."""
    Nm = Nm.tocoo()
    d = grid.ijk[Nm.col] - grid.ijk[Nm.row]
    sidx = np.array([grid.sidx[tuple(t)] for t in d])
    p = grid.pos[Nm.row, sidx]
    assert np.all(p >= 0)
    np.add.at(vals, p, scale * Nm.data[:, None, None] * np.eye(b)[None])


def _node_bsr(Nm, b, scale):
    """BSR of b x b blocks scale * Nm kron I_b from a node-level CSR."""
    Nm = Nm.tocsr()
    Nm.sort_indices()
    return BSR(b, b, Nm.shape[0], Nm.shape[1], Nm.indptr.astype(np.int32), Nm.indices.astype(np.int32),
               scale * Nm.data[:, None, None] * np.eye(b)[None])


def _dirichlet_fields(blocks, dmasks):
    """Symmetric elimination with a Dirichlet node mask per field."""
    for (i, j), m in blocks.items():
        rows = np.repeat(np.arange(m.nbrows), np.diff(m.rowptr))
        kill = dmasks[i][rows] | dmasks[j][m.colind]
        m.vals[kill] = 0.0
        if i == j:
            diag = dmasks[i][rows] & (rows == m.colind)
            m.vals[diag] = np.eye(m.br)


def fsi_box(ne=48, nu=1e-2, E=1e3, poisson=0.3, gamma=1.0, eta=1e-3, seed=2, wind=None):
    """Fluid / structure / mesh-motion-like saddle system on the unit cube split
    at z = 0.5 (stand-in for the FSI block system of Sec. 6.2).  Fields:
      0 S  elasticity (3 dof/node, E, clamped top face) on the upper half;
      1 G  mesh motion, vector Laplacian (3 dof/node, zero on the lower half's
           outer faces) on the lower half;
      2 Fu Stokes velocity, nu * vector Laplacian (no-slip lateral faces, open
           bottom) on the lower half;
      3 Fp pressure (PSPG: -tau L, tau = h^2/(12 nu), p = 0 on the bottom face).
    Couplings: Fu-Fp discrete divergence and gradient; S-Fu and G-Fu interface
    penalties gamma * M_Gamma on the z = 0.5 plane (-M off the diagonal, +M on
    it); Fu <- G volume block eta * int N dN/dz.  S-G, S-Fp, G-Fp are zero.
    With `wind` (a constant 3-vector) the velocity block becomes the Oseen
    operator nu * L + int N (wind . grad N) per component, non-symmetric, and
    the velocity field is marked for Petrov-Galerkin transfers (the paper's
    fluid field, Sec. 7.2)."""
    h = 1.0 / ne
    nz = ne // 2
    up = _Grid(ne, 3, shape=(ne, ne, ne - nz), h=h, origin=(0.0, 0.0, nz * h))
    lo = _Grid(ne, 3, shape=(ne, ne, nz), h=h, origin=(0.0, 0.0, 0.0))
    Ke, Kl, Me, Ce = q1_element_matrices(3, h, E, poisson)
    Gd, Dz = q1_flow_matrices(h)
    tau = h * h / (12.0 * nu)
    blocks = {
        (0, 0): up.bsr(up.assemble(Ke, 3, 3), 3, 3),
        (1, 1): lo.bsr(lo.assemble(_vector_cell(Kl, 3), 3, 3), 3, 3),
        (2, 2): lo.bsr(lo.assemble(_vector_cell(nu * Kl + (q1_convection_matrix(h, wind) if wind is not None
                                                           else 0.0), 3), 3, 3), 3, 3),
        (3, 3): lo.bsr(lo.assemble(-tau * Kl, 1, 1), 1, 1),
        (2, 3): lo.bsr(lo.assemble(Gd, 3, 1), 3, 1),
        (3, 2): lo.bsr(lo.assemble(Gd.T.copy(), 1, 3), 1, 3),
        (2, 1): lo.bsr(lo.assemble(eta * _vector_cell(Dz, 3), 3, 3), 3, 3),
    }
    Mup = _interface_nodes(up, 0)        # S side of the interface (local layer 0)
    Mlo = _interface_nodes(lo, nz)       # fluid / mesh side (top layer of the lower half)
    _add_to_grid_block(up, blocks[(0, 0)].vals, Mup, gamma, 3)
    _add_to_grid_block(lo, blocks[(2, 2)].vals, Mlo, 2 * gamma, 3)
    _add_to_grid_block(lo, blocks[(1, 1)].vals, Mlo, gamma, 3)
    # S <-> Fu: upper layer-0 node (i, j) pairs with lower layer-nz node (i, j)
    shift = nz * lo.stride[2]
    Mx = Mlo.tocoo()
    rows_up = Mx.row - shift
    import scipy.sparse as sp
    Msf = sp.csr_matrix((Mx.data, (rows_up, Mx.col)), shape=(up.nnodes, lo.nnodes))
    blocks[(0, 2)] = _node_bsr(Msf, 3, -gamma)
    blocks[(2, 0)] = _node_bsr(Msf.T.tocsr(), 3, -gamma)
    blocks[(1, 2)] = _node_bsr(Mlo, 3, -gamma)
    dS = up.ijk[:, 2] == (ne - nz)
    xi, yi, zi = lo.ijk[:, 0], lo.ijk[:, 1], lo.ijk[:, 2]
    lateral = (xi == 0) | (xi == ne) | (yi == 0) | (yi == ne)
    dG = lateral | (zi == 0)
    dF = lateral
    dP = zi == 0
    _dirichlet_fields(blocks, [dS, dG, dF, dP])
    fields = [
        Field("structure", 3, up.nnodes, 3, up.coords, "rbm", 0.0, np.nonzero(dS)[0]),
        Field("mesh", 3, lo.nnodes, 3, lo.coords, "const", 0.0, np.nonzero(dG)[0]),
        Field("fluid_velocity", 3, lo.nnodes, 3, lo.coords, "const", 0.0, np.nonzero(dF)[0],
              petrov_galerkin=wind is not None),
        Field("fluid_pressure", 1, lo.nnodes, 3, lo.coords, "const", 0.0, np.nonzero(dP)[0]),
    ]
    rng = np.random.default_rng(seed)
    rhs = rng.standard_normal(sum(f.ndofs for f in fields))
    off = 0
    for f in fields:
        d = (f.dirichlet_nodes[:, None] * f.b + np.arange(f.b)[None, :]).ravel()
        rhs[off + d] = 0.0
        off += f.ndofs
    name = f"fsi_box_ne{ne}" if wind is None else f"oseen_fsi_box_ne{ne}"
    return BlockSystem(fields, blocks, rhs, name=name, meta=dict(ne=ne, nu=nu, seed=seed, wind=wind))


def batch_sizes_log_uniform(nsys=256, lo=12, hi=48, seed=3):
    """Per-system mesh edge n_e = round(exp(U(ln lo, ln hi)))."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=nsys))).astype(int)


def system_rhs(system, seed):
    """A fresh seeded N(0,1) right-hand side for an existing system (zero on
    its Dirichlet nodes)."""
    return _seeded_rhs(system.fields, seed, system.fields[0].dirichlet_nodes)


def batch_workload(nsys=256, lo=12, hi=48, seed=3, nfields=2):
    """Batch of independent 3D coupled boxes: mesh edge n_e log-uniform in
    [lo, hi] per system (the matrix depends on n_e only), right-hand side
    seeded with seed*1000 + k.  Returns (sizes, {n_e: BlockSystem}, [rhs_k])."""
    sizes = batch_sizes_log_uniform(nsys, lo, hi, seed)
    mats = {int(ne): coupled_box_3d(ne=int(ne), nfields=nfields, seed=seed) for ne in sorted(set(sizes.tolist()))}
    rhs = [system_rhs(mats[int(ne)], seed * 1000 + k) for k, ne in enumerate(sizes)]
    return sizes, mats, rhs
