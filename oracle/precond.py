"""Block preconditioners for the N x N system A x = b, FP64.

TEST INFRASTRUCTURE (oracle).  Each preconditioner is the stationary block
method run for k_max sweeps from x^(0) = 0 (Sec. 7.1 uses k_max = 1):

* BGS (Sec. 4.1): x^(k) = x^(k-1) + M_BGS^-1 (b - A x^(k-1)).  In field form a
  forward sweep visits i = 1..N and sets
      x_i <- x_i + A_ii^-1 [b_i - sum_j A_ij x_j]
  with the latest x_j - the field-form equation of Sec. 4.1 with the sign of
  its second sum corrected to minus (that is what M_BGS = lower block
  triangle gives).  Backward visits i = N..1 (M_BGS = upper block triangle);
  symmetric does a forward then a backward sweep.  A_ii^-1 is one AMG
  V-cycle (BGS(AMG)) or, for checks, an exact solve.
* SIMPLE (Sec. 4.2): the predictor / Schur / update steps of the SIMPLE
  iteration with x^(0) = 0, so the A_22 x_2 term of the Schur right-hand
  side vanishes; fields are merged into a predictor group and a Schur group
  (Sec. 4.2, merging for N > 2); a multi-field predictor group is solved by
  one BGS(AMG) sweep or, with simple_pred = "amg_bgs", one monolithic
  AMG(BGS) V-cycle (SIMPLE(BGS(AMG)) and SIMPLE(AMG(BGS)) of Sec. 6.3); a
  Schur group at or below coarse_max dofs gets a one-level hierarchy, i.e. the
  dense LU of S~ (Sec. 6.3 solves the small constraint Schur complement
  directly).
  A~_11 is SIMPLEC's diagonal of absolute row sums of the merged A_11 block
  (read as the sum of absolute entries of each row) or, optionally, diag(A_11).
  S~ = A_22 - A_21 A~_11^-1 A_12 is formed explicitly.
* monolithic AMG(SIMPLE) (Sec. 4.3): the same V-cycle with a SIMPLE step as
  level smoother (see MonoAMGSimple).
* monolithic AMG(BGS) (Sec. 4.3): block-diagonal transfers diag(P_i),
  diag(R_i) from the single-field hierarchies, coarse blocks
  A^{l+1}_ij = R_i A^l_ij P_j, a V-cycle whose level smoother is a BGS sweep
  over the fields with the single-field smoothers S^l_i as block solvers, and
  a direct solve of the assembled coupled coarsest matrix.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import amg
from .cycles import SmootherParams, gauss_seidel, smooth, vcycle


class Params:
    """Mirrors the solver library's parameter block."""

    def __init__(self, precond="bgs_amg", bgs_order="bwd", bgs_sweeps=1, simple_group=None,
                 simple_approx="absrowsum", max_levels=4, coarse_max=1000, seed=7,
                 smoother=None, simple_pred="bgs_amg"):
        self.precond = precond
        self.bgs_order = bgs_order
        self.bgs_sweeps = bgs_sweeps
        self.simple_group = simple_group
        self.simple_approx = simple_approx
        self.max_levels = max_levels
        self.coarse_max = coarse_max
        self.seed = seed
        self.smoother = smoother or SmootherParams()
        self.simple_pred = simple_pred


def split(v, sizes):
    out, o = [], 0
    for n in sizes:
        out.append(v[o:o + n])
        o += n
    return out


def coupled_matvec(blocks, x, nf):
    """y_i = sum_j A_ij x_j over the nonzero blocks."""
    y = [np.zeros(blocks[(i, i)].shape[0]) for i in range(nf)]
    for (i, j), M in blocks.items():
        y[i] = y[i] + M @ x[j]
    return y


def assemble(blocks, nf):
    return sp.bmat([[blocks.get((i, j)) for j in range(nf)] for i in range(nf)], format="csr")


def sweep_orders(order, nf):
    fwd, bwd = list(range(nf)), list(range(nf - 1, -1, -1))
    return {"fwd": [fwd], "bwd": [bwd], "sym": [fwd, bwd]}[order]


class AMGLeaf:
    """A_ii^-1 ~ one V-cycle of field i of a group hierarchy."""

    def __init__(self, levels, i, coarse, sp_):
        self.levels, self.i, self.coarse, self.sp = levels, i, coarse, sp_

    def __call__(self, b):
        return vcycle(self.levels, self.i, self.coarse, b, self.sp)


class DirectLeaf:
    def __init__(self, M):
        self.lu = spla.splu(sp.csc_matrix(M))

    def __call__(self, b):
        return self.lu.solve(b)


class GSLeaf:
    """Block solver of the single-level BGS(GS): Gauss-Seidel sweeps from zero
    (forward colour order) on the fine diagonal block."""

    def __init__(self, A, b, sp_):
        if sp_.kind != "gs":
            raise ValueError("BGS(GS) needs the Gauss-Seidel smoother")
        self.fl = amg.FieldLevel(A, b)
        if not np.all(np.isfinite(self.fl.dinv)):
            raise ValueError("zero diagonal entry in a diagonal block")
        self.sp = sp_

    def __call__(self, b):
        return gauss_seidel(self.fl, b, np.zeros_like(b), self.sp.omega, self.sp.sweeps)


class BGS:
    """Block Gauss-Seidel over fields 0..nf-1 of `blocks` with block solvers."""

    def __init__(self, blocks, nf, solvers, order="bwd", sweeps=1):
        self.blocks, self.nf, self.solvers = blocks, nf, solvers
        self.order, self.sweeps = order, sweeps

    def __call__(self, b):
        nf = self.nf
        x = [np.zeros_like(bi) for bi in b]
        for _ in range(self.sweeps):
            for seq in sweep_orders(self.order, nf):
                for i in seq:
                    c = b[i].copy()
                    for j in range(nf):
                        M = self.blocks.get((i, j))
                        if M is not None:
                            c = c - M @ x[j]
                    x[i] = x[i] + self.solvers[i](c)
        return x


class SIMPLE:
    """SIMPLE step with x^(0) = 0 on a 2 x 2 grouping of fields.
    pred / schur act on lists of group vectors; a11t_inv applies A~_11^-1."""

    def __init__(self, blocks, g1, g2, pred, schur, a11t_inv):
        self.blocks, self.g1, self.g2 = blocks, g1, g2
        self.pred, self.schur, self.a11t_inv = pred, schur, a11t_inv

    def __call__(self, b):
        g1, g2, A = self.g1, self.g2, self.blocks
        dx1 = self.pred([b[j] for j in g1])
        r2 = []
        for k in g2:
            r = b[k].copy()
            for jj, j in enumerate(g1):
                if (k, j) in A:
                    r = r - A[(k, j)] @ dx1[jj]
            r2.append(r)
        dx2 = self.schur(r2)
        t = []
        for j in g1:
            s = np.zeros(A[(j, j)].shape[0])
            for kk, k in enumerate(g2):
                if (j, k) in A:
                    s = s + A[(j, k)] @ dx2[kk]
            t.append(s)
        corr = self.a11t_inv(t)
        x = [None] * (len(g1) + len(g2))
        for jj, j in enumerate(g1):
            x[j] = dx1[jj] - corr[jj]
        for kk, k in enumerate(g2):
            x[k] = dx2[kk]
        return x


def simple_dtilde(blocks, g1, approx):
    """Diagonal A~_11 of the merged predictor block, one vector per field."""
    out = []
    for j in g1:
        if approx == "diag":
            out.append(blocks[(j, j)].diagonal().copy())
        elif approx == "absrowsum":
            s = np.zeros(blocks[(j, j)].shape[0])
            for l in g1:
                if (j, l) in blocks:
                    s = s + np.asarray(abs(blocks[(j, l)]).sum(axis=1)).ravel()
            out.append(s)
        else:
            raise ValueError(approx)
    return out


def simple_schur(blocks, g1, g2, dtilde):
    """Explicit S~_kl = A_kl - sum_j A_kj diag(1/d~_j) A_jl for k, l in the Schur group."""
    S = {}
    for kk, k in enumerate(g2):
        for ll, l in enumerate(g2):
            M = blocks.get((k, l))
            M = M.copy() if M is not None else None
            for jj, j in enumerate(g1):
                if (k, j) in blocks and (j, l) in blocks:
                    T = blocks[(k, j)] @ sp.diags(1.0 / dtilde[jj]) @ blocks[(j, l)]
                    M = -T if M is None else M - T
            if M is not None:
                S[(kk, ll)] = M.tocsr()
    return S


class GroupAMG:
    """Single-field hierarchies of a group of fields + one coarse LU each."""

    def __init__(self, diag_blocks, specs, prm):
        self.levels = amg.build_group(diag_blocks, specs, prm.max_levels, prm.coarse_max, prm.seed)
        self.coarse = [amg.DenseLU(fl.A) for fl in self.levels[-1]]
        self.sp = prm.smoother

    def leaf(self, i):
        return AMGLeaf(self.levels, i, self.coarse[i], self.sp)


def bgs_amg_over(blocks, specs, prm, nf):
    grp = GroupAMG([blocks[(i, i)] for i in range(nf)], specs, prm)
    if nf == 1:
        leaf = grp.leaf(0)
        return (lambda b: [leaf(b[0])]), grp
    return BGS(blocks, nf, [grp.leaf(i) for i in range(nf)], prm.bgs_order, prm.bgs_sweeps), grp


def sub_blocks(blocks, idx):
    pos = {g: k for k, g in enumerate(idx)}
    return {(pos[i], pos[j]): M for (i, j), M in blocks.items() if i in pos and j in pos}


class MonoAMG:
    """Monolithic AMG(BGS): coupled V-cycle with BGS level smoothing."""

    def __init__(self, blocks, specs, prm, nf):
        self.nf = nf
        self.grp = GroupAMG([blocks[(i, i)] for i in range(nf)], specs, prm)
        lv = self.grp.levels
        self.A = [dict(blocks)]
        for l in range(len(lv) - 1):
            nxt = {}
            for (i, j), M in self.A[-1].items():
                if i == j:
                    nxt[(i, j)] = lv[l + 1][i].A
                else:
                    nxt[(i, j)] = amg.coarse_block(lv[l][i].R, M, lv[l][j].P)
            self.A.append(nxt)
        self.coarse = amg.DenseLU(assemble(self.A[-1], nf))
        self.prm = prm

    def smooth(self, l, b, x, post=False):
        lv, A = self.grp.levels[l], self.A[l]
        for _ in range(self.prm.bgs_sweeps):
            for seq in sweep_orders(self.prm.bgs_order, self.nf):
                for i in seq:
                    c = b[i].copy()
                    for j in range(self.nf):
                        if j != i and (i, j) in A:
                            c = c - A[(i, j)] @ x[j]
                    x[i] = smooth(lv[i], c, x[i], self.prm.smoother, post)
        return x

    def cycle(self, l, b):
        lv = self.grp.levels
        if l == len(lv) - 1:
            sizes = [bi.shape[0] for bi in b]
            return split(self.coarse.solve(np.concatenate(b)), sizes)
        x = [np.zeros_like(bi) for bi in b]
        x = self.smooth(l, b, x)
        Ax = coupled_matvec(self.A[l], x, self.nf)
        bc = [lv[l][i].R @ (b[i] - Ax[i]) for i in range(self.nf)]
        xc = self.cycle(l + 1, bc)
        x = [x[i] + lv[l][i].P @ xc[i] for i in range(self.nf)]
        return self.smooth(l, b, x, post=True)

    def __call__(self, b):
        return self.cycle(0, list(b))


class MonoAMGSimple(MonoAMG):
    """Monolithic AMG(SIMPLE) (Sec. 4.3): the coupled V-cycle of AMG(BGS) with a
    SIMPLE step as level smoother.  On level l, with residual r = b - A^l x:
    predictor  d_1 = one BGS sweep over the predictor fields, each block solve
               one application of the single-field smoother S^l_i from zero;
    Schur      d_2 = one application of a Chebyshev smoother on the explicit
               S~^l = A^l_22 - A^l_21 (A~^l_11)^-1 A^l_12 (its own lambda), from zero,
               with right-hand side r_2 - A^l_21 d_1;
    update     d_1 -= (A~^l_11)^-1 A^l_12 d_2;  x += d.
    A~^l_11 is SIMPLEC / diagonal of the level's merged predictor block; one
    Schur field."""

    def __init__(self, blocks, specs, prm, nf, g1, g2):
        super().__init__(blocks, specs, prm, nf)
        if len(g2) != 1:
            raise ValueError("AMG(SIMPLE) takes one Schur field")
        self.g1, self.g2 = g1, g2
        self.dt, self.S = [], []
        for l in range(len(self.grp.levels) - 1):
            dt = simple_dtilde(self.A[l], g1, prm.simple_approx)
            S = simple_schur(self.A[l], g1, g2, dt)[(0, 0)]
            fl = amg.FieldLevel(S, specs[g2[0]].b)
            fl.lam = amg.power_lambda(fl.A, fl.dinv, prm.seed)
            self.dt.append(dt)
            self.S.append(fl)

    def smooth(self, l, b, x, post=False):
        lv, A, sp_ = self.grp.levels[l], self.A[l], self.prm.smoother
        g1, k = self.g1, self.g2[0]
        for _ in range(self.prm.bgs_sweeps):
            Ax = coupled_matvec(A, x, self.nf)
            r = [b[i] - Ax[i] for i in range(self.nf)]
            d = {}
            for seq in sweep_orders(self.prm.bgs_order, len(g1)):
                for jj in seq:
                    i = g1[jj]
                    c = r[i].copy()
                    for j in d:
                        if j != i and (i, j) in A:
                            c = c - A[(i, j)] @ d[j]
                    d[i] = (d[i] if i in d else 0.0) + smooth(lv[i], c - (A[(i, i)] @ d[i] if i in d else 0.0),
                                                             np.zeros_like(c), sp_, post)
            c2 = r[k].copy()
            for j in g1:
                if (k, j) in A:
                    c2 = c2 - A[(k, j)] @ d[j]
            d2 = smooth(self.S[l], c2, np.zeros_like(c2), sp_, post)
            for jj, j in enumerate(g1):
                if (j, k) in A:
                    d[j] = d[j] - (A[(j, k)] @ d2) / self.dt[l][jj]
            for j in g1:
                x[j] = x[j] + d[j]
            x[k] = x[k] + d2
        return x


class Preconditioner:
    """z = M^-1 v for the whole coupled vector (field-major concatenation)."""

    def __init__(self, blocks, specs, prm):
        nf = len(specs)
        self.sizes = [blocks[(i, i)].shape[0] for i in range(nf)]
        self.prm = prm
        if prm.precond == "bgs_amg":
            self.op, self.grp = bgs_amg_over(blocks, specs, prm, nf)
            self.groups = [self.grp]
        elif prm.precond == "amg_bgs":
            self.op = MonoAMG(blocks, specs, prm, nf)
            self.grp = self.op.grp
            self.groups = [self.grp]
        elif prm.precond == "amg_simple":
            grp_of = prm.simple_group or [0] * (nf - 1) + [1]
            g1 = [i for i in range(nf) if grp_of[i] == 0]
            g2 = [i for i in range(nf) if grp_of[i] == 1]
            self.op = MonoAMGSimple(blocks, specs, prm, nf, g1, g2)
            self.grp = self.op.grp
            self.groups = [self.grp]
        elif prm.precond == "bgs_gs":
            # single-level BGS(DD(GS)) of Sec. 7.1 on one subdomain: each block
            # solve is prm.smoother's Gauss-Seidel sweeps from zero on A_ii
            leaves = [GSLeaf(blocks[(i, i)], specs[i].b, prm.smoother) for i in range(nf)]
            self.op = BGS(blocks, nf, leaves, prm.bgs_order, prm.bgs_sweeps)
            self.groups = []
        elif prm.precond == "simple":
            grp_of = prm.simple_group or [0] * (nf - 1) + [1]
            g1 = [i for i in range(nf) if grp_of[i] == 0]
            g2 = [i for i in range(nf) if grp_of[i] == 1]
            if prm.simple_pred == "amg_bgs":
                pred = MonoAMG(sub_blocks(blocks, g1), [specs[i] for i in g1], prm, len(g1))
                grp1 = pred.grp
            else:
                pred, grp1 = bgs_amg_over(sub_blocks(blocks, g1), [specs[i] for i in g1], prm, len(g1))
            dt = simple_dtilde(blocks, g1, prm.simple_approx)
            S = simple_schur(blocks, g1, g2, dt)
            sspecs = [amg.FieldSpec(specs[k].b, specs[k].dim, "const", None, specs[k].theta) for k in g2]
            schur, grp2 = bgs_amg_over(S, sspecs, prm, len(g2))
            self.dtilde, self.schur_blocks = dt, S
            self.op = SIMPLE(blocks, g1, g2, pred, schur, lambda t: [ti / d for ti, d in zip(t, dt)])
            self.groups = [grp1, grp2]
        else:
            raise ValueError(prm.precond)

    def __call__(self, v):
        return np.concatenate(self.op(split(v, self.sizes)))
