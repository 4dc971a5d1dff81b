"""Build oracle preconditioners from a libmfs handle's exported hierarchy.

Used by the GPU parity tests so that the CUDA apply and the oracle apply run
on the same multigrid objects (aggregates, P, R, coarse blocks, lambda):
then the two may differ only by floating-point rounding.
"""
import numpy as np

from oracle import amg, precond
from oracle.cycles import SmootherParams


def _colors(lib, fl, group, l, i):
    """Gauss-Seidel colours exported by the library (equal to the oracle's own
    node_colors on the same matrix; taken over so both sweep one order)."""
    c = lib.export_array("colors", group, l, i)
    fl.colors = c
    fl.b = fl.A.shape[0] // len(c)


def _levels(lib, group, nf, blocks_b, smoothed_all=False):
    L = lib.num_levels(group)
    gs = lib.params.smoother == 2
    levels = []
    for l in range(L):
        row = []
        for i in range(nf):
            A = lib.export_csr("A", group, l, i, i)
            fl = amg.FieldLevel(A, blocks_b[i] if l == 0 else None)
            if l < L - 1:
                fl.P = lib.export_csr("P", group, l, i)
                fl.R = lib.export_csr("R", group, l, i)
                fl.lam = lib.export_array("lambda", group, l, i)
                fl.agg = lib.export_array("agg", group, l, i)
            if gs and (l < L - 1 or smoothed_all):
                _colors(lib, fl, group, l, i)
            row.append(fl)
        levels.append(row)
    return levels


class _Grp:
    def __init__(self, levels, sp_):
        self.levels = levels
        self.coarse = [amg.DenseLU(fl.A) for fl in levels[-1]]
        self.sp = sp_

    def leaf(self, i):
        return precond.AMGLeaf(self.levels, i, self.coarse[i], self.sp)


def smoother_params(p):
    if p.smoother == 2:
        return SmootherParams("gs", omega=p.gs_omega, sweeps=p.gs_sweeps)
    if p.smoother == 1:
        return SmootherParams("jacobi", omega=p.jacobi_omega, sweeps=p.jacobi_sweeps)
    return SmootherParams("chebyshev", degree=p.cheb_degree, ratio=p.cheb_ratio, boost=p.cheb_boost)


def oracle_preconditioner(lib, system):
    """Oracle preconditioner callable (full vector -> full vector) on lib's hierarchy."""
    p = lib.params
    sp_ = smoother_params(p)
    order = {0: "bwd", 1: "fwd", 2: "sym"}[p.bgs_order]
    nf = system.nfields
    A = system.scipy_blocks()
    sizes = [f.ndofs for f in system.fields]
    bsz = [f.b for f in system.fields]
    kind = p.precond
    sg = list(p.simple_group)[:nf]
    if not any(sg):
        sg = [0] * (nf - 1) + [1]
    g1 = [i for i in range(nf) if sg[i] == 0]
    g2 = [i for i in range(nf) if sg[i] == 1]

    def monolithic(cls, name, Afine, nfg, grp):
        # AMG(BGS)-type hierarchy of group 0 from the exported blockwise Galerkin blocks
        mono = cls.__new__(cls)
        mono.nf = nfg
        mono.grp = grp
        mono.prm = precond.Params(name, bgs_order=order, bgs_sweeps=p.bgs_sweeps, smoother=sp_)
        mono.A = [dict(Afine)]
        for l in range(1, len(grp.levels)):
            d = {}
            for (i, j) in Afine:
                d[(i, j)] = grp.levels[l][i].A if i == j else lib.export_csr("A", 0, l, i, j)
            mono.A.append(d)
        mono.coarse = amg.DenseLU(precond.assemble(mono.A[-1], nfg))
        return mono

    if kind == 4:
        # single-level BGS(GS): Gauss-Seidel sweeps on the exported fine blocks
        leaves = []
        for i in range(nf):
            lf = precond.GSLeaf(lib.export_csr("A", 0, 0, i, i), bsz[i], sp_)
            _colors(lib, lf.fl, 0, 0, i)
            leaves.append(lf)
        op = precond.BGS(A, nf, leaves, order, p.bgs_sweeps)
        return lambda v: np.concatenate(op(precond.split(v, sizes)))
    if kind in (0, 2, 3):
        grp = _Grp(_levels(lib, 0, nf, bsz), sp_)
        if kind == 0:
            op = precond.BGS(A, nf, [grp.leaf(i) for i in range(nf)], order, p.bgs_sweeps)
        else:
            mono = monolithic(precond.MonoAMG if kind == 2 else precond.MonoAMGSimple,
                              "amg_bgs" if kind == 2 else "amg_simple", A, nf, grp)
            if kind == 3:
                # level Schur complements S~^l (group 1) and A~_11 per level
                mono.g1, mono.g2 = g1, g2
                mono.S, mono.dt = [], []
                for l in range(len(grp.levels) - 1):
                    fl = amg.FieldLevel(lib.export_csr("A", 1, l, 0, 0), None)
                    fl.lam = lib.export_array("lambda", 1, l, 0)
                    if p.smoother == 2:
                        _colors(lib, fl, 1, l, 0)
                    mono.S.append(fl)
                    mono.dt.append([lib.export_array("dtilde", 0, l, jj) for jj in range(len(g1))])
            op = mono
    else:
        grp0 = _Grp(_levels(lib, 0, len(g1), [bsz[i] for i in g1]), sp_)
        grp1 = _Grp(_levels(lib, 1, len(g2), [bsz[i] for i in g2]), sp_)
        sub = precond.sub_blocks(A, g1)
        if p.simple_pred == 1:
            pred = monolithic(precond.MonoAMG, "amg_bgs", sub, len(g1), grp0)
        elif len(g1) == 1:
            leaf = grp0.leaf(0)
            pred = lambda b: [leaf(b[0])]
        else:
            pred = precond.BGS(sub, len(g1), [grp0.leaf(i) for i in range(len(g1))], order, p.bgs_sweeps)
        S = {}
        for kk in range(len(g2)):
            for ll in range(len(g2)):
                try:
                    S[(kk, ll)] = lib.export_csr("A", 1, 0, kk, ll)
                except Exception:
                    pass
        if len(g2) == 1:
            sleaf = grp1.leaf(0)
            schur = lambda b: [sleaf(b[0])]
        else:
            schur = precond.BGS(S, len(g2), [grp1.leaf(i) for i in range(len(g2))], order, p.bgs_sweeps)
        dt = [lib.export_array("dtilde", 0, 0, jj) for jj in range(len(g1))]
        op = precond.SIMPLE(A, g1, g2, pred, schur, lambda t: [ti / d for ti, d in zip(t, dt)])
    return lambda v: np.concatenate(op(precond.split(v, sizes)))
