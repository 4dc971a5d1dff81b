"""Smoothers and the multigrid V-cycle, FP64.

TEST INFRASTRUCTURE (oracle).

* Chebyshev smoother S(A, b, x): polynomial acceleration of the point-Jacobi
  iteration on D^-1 A over [lambda_max / ratio, boost * lambda_max] (Saad,
  "Iterative Methods for Sparse Linear Systems", Sec. 12.3, Chebyshev
  acceleration; ratio 30 and boost 1.1 as in Adams, Brezina, Hu & Tuminaro
  2003).  The paper's own smoother (Sec. 7.1: additive Schwarz with damped
  Gauss-Seidel) is replaced by this one.
* damped Jacobi x <- x + omega D^-1 (b - A x), the optional alternative.
* multicolour damped Gauss-Seidel, the GPU analogue of the paper's DD(GS(omega))
  (Sec. 7.1, omega = 0.79): nodes are coloured greedily (node_colors) so that
  no two coupled nodes share a colour; a forward sweep visits the colours in
  increasing order and inside a node its dofs in increasing order, setting
  x_p <- x_p + omega (b_p - sum_q a_pq x_q) / a_pp with the latest values,
  which is SOR(omega) in that ordering; nodes of one colour never couple, so
  they update together.  Pre-smoothing sweeps forward, post-smoothing
  backward (colours and dofs in decreasing order), so the V-cycle stays
  symmetric for symmetric blocks.
* V-cycle: Algorithm 1 - pre-smooth, restrict the residual, recurse with a
  zero initial guess, prolongate the correction, post-smooth; direct solve on
  the coarsest level.  The coarse operators come from the setup (the
  algorithm lists the Galerkin product inside the cycle; it does not depend
  on the iterate, so it is formed once).
"""
from __future__ import annotations

import numpy as np


class SmootherParams:
    def __init__(self, kind="chebyshev", degree=2, ratio=30.0, boost=1.1, omega=2.0 / 3.0, sweeps=1):
        self.kind, self.degree, self.ratio, self.boost = kind, degree, ratio, boost
        self.omega, self.sweeps = omega, sweeps


def chebyshev(A, dinv, lam, b, x, degree, ratio=30.0, boost=1.1):
    """Chebyshev polynomial smoother of the given degree (degree residual
    evaluations); returns the new iterate."""
    hi = boost * lam
    lo = lam / ratio
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = x.copy()
    r = b - A @ x
    d = (dinv * r) / theta
    x = x + d
    for _ in range(1, degree):
        r = b - A @ x
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = (rho_new * rho) * d + (2.0 * rho_new / delta) * (dinv * r)
        x = x + d
        rho = rho_new
    return x


def jacobi(A, dinv, b, x, omega, sweeps):
    x = x.copy()
    for _ in range(sweeps):
        x = x + omega * dinv * (b - A @ x)
    return x


# a block (i, j) couples nodes i != j when one of its entries exceeds this
# fraction of the largest entry of node i's rows (rounding-level Galerkin
# entries do not count)
COUPLING_REL = 1e-12


def node_colors(A, b):
    """Greedy node colouring of the point matrix A with b dofs per node: node
    i (in increasing order) takes the smallest colour not taken by a
    lower-numbered node it couples with (either direction)."""
    C = A.tocoo()
    n = A.shape[0] // b
    ri, ci = C.row.astype(np.int64) // b, C.col.astype(np.int64) // b
    rowmax = np.zeros(n)
    np.maximum.at(rowmax, ri, np.abs(C.data))
    keep = (ri != ci) & (np.abs(C.data) > COUPLING_REL * rowmax[ri])
    # symmetrised coupling graph as sorted unique neighbour lists
    e = np.unique(np.concatenate([ri[keep] * n + ci[keep], ci[keep] * n + ri[keep]]))
    src, dst = e // n, e % n
    ptr = np.searchsorted(src, np.arange(n + 1))
    color = np.full(n, -1, np.int64)
    for i in range(n):
        nb = dst[ptr[i]:ptr[i + 1]]
        taken = set(color[nb[nb < i]].tolist())
        c = 0
        while c in taken:
            c += 1
        color[i] = c
    return color


def gauss_seidel(fl, b, x, omega, sweeps, backward=False):
    """Multicolour damped Gauss-Seidel sweeps (see the module header)."""
    if getattr(fl, "colors", None) is None:
        fl.colors = node_colors(fl.A, fl.b)
    A, nb = fl.A, fl.b
    d = fl.A.diagonal()
    ncol = int(fl.colors.max()) + 1 if len(fl.colors) else 0
    x = x.copy()
    cols = range(ncol - 1, -1, -1) if backward else range(ncol)
    dofs = range(nb - 1, -1, -1) if backward else range(nb)
    for _ in range(sweeps):
        for c in cols:
            nodes = np.nonzero(fl.colors == c)[0]
            for r in dofs:
                p = nodes * nb + r
                x[p] = x[p] + omega * (b[p] - A[p] @ x) / d[p]
    return x


def smooth(fl, b, x, sp_, post=False):
    """Apply the single-field level smoother S^l_i of field-level `fl`
    (`post`: the application after the coarse correction)."""
    if sp_.kind == "chebyshev":
        return chebyshev(fl.A, fl.dinv, fl.lam, b, x, sp_.degree, sp_.ratio, sp_.boost)
    if sp_.kind == "jacobi":
        return jacobi(fl.A, fl.dinv, b, x, sp_.omega, sp_.sweeps)
    if sp_.kind == "gs":
        return gauss_seidel(fl, b, x, sp_.omega, sp_.sweeps, backward=post)
    raise ValueError(sp_.kind)


def vcycle(levels, i, coarse_solver, b, sp_, l=0):
    """Algorithm 1 for field i of a hierarchy levels[l][i]; x^l starts at 0."""
    fl = levels[l][i]
    if l == len(levels) - 1:
        return coarse_solver.solve(b)
    x = np.zeros_like(b)
    x = smooth(fl, b, x, sp_)
    bc = fl.R @ (b - fl.A @ x)
    xc = vcycle(levels, i, coarse_solver, bc, sp_, l + 1)
    x = x + fl.P @ xc
    x = smooth(fl, b, x, sp_, post=True)
    return x
