"""Smoothers and the multigrid V-cycle, FP64.

TEST INFRASTRUCTURE (oracle).

* Chebyshev smoother S(A, b, x): polynomial acceleration of the point-Jacobi
  iteration on D^-1 A over [lambda_max / ratio, boost * lambda_max] (Saad,
  "Iterative Methods for Sparse Linear Systems", Sec. 12.3, Chebyshev
  acceleration; ratio 30 and boost 1.1 as in Adams, Brezina, Hu & Tuminaro
  2003).  The paper's own smoother (Sec. 7.1: additive Schwarz with damped
  Gauss-Seidel) is replaced by this one.
* damped Jacobi x <- x + omega D^-1 (b - A x), the optional alternative.
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


def smooth(fl, b, x, sp_):
    """Apply the single-field level smoother S^l_i of field-level `fl`."""
    if sp_.kind == "chebyshev":
        return chebyshev(fl.A, fl.dinv, fl.lam, b, x, sp_.degree, sp_.ratio, sp_.boost)
    if sp_.kind == "jacobi":
        return jacobi(fl.A, fl.dinv, b, x, sp_.omega, sp_.sweeps)
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
    x = smooth(fl, b, x, sp_)
    return x
