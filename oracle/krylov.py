"""Right-preconditioned flexible GMRES(m), FP64.

TEST INFRASTRUCTURE (oracle).  The accelerator solves (A P) y = b and
returns x = P y (Sec. 3.2, the right-preconditioned system), GMRES after
Saad & Schultz (Sec. 3.1).  Flexible form (Saad 1993): the preconditioned
vectors z_j = P v_j are stored and x = x0 + Z y, which equals right-
preconditioned GMRES for a fixed linear P.  Orthogonalisation is classical
Gram-Schmidt applied twice (CGS2); the least-squares problem is reduced by
Givens rotations.  Stopping rule (Sec. 7.1): ||r||_2 / ||r^0||_2 <= tol with
r^0 = b - A x0; the Givens estimate ends a cycle, the true residual decides
whether to stop or restart.  The iteration count is the number of
preconditioner applications.
"""
from __future__ import annotations

import numpy as np

BREAKDOWN = 1e-14


class Result:
    def __init__(self, x, iters, relres, est, history, converged, restarts):
        self.x, self.iters, self.relres, self.est = x, iters, relres, est
        self.history, self.converged, self.restarts = history, converged, restarts


def givens(a, b):
    """(c, s) with [c s; -s c] [a; b] = [r; 0]."""
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def fgmres(A, P, b, tol=1e-8, restart=50, maxiter=1000, x0=None):
    """A, P: callables on full vectors.  Returns a Result."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else x0.copy()
    r = b - A(x)
    r0 = np.linalg.norm(r)
    history = [1.0]
    if r0 == 0.0:
        return Result(x, 0, 0.0, 0.0, history, True, 0)
    iters, restarts = 0, 0
    est = 1.0
    while True:
        beta = np.linalg.norm(r)
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            Z[j] = P(V[j])
            w = A(Z[j])
            nw0 = np.linalg.norm(w)
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            H[:j + 1, j] = h + h2
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            for k in range(j):
                a, c = H[k, j], H[k + 1, j]
                H[k, j] = cs[k] * a + sn[k] * c
                H[k + 1, j] = -sn[k] * a + cs[k] * c
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            j_end = j + 1
            est = abs(g[j + 1]) / r0
            history.append(est)
            happy = hn <= BREAKDOWN * nw0
            if est <= tol or happy or iters >= maxiter:
                break
            V[j + 1] = w / hn
        y = np.zeros(j_end)
        for k in range(j_end - 1, -1, -1):
            y[k] = (g[k] - H[k, k + 1:j_end] @ y[k + 1:j_end]) / H[k, k]
        x = x + Z[:j_end].T @ y
        r = b - A(x)
        relres = np.linalg.norm(r) / r0
        if relres <= tol:
            return Result(x, iters, relres, est, history, True, restarts)
        if iters >= maxiter:
            return Result(x, iters, relres, est, history, False, restarts)
        restarts += 1
