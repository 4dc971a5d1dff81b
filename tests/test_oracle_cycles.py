"""Pins for the oracle's smoother and V-cycle (Algorithm 1), CPU only."""
import numpy as np
import scipy.sparse as sp
import pytest

from oracle import amg
from oracle.cycles import chebyshev, jacobi, vcycle, SmootherParams
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
