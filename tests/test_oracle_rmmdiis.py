"""Pins of the RMM-DIIS oracle (oracle/rmmdiis.py): the DIIS coefficients
against their optimality conditions and a brute-force minimiser, the depth-1
special case, and convergence to eigenpairs of a dense-diagonalised matrix."""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle.rmmdiis as R
from conftest import dense, make_matrix


def test_diis_coefficients_are_the_constrained_minimiser():
    rng = np.random.Generator(np.random.PCG64(1))
    for m in (1, 2, 5, 8):
        V = rng.standard_normal((40, m))
        G = V.T @ V
        c = R.diis_coefficients(G)
        assert abs(c.sum() - 1.0) < 1e-12
        # KKT: G c is a constant vector (the multiplier), up to the regularisation
        g = G @ c
        assert np.ptp(g) <= 1e-9 * max(1.0, np.abs(g).max())
        # brute force on the affine set sum c = 1
        f = lambda t: float(np.sum((V @ np.concatenate([t, [1.0 - t.sum()]])) ** 2))  # noqa: E731
        best = minimize(f, np.zeros(m - 1), method="BFGS", tol=1e-14).x if m > 1 else np.zeros(0)
        cb = np.concatenate([best, [1.0 - best.sum()]])
        assert np.allclose(c, cb, atol=1e-5)


def test_depth_one_is_the_preconditioned_residual_step():
    """With a history of one, c = [1] and the update is x - (D - theta)^-1 r."""
    w, rp, c, v = make_matrix("small")
    A = dense(rp, c, v)
    rng = np.random.Generator(np.random.PCG64(2))
    x0 = rng.standard_normal((w.n, 1))
    th, rs, done, rec = R.rmm_diis(rp, c, v, x0, tol=0.0, maxit=1, depth=1)
    x = x0[:, 0] / np.linalg.norm(x0)
    t = x @ A @ x
    r = A @ x - t * x
    x1 = x - R.shifted_diag_inv(np.diag(A).copy(), t, 1e-2) * r
    x1 /= np.linalg.norm(x1)
    # the second record is the Rayleigh quotient of x1
    assert np.isclose(rec[1].theta[0], x1 @ A @ x1, rtol=1e-13)


def test_sppc_rmm_converges_to_eigenpairs():
    """From SPPC's Ritz vectors each pair converges to an eigenpair of H (the
    lowest, well separated, to the lowest eigenvalue); no pair goes below
    lambda_min (Rayleigh quotients)."""
    w, rp, c, v = make_matrix("small")
    lam = np.linalg.eigvalsh(dense(rp, c, v))
    th, rs, conv, r, rec = R.sppc_rmm(rp, c, v, w.small_dim, w.k, switch_order=4, tol=1e-8, maxit=1000)
    assert conv and np.all(rs <= 1e-8)
    for t in th:
        assert np.min(np.abs(lam - t)) <= 1e-9 * abs(t)
    assert np.isclose(th[0], lam[0], rtol=1e-10)
    assert np.all(th >= lam[0] - 1e-10 * abs(lam[0]))
    # one SpMV per running pair and iteration
    assert rec[0].spmv == w.k
