"""MINRES for symmetric (possibly indefinite) systems, oracle version.

The paper solves the small shifted systems (H0_hat - E_k^(0)) x1 = b1 of
Eq. (sm_lin_proj) with an iterative method and names MINRES as one choice
(Sec. 4.3).  This is MINRES as published by Paige and Saunders (1975): the
Lanczos three-term recurrence builds an orthonormal Krylov basis V_j with
A V_j = V_{j+1} T_j; the least-squares problem min ||beta1 e1 - T_j y|| is
solved by a QR factorisation of T_j kept up to date with one Givens rotation
per step; the iterate x_j = V_j y_j is updated through the search directions
W_j = V_j R_j^{-1} (three-term recurrence).  Residual norms come from the
rotations, so no extra product is needed.

Reading used here (the paper is silent): x0 = 0, no preconditioner, stop when
the (recurrence) residual norm is <= tol * ||b|| or after maxit steps.
"""
from __future__ import annotations

import numpy as np


def minres(apply_a, b: np.ndarray, tol: float = 1e-12, maxit: int | None = None):
    """Solve A x = b for symmetric A given as a function v -> A v.

    Returns (x, iterations, residual_norm_estimate).  b == 0 returns x = 0.
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    if maxit is None:
        maxit = n
    x = np.zeros(n)
    beta1 = float(np.linalg.norm(b))
    if beta1 == 0.0:
        return x, 0, 0.0
    v_prev = np.zeros(n)
    v = b / beta1
    beta = beta1            # beta_j (couples v_j and v_{j-1})
    eta = beta1             # running right-hand side of the rotated system
    # rotation cosines/sines of the two previous steps
    c_prev, c_cur = 1.0, 1.0
    s_prev, s_cur = 0.0, 0.0
    w_prev2 = np.zeros(n)
    w_prev1 = np.zeros(n)
    rnorm = beta1
    it = 0
    for it in range(1, maxit + 1):
        # Lanczos step: A v_j = beta_j v_{j-1} + alpha_j v_j + beta_{j+1} v_{j+1}
        p = apply_a(v) - beta * v_prev
        alpha = float(v @ p)
        p = p - alpha * v
        beta_next = float(np.linalg.norm(p))
        # new column of T_j is (beta_j, alpha_j, beta_{j+1}); apply the two
        # previous rotations, then form the new one that zeroes beta_{j+1}
        delta = c_cur * alpha - c_prev * s_cur * beta
        rho1 = float(np.hypot(delta, beta_next))
        rho2 = s_cur * alpha + c_prev * c_cur * beta
        rho3 = s_prev * beta
        if rho1 == 0.0:
            break
        c_next = delta / rho1
        s_next = beta_next / rho1
        w = (v - rho3 * w_prev2 - rho2 * w_prev1) / rho1
        x = x + (c_next * eta) * w
        rnorm = abs(s_next) * rnorm
        eta = -s_next * eta
        # shift the recurrences
        w_prev2, w_prev1 = w_prev1, w
        c_prev, c_cur = c_cur, c_next
        s_prev, s_cur = s_cur, s_next
        if rnorm <= tol * beta1 or beta_next == 0.0:
            break
        v_prev = v
        v = p / beta_next
        beta = beta_next
    return x, it, rnorm
