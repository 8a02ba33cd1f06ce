"""SPPC followed by per-pair RMM-DIIS (paper Sec. 6): plain FP64 reference (test
infrastructure only).

The paper switches from SPPC to RMM-DIIS (residual minimisation with direct
inversion in the iterative subspace; Wood and Zunger 1985, Kresse and
Furthmueller 1996) once SPPC stagnates, refining each eigenpair separately from
its Ritz vector at the switch, one SpMV per pair and iteration, with a diagonal
preconditioner.  The paper leaves the preconditioner, the history length and
the step length open.  Reading used here (the GPU path takes the same steps):

For each pair j independently, from x_0 = z_j / ||z_j||:
 1. w = H x; theta = x^T w / x^T x; r = w - theta x; rho = ||r|| / |theta|.
    Stop (the pair is frozen) once rho <= tol.
 2. Append (x, r) to the history; keep the last `depth` (default 8) entries.
 3. DIIS: c minimises ||sum_a c_a r_a|| subject to sum_a c_a = 1, from the
    bordered system [G 1; 1^T 0] [c; mu] = [0; 1] with G_ab = r_a^T r_b
    (G's diagonal raised by 1e-14 max_a G_aa against exact singularity).
 4. x_bar = sum c_a x_a, r_bar = sum c_a r_a;
    x <- x_bar - lam (D - theta I)^-1 r_bar with D = diag(H), every |D_i - theta|
    clamped to >= clamp (the Jacobi preconditioner; lam = 1), then normalised.
No orthogonalisation between pairs (each pair is its own run, as in the paper).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .spmm import csr_spmm
from .sppc import sppc

DIIS_REG = 1e-14


@dataclass
class RMMRecord:
    it: int
    theta: np.ndarray
    resid: np.ndarray
    spmv: int


def diis_coefficients(G: np.ndarray) -> np.ndarray:
    """c minimising c^T G c subject to sum c = 1 (bordered system)."""
    m = G.shape[0]
    Gr = G + DIIS_REG * max(float(np.max(np.diag(G))), 1e-300) * np.eye(m)
    A = np.zeros((m + 1, m + 1))
    A[:m, :m] = Gr
    A[:m, m] = 1.0
    A[m, :m] = 1.0
    rhs = np.zeros(m + 1)
    rhs[m] = 1.0
    return np.linalg.solve(A, rhs)[:m]


def shifted_diag_inv(diag, theta: float, clamp: float):
    den = diag - theta
    small = np.abs(den) < clamp
    den[small] = np.where(den[small] >= 0, clamp, -clamp)
    return 1.0 / den


def rmm_diis(row_ptr, col, val, Z0: np.ndarray, tol: float, maxit: int, depth: int = 8, clamp: float = 1e-2,
             lam: float = 1.0):
    """Per-pair RMM-DIIS from the columns of Z0.  Returns (theta, resid, converged
    flags, records); every iteration costs one SpMV per pair still running."""
    n, k = Z0.shape
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    diag = np.zeros(n)
    on = rows == col
    diag[rows[on]] = val[on]
    X = Z0 / np.linalg.norm(Z0, axis=0)
    hist_x = [[] for _ in range(k)]
    hist_r = [[] for _ in range(k)]
    done = np.zeros(k, dtype=bool)
    theta = np.zeros(k)
    resid = np.zeros(k)
    records = []
    spmv = 0
    for it in range(maxit + 1):
        W = csr_spmm(row_ptr, col, val, X)
        spmv += int(np.count_nonzero(~done))
        for j in range(k):
            x, w = X[:, j], W[:, j]
            th = float(x @ w / (x @ x))
            r = w - th * x
            if not done[j]:
                theta[j] = th
                resid[j] = float(np.linalg.norm(r) / abs(th))
                if resid[j] <= tol:
                    done[j] = True
                    continue
                hist_x[j].append(x.copy())
                hist_r[j].append(r)
                if len(hist_x[j]) > depth:
                    hist_x[j].pop(0)
                    hist_r[j].pop(0)
                Rm = np.array(hist_r[j])
                c = diis_coefficients(Rm @ Rm.T)
                xb = c @ np.array(hist_x[j])
                rb = c @ Rm
                xn = xb - lam * shifted_diag_inv(diag, th, clamp) * rb
                X[:, j] = xn / np.linalg.norm(xn)
        records.append(RMMRecord(it, theta.copy(), resid.copy(), spmv))
        if done.all():
            break
    return theta, resid, done, records


def sppc_rmm(row_ptr, col, val, n1: int, k: int, *, switch_order: int = 15, tol: float = 1e-6, maxit: int = 500,
             depth: int = 8, clamp: float = 1e-2, lam: float = 1.0, solver: str = "pinv"):
    """SPPC (Algorithm 2) for switch_order orders (stopping early if converged),
    then per-pair RMM-DIIS from the last Ritz vectors.  Returns (theta, resid,
    converged, SPPC result, RMM-DIIS records)."""
    r = sppc(row_ptr, col, val, n1, k, p_max=switch_order, tol=tol, solver=solver, keep=True)
    if r.converged:
        return r.theta, r.resid, True, r, []
    Ht = r.Q.T @ r.W
    th, Y = np.linalg.eigh(0.5 * (Ht + Ht.T))
    Z0 = r.Q @ Y[:, :k]
    theta, resid, done, rec = rmm_diis(row_ptr, col, val, Z0, tol, maxit, depth, clamp, lam)
    return theta, resid, bool(done.all()), r, rec
