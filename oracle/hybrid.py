"""SPPC followed by a block continuation once SPPC stagnates (paper Sec. 5 and 6).

The paper switches from SPPC to a second eigensolver that starts from SPPC's
eigenvector approximations when adding corrections stops improving the
subspace (around order 15); it lists Lanczos, block Lanczos, LOBPCG (with a
shifted block-diagonal preconditioner) and RMM-DIIS (with a diagonal
preconditioner) as partners.  Reading used here: the continuation keeps the
whole SPPC subspace and extends it, one block per step, with the residuals of
the k lowest Ritz pairs, preconditioned by the diagonal of H shifted by each
Ritz value (block Davidson, Davidson 1975 / Liu 1978); with the identity as
preconditioner the same loop extends the block Krylov space (block Lanczos
with full reorthogonalisation and thick restart).  When the basis would exceed
`max_blocks` blocks of k vectors it restarts from the 2k lowest Ritz vectors.

Step by step, from Q (orthonormal, n x m), W = H Q, Ht = Q^T W:
 1. k lowest eigenpairs (theta, Y) of the symmetrised Ht; Z = Q Y, R = W Y - Z theta;
    rho_j = ||R_j|| / |theta_j| (Eq. rrn); stop when every rho_j <= tol.
 2. T_j = R_j / (diag(H) - theta_j) elementwise, each denominator clamped to
    magnitude >= clamp (Jacobi preconditioner), or T = R without preconditioner.
    With precond="lead" the leading nl rows of T_j (nl = n1 unless lead_rows
    says otherwise; H_L = H[:nl, :nl]) are then replaced by an approximate
    solve with the leading block: z_hat = Z_j[:nl] / ||Z_j[:nl]||,
    P = I - z_hat z_hat^T, and `lead_iters` MINRES steps (x0 = 0, no stopping
    test) on P (H_L - theta_j) P t = P R_j[:nl], then t <- P t.  This is this
    repository's reading of the paper's shifted block-diagonal preconditioner:
    the exact leading block, shifted by the Ritz value and deflated by the Ritz
    vector (the projection of Jacobi-Davidson, Sleijpen and van der Vorst 1996),
    and the shifted diagonal on the other levels.
 3. Restart if m + k > max_blocks * k: Q <- Q Y_2k, W <- W Y_2k, Ht <- Q^T W.
 4. Phi = (I - Q Q^T) T; a second application when the first left some
    column with less than half of its norm (the reorthogonalisation criterion of
    Daniel, Gragg, Kaufman and Stewart, 1976, with the factor 1/2 of Kahan's
    "twice is enough" analysis; reorth="twice" always applies it);
    Phi = q R (Householder QR), Q <- [Q, q], W <- [W, H q], Ht bordered.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .minres import minres
from .spmm import csr_spmm
from .sppc import sppc


@dataclass
class HybridRecord:
    phase: str          # "sppc" or "davidson"
    step: int           # SPPC order or Davidson iteration
    theta: np.ndarray
    resid: np.ndarray
    spmv: int
    m: int              # basis size after the step


def _leading_block(row_ptr, col, val, n1: int):
    """H0_hat = H[:n1, :n1] as a scipy CSR matrix (the oracle's own copy)."""
    import scipy.sparse as sp
    H = sp.csr_matrix((val, col, row_ptr), shape=(row_ptr.shape[0] - 1,) * 2)
    return H[:n1, :n1].tocsr()


def lead_block_correction(H11, z_lead: np.ndarray, r_lead: np.ndarray, theta: float, iters: int) -> np.ndarray:
    """`iters` MINRES steps (x0 = 0, no stopping test) on P (H11 - theta) P t =
    P r with P = I - z z^T, z = z_lead / ||z_lead||; returns P t."""
    nz = float(np.linalg.norm(z_lead))
    z = z_lead / nz if nz > 0.0 else np.zeros_like(z_lead)
    b = r_lead - z * (z @ r_lead)

    def op(x):
        y = H11 @ x - theta * x
        return y - z * (z @ y)

    t, _, _ = minres(op, b, tol=0.0, maxit=iters)
    return t - z * (z @ t)


def _ritz(Q, W, k, nev):
    Ht = Q.T @ W
    Ht = 0.5 * (Ht + Ht.T)
    th, Y = np.linalg.eigh(Ht)
    return th[:nev], Y[:, :nev]


def sppc_hybrid(row_ptr, col, val, n1: int, k: int, *, switch_order: int = 15, tol: float = 1e-6,
                max_blocks: int = 16, maxit: int = 500, precond: str = "jacobi", clamp: float = 1e-2,
                solver: str = "pinv", minres_tol: float = 1e-12, reorth: str = "cond",
                perturb: float = 0.0, perturb_seed: int = 0, lead_iters: int = 20, lead_rows: int | None = None,
                small_eig=None, on_step=None, out: dict | None = None):
    """Run SPPC (Algorithm 2) for up to `switch_order` orders (stopping early if
    every scaled residual is below tol), then the block continuation above.
    Returns (theta, resid, converged, records).

    perturb > 0 multiplies every entry of T by (1 + perturb * N(0, 1)) each step
    (seeded): a test hook that measures how far rounding-sized differences carry
    along the trajectory.  lead_rows (default n1): rows of the leading block that
    precond="lead" solves with MINRES (a level boundary; more levels than the
    small space make a stronger preconditioner).  small_eig: optional eigenpairs of
    H0_hat passed to the SPPC phase (see sppc).  on_step: optional timing hook,
    callable(phase, index), called after each SPPC order ("sppc", p) and each
    continuation step ("davidson", it); it does not change the result.  out:
    optional dict that receives the final Ritz vectors as out["Z"] (n x k)."""
    n = row_ptr.shape[0] - 1
    r = sppc(row_ptr, col, val, n1, k, p_max=switch_order, tol=tol, solver=solver, minres_tol=minres_tol,
             keep=True, small_eig=small_eig,
             on_order=None if on_step is None else (lambda p: on_step("sppc", p)))
    records = [HybridRecord("sppc", o.p, o.theta, o.resid, o.spmv, k * (o.p + 1)) for o in r.orders]
    spmv = r.spmv
    if r.converged:
        if out is not None:
            out["Z"] = r.Z
        return r.theta, r.resid, True, records
    Q, W = r.Q, r.W
    rng = np.random.Generator(np.random.PCG64(perturb_seed))
    nl = n1 if lead_rows is None else int(lead_rows)
    H11 = _leading_block(row_ptr, col, val, nl) if precond == "lead" else None
    diag = np.zeros(n)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    on = rows == col
    diag[rows[on]] = val[on]
    for it in range(1, maxit + 1):
        nev = min(2 * k, Q.shape[1])
        th_all, Y_all = _ritz(Q, W, k, nev)
        th, Y = th_all[:k], Y_all[:, :k]
        Z = Q @ Y
        R = W @ Y - Z * th
        # step 2: preconditioned residuals
        if precond == "jacobi":
            den = diag[:, None] - th[None, :]
            small = np.abs(den) < clamp
            den[small] = np.where(den[small] >= 0, clamp, -clamp)
            T = R / den
        elif precond == "lead":
            den = diag[:, None] - th[None, :]
            small = np.abs(den) < clamp
            den[small] = np.where(den[small] >= 0, clamp, -clamp)
            T = R / den
            for j in range(k):
                T[:nl, j] = lead_block_correction(H11, Z[:nl, j], R[:nl, j], th[j], lead_iters)
        else:
            T = R.copy()
        if perturb > 0.0:
            T = T * (1.0 + perturb * rng.standard_normal(T.shape))
        # step 3: thick restart
        if Q.shape[1] + k > max_blocks * k:
            Q = Q @ Y_all[:, :2 * k]
            W = W @ Y_all[:, :2 * k]
        # step 4: block Gram-Schmidt (second pass by the criterion) + QR, extend
        # the basis by k SpMVs
        Phi = T - Q @ (Q.T @ T)
        if reorth == "twice" or np.any(np.linalg.norm(Phi, axis=0) < 0.5 * np.linalg.norm(T, axis=0)):
            Phi = Phi - Q @ (Q.T @ Phi)
        q, _ = np.linalg.qr(Phi)
        Wq = csr_spmm(row_ptr, col, val, q)
        spmv += k
        Q = np.hstack([Q, q])
        W = np.hstack([W, Wq])
        th, Y = _ritz(Q, W, k, k)
        Z = Q @ Y
        res = np.linalg.norm(W @ Y - Z * th, axis=0) / np.abs(th)
        records.append(HybridRecord("davidson", it, th, res, spmv, Q.shape[1]))
        if on_step is not None:
            on_step("davidson", it)
        if np.all(res <= tol):
            if out is not None:
                out["Z"] = Z
            return th, res, True, records
    if out is not None:
        out["Z"] = Z
    return th, res, False, records
