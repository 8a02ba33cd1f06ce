"""Eigenvalue truth for the oracle tests.

dense_lowest:   the k lowest eigenpairs of the whole matrix from a dense
                symmetric eigendecomposition (numpy.linalg.eigh), for small n.
block_lanczos:  block Lanczos (Golub and Underwood, 1977) with full
                reorthogonalisation, for matrices too large for dense eigh.
                The hybrid partners of Sec. 5 include it; here it is the truth
                that SPPC's Ritz values approach.
"""
from __future__ import annotations

import numpy as np

from .spmm import csr_spmm


def to_dense(row_ptr, col, val, n: int | None = None) -> np.ndarray:
    n = row_ptr.shape[0] - 1 if n is None else n
    A = np.zeros((row_ptr.shape[0] - 1, n))
    for i in range(row_ptr.shape[0] - 1):
        lo, hi = row_ptr[i], row_ptr[i + 1]
        np.add.at(A[i], col[lo:hi], val[lo:hi])
    return A


def dense_lowest(row_ptr, col, val, k: int):
    A = to_dense(row_ptr, col, val)
    w, U = np.linalg.eigh(A)
    return w[:k], U[:, :k]


def block_lanczos(row_ptr, col, val, k: int, X0: np.ndarray, tol: float = 1e-10, max_blocks: int = 200,
                  check_every: int = 2):
    """k lowest eigenpairs by block Lanczos from the start block X0 (n x b, b >= k).

    Every block is orthogonalised against all previous ones twice (full
    reorthogonalisation).  Ritz pairs come from the projected matrix
    Q^T H Q; the run stops when every relative residual ||Hz - theta z|| /
    |theta| of the k lowest is <= tol.  Returns (theta, Z, resid, spmv).
    """
    n, b = X0.shape
    Qb, _ = np.linalg.qr(X0)
    Qs = [Qb]
    HQs = []
    spmv = 0
    theta = Z = res = None
    for j in range(max_blocks):
        Wj = csr_spmm(row_ptr, col, val, Qs[-1])
        spmv += b
        HQs.append(Wj)
        Q = np.hstack(Qs)
        HQ = np.hstack(HQs)
        if (j + 1) % check_every == 0 or j == max_blocks - 1:
            T = Q.T @ HQ
            T = 0.5 * (T + T.T)
            w, Y = np.linalg.eigh(T)
            theta = w[:k]
            Z = Q @ Y[:, :k]
            res = np.linalg.norm(HQ @ Y[:, :k] - Z * theta, axis=0) / np.abs(theta)
            if np.all(res <= tol):
                break
        R = Wj.copy()
        for _ in range(2):
            R = R - Q @ (Q.T @ R)
        Qn, _ = np.linalg.qr(R)
        Qs.append(Qn)
    return theta, Z, res, spmv
