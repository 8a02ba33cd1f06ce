"""SPPC for the k lowest eigenpairs (Algorithm 2), plain FP64, step by step.

Notation follows the paper: H = H0 + V with H0 = diag(H0_hat, 0) and
V = [[0, V12], [V21, V22]] (Eqs. split, split2); H0_hat is the leading n1 x n1
block (here called H11).  Psi^(p) is the n x k block of p-th order corrections,
E^(p) the k correction energies, Q the orthonormal basis of the combined
subspace M^(p) (Eq. comb_sub), W = H Q, Ht the projected matrix Q^T H Q.

Readings where the paper is silent (each also listed in the design notes):
* eigenvectors of H0_hat: ascending eigenvalues, each vector's largest-|entry|
  component made positive;
* the singular direction of Eq. (sm_lin_proj) is psi_hat_k; an eigenvector of
  H0_hat whose eigenvalue lies within `degeneracy_tol * ||H0_hat||` of E_k^(0)
  is deflated as well;
* the small solve is done either exactly on the complement of the deflated
  directions (spectral pseudo-inverse from the dense eigendecomposition) or by
  MINRES on the projected operator P (H0_hat - E_k) P, x0 = 0;
* block Gram-Schmidt (Eq. blkGS) applies the projector I - Q Q^T twice (the
  projector is idempotent; the second application only removes rounding);
* QR of Eq. (QR) is Householder QR (numpy.linalg.qr);
* the projected matrix is symmetrised, Ritz values sorted ascending;
* convergence: every relative residual ||H z - theta z|| / |theta| (Eq. rrn)
  below tol, checked after each order (Alg. 2), or a fixed number of orders.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .minres import minres
from .spmm import csr_spmm


@dataclass
class OrderRecord:
    p: int
    theta: np.ndarray          # k lowest Ritz values after order p
    resid: np.ndarray          # relative residual norms (Eq. rrn)
    E: np.ndarray              # E^(p) (E^(0) for p = 0)
    angle: np.ndarray | None   # ||Phi_j|| / ||Psi_j^(p)||: sine of the angle to M^(p-1)
    minres_iters: list | None
    spmv: int                  # cumulative count of H times one vector


@dataclass
class SPPCResult:
    orders: list
    E0: np.ndarray
    psi_hat: np.ndarray
    converged: bool
    Z: np.ndarray | None = None
    Q: np.ndarray | None = None
    W: np.ndarray | None = None
    Ht: np.ndarray | None = None
    Psi: list = field(default_factory=list)
    E: list = field(default_factory=list)
    VPsi: list = field(default_factory=list)
    HPsi_direct: list = field(default_factory=list)
    HPsi_recycled: list = field(default_factory=list)

    @property
    def theta(self) -> np.ndarray:
        return self.orders[-1].theta

    @property
    def resid(self) -> np.ndarray:
        return self.orders[-1].resid

    @property
    def spmv(self) -> int:
        return self.orders[-1].spmv


def small_eigenpairs(H11: np.ndarray):
    """All eigenpairs of H0_hat (dense), ascending, sign-normalised.

    Algorithm 2 step 1 and Eq. (EP_small): the eigenvectors of H0 are those of
    H0_hat padded with zeros.
    """
    w, U = np.linalg.eigh(H11)
    idx = np.argmax(np.abs(U), axis=0)
    sgn = np.sign(U[idx, np.arange(U.shape[1])])
    sgn[sgn == 0] = 1.0
    return w, U * sgn


def _ritz(Ht: np.ndarray, Q: np.ndarray, W: np.ndarray, k: int):
    """k lowest Ritz pairs of the projected matrix and their residuals (Eq. rrn)."""
    Hs = 0.5 * (Ht + Ht.T)
    th, Y = np.linalg.eigh(Hs)
    th, Y = th[:k], Y[:, :k]
    Z = Q @ Y
    HZ = W @ Y
    res = np.linalg.norm(HZ - Z * th, axis=0) / np.abs(th)
    return th, Y, Z, res


def sppc(row_ptr, col, val, n1: int, k: int, *, p_max: int = 15, tol: float = 1e-6,
         fixed_orders: int | None = None, solver: str = "pinv", minres_tol: float = 1e-12,
         minres_maxit: int | None = None, vpsi: str = "recycled", degeneracy_tol: float = 1e-10,
         keep: bool = False, small_eig=None, on_order=None) -> SPPCResult:
    """Run Algorithm 2 on the CSR matrix (row_ptr, col, val).

    solver: "pinv" (exact spectral solve) or "minres" for Eq. (sm_lin_proj).
    vpsi:   "recycled" (Eq. HPsip), "direct" (a fresh product H Psi^(p-1)) or
            "both" (both computed, recycled one used, both kept when keep=True).
    fixed_orders: run exactly this many correction orders (no early stop).
    small_eig: optional (eigenvalues, eigenvectors) of H0_hat, ascending; "pinv"
            needs all of them, "minres" only those the deflation rule can touch.
    on_order: optional callable(p), called after the Rayleigh-Ritz step of each
            order p (0 included); a timing hook, it does not change the result.
    """
    n = row_ptr.shape[0] - 1
    P = fixed_orders if fixed_orders is not None else p_max

    def spmm(X):
        return csr_spmm(row_ptr, col, val, X)

    # leading block H0_hat = H11 (sparse for products; dense only for its eigendecomposition)
    rows = np.repeat(np.arange(n1), np.diff(row_ptr[: n1 + 1]))
    c1 = col[: row_ptr[n1]]
    m1 = c1 < n1
    H11 = sp.csr_matrix((val[: row_ptr[n1]][m1], (rows[m1], c1[m1])), shape=(n1, n1))
    w_all, U_all = small_eig if small_eig is not None else small_eigenpairs(H11.toarray())
    normH11 = float(max(abs(w_all[0]), abs(w_all[-1])))
    E0 = w_all[:k].copy()
    psi_hat = U_all[:, :k].copy()
    if np.any(np.abs(E0) <= 1e-8 * normH11):
        raise ValueError("E^(0) too close to zero: x2 = -b2/E^(0) is undefined (Eq. sm_first)")

    def deflation_set(j):
        return np.nonzero(np.abs(w_all - E0[j]) <= degeneracy_tol * normH11)[0]

    # order 0 (Alg. 2 steps 1-4)
    Psi0 = np.zeros((n, k))
    Psi0[:n1] = psi_hat
    m_max = k * (P + 1)
    Qbuf = np.zeros((n, m_max))
    Wbuf = np.zeros((n, m_max))
    Qbuf[:, :k] = Psi0
    Wbuf[:, :k] = spmm(Psi0)
    spmv = k
    m = k
    Ht = Qbuf[:, :k].T @ Wbuf[:, :k]
    th, Y, Z, res = _ritz(Ht, Qbuf[:, :m], Wbuf[:, :m], k)
    orders = [OrderRecord(0, th, res, E0.copy(), None, None, spmv)]
    result = SPPCResult(orders, E0, psi_hat, False)
    if on_order is not None:
        on_order(0)
    if fixed_orders is None and np.all(res < tol):
        result.converged = True
        result.E = [E0.copy()]
        _finish(result, keep, Z, Qbuf[:, :m], Wbuf[:, :m], Ht)
        return result

    # V Psi^(0) = H Psi^(0) - H0 Psi^(0) (Eq. avoid_SpMV2); H Psi^(0) = W_0
    H0Psi0 = np.zeros((n, k))
    H0Psi0[:n1] = H11 @ psi_hat
    VPsi0 = Wbuf[:, :k] - H0Psi0
    Psis = [Psi0]
    Es = [E0.copy()]
    HPsi_prev = Wbuf[:, :k].copy()      # Psi^(0) = q^(0), R^(0) = I
    if keep:
        result.VPsi.append(VPsi0.copy())

    for p in range(1, P + 1):
        Psi_prev = Psis[p - 1]
        # H Psi^(p-1): recycled (Eq. HPsip) and/or a direct product
        if vpsi in ("direct", "both"):
            HPsi_d = spmm(Psi_prev)
            if keep:
                result.HPsi_direct.append(HPsi_d)
        if vpsi == "direct":
            HPsi = HPsi_d
        else:
            HPsi = HPsi_prev
            if keep:
                result.HPsi_recycled.append(HPsi_prev.copy())
        # V Psi^(p-1) = H Psi^(p-1) - H0 Psi^(p-1) (Eq. avoid_SpMV2)
        H0Psi = np.zeros((n, k))
        H0Psi[:n1] = H11 @ Psi_prev[:n1]
        VPsi = HPsi - H0Psi
        if keep and p > 1:
            result.VPsi.append(VPsi.copy())
        # E^(p) = (Psi^(p-1))^T V Psi^(0), per eigenpair (Eq. exp_seq)
        Ep = np.einsum("ij,ij->j", Psi_prev, VPsi0)
        Es.append(Ep)
        # right-hand side of Eq. (exp_seq2): -V Psi^(p-1) + sum_{l=0}^{p-2} E^(p-l) Psi^(l)
        b = -VPsi
        for l in range(0, p - 1):
            b = b + Es[p - l][None, :] * Psis[l]
        # Eq. (sm_first): x2 = -b2 / E^(0)
        x2 = -b[n1:] / E0[None, :]
        # Eq. (sm_lin_proj): deflate psi_hat_k, solve (H0_hat - E_k^(0)) x1 = b1'
        x1 = np.zeros((n1, k))
        its = []
        for j in range(k):
            D = deflation_set(j)
            Ud = U_all[:, D]
            b1 = b[:n1, j] - Ud @ (Ud.T @ b[:n1, j])
            if solver == "pinv":
                coef = U_all.T @ b1
                denom = w_all - E0[j]
                inv = np.zeros_like(denom)
                keepmask = np.ones(w_all.shape[0], dtype=bool)
                keepmask[D] = False
                inv[keepmask] = 1.0 / denom[keepmask]
                x1[:, j] = U_all @ (coef * inv)
                its.append(0)
            elif solver == "minres":
                def apply_a(v, Ud=Ud, e=E0[j]):
                    y = H11 @ v - e * v
                    return y - Ud @ (Ud.T @ y)
                xs, it, _ = minres(apply_a, b1, tol=minres_tol, maxit=minres_maxit or 20 * n1)
                x1[:, j] = xs - Ud @ (Ud.T @ xs)
                its.append(it)
            else:
                raise ValueError(solver)
        Psi_p = np.vstack([x1, x2])
        Psis.append(Psi_p)
        # Eq. (blkGS): Phi = (I - Q Q^T) Psi^(p), projector applied twice
        Q = Qbuf[:, :m]
        C = Q.T @ Psi_p
        Phi = Psi_p - Q @ C
        C2 = Q.T @ Phi
        Phi = Phi - Q @ C2
        C = C + C2
        angle = np.linalg.norm(Phi, axis=0) / np.linalg.norm(Psi_p, axis=0)
        # Eq. (QR): Phi = q R
        q, R = np.linalg.qr(Phi)
        # k SpMVs: H q^(p) (Sec. 4.2)
        Wp = spmm(q)
        spmv += k
        # Eq. (proj): border the projected matrix
        Bq = Q.T @ Wp
        Cq = q.T @ Wp
        Ht = np.block([[Ht, Bq], [Bq.T, Cq]])
        # Eq. (HPsip): H Psi^(p) = H Q^(p-1) (Q^(p-1)^T Psi^(p)) + H q^(p) R^(p)
        HPsi_prev = Wbuf[:, :m] @ C + Wp @ R
        # Eq. (Qp)
        Qbuf[:, m:m + k] = q
        Wbuf[:, m:m + k] = Wp
        m += k
        th, Y, Z, res = _ritz(Ht, Qbuf[:, :m], Wbuf[:, :m], k)
        orders.append(OrderRecord(p, th, res, Ep.copy(), angle, its, spmv))
        if on_order is not None:
            on_order(p)
        if fixed_orders is None and np.all(res < tol):
            result.converged = True
            break
    result.E = Es
    if keep:
        result.Psi = Psis
    _finish(result, keep, Z, Qbuf[:, :m], Wbuf[:, :m], Ht)
    return result


def _finish(result, keep, Z, Q, W, Ht):
    result.Z = Z
    result.Ht = Ht
    if keep:
        result.Q = Q.copy()
        result.W = W.copy()
