"""Parity with the FP64 oracle on the bench's own workload (c2: n = 2,000,000 in
7 levels, n1 = 9,660, 4.0e8 entries, k = 8), through the C ABI.  GPU only.

The smaller parity tests (test_gpu_parity.py) stay below the sizes at which the
library switches paths; these two cover what only c2 reaches:

* the 9,660-row small space (MINRES on about 151 CTAs, the deflation by 16
  small-space eigenvectors), the 1.31M-column tiles of the SpMM and 2M-row
  dense reductions: three SPPC orders (Algorithm 2) against the oracle's three
  orders in its MINRES mode, Ritz values to 1e-10 relative at every order;
* the 77,670-row leading block (levels 0-2, above the 65,536-row switch from the
  CSR to the SELL product) of the continuation's preconditioner (Sec. 5): the
  block the GPU appends after three orders against the oracle's
  lead_block_correction (20 MINRES steps) and shifted-diagonal rows, computed
  from the GPU's own Ritz pairs.

The oracle's small-space start is ARPACK (k + 8 lowest pairs of H0_hat), which
is all its MINRES mode needs.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import oracle
from conftest import make_matrix
from oracle.hybrid import lead_block_correction
from oracle.spmm import csr_spmm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ORDERS = 3
LEAD_LEVELS = 3
LEAD_ITERS = 20


def _small_start(rp, c, v, n1, k):
    rows = np.repeat(np.arange(n1), np.diff(rp[: n1 + 1]))
    cc = c[: rp[n1]]
    m = cc < n1
    H11 = sp.csr_matrix((v[: rp[n1]][m], (rows[m], cc[m])), shape=(n1, n1))
    ev, U = sla.eigsh(H11, k=k + 8, which="SA", tol=1e-14)
    o = np.argsort(ev)
    return ev[o], U[:, o]


_ORACLE = {}


def _oracle_orders(rp, c, v, n1, k):
    """The oracle's three orders on c2 (computed once per test session)."""
    if "c2" not in _ORACLE:
        _ORACLE["c2"] = oracle.sppc(rp, c, v, n1, k, fixed_orders=ORDERS, solver="minres",
                                    small_eig=_small_start(rp, c, v, n1, k))
    return _ORACLE["c2"]


def _leading(rp, c, v, nl):
    H = sp.csr_matrix((v, c, rp), shape=(rp.shape[0] - 1,) * 2)
    return H[:nl, :nl].tocsr()


@pytest.mark.parametrize("prec", [0, -1])
def test_c2_orders_match_oracle(prec):
    """Double-float (precision 0) and native FP64 (precision -1) paths."""
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix("c2")
    k, n1 = w.k, w.small_dim
    h = S.sppc_create(rp, c, v, w.level_offsets, n1, k, S.sppc_default_opts(p_max=ORDERS, precision=prec))
    try:
        conv, th, rs, st = S.sppc_solve(h, k, tol=1e-300, p_max=ORDERS)
        assert st["orders"] == ORDERS and st["spmv_h"] == k * (ORDERS + 1)
        ref = _oracle_orders(rp, c, v, n1, k)
        E0 = S.sppc_get_state(h, 5, (k,))
        assert np.allclose(E0, ref.E0, rtol=1e-12, atol=0), (E0 - ref.E0) / ref.E0
        for o in ref.orders:
            info = S.sppc_order_info(h, o.p, k)
            rel = np.abs(info["theta"] - o.theta) / np.abs(o.theta)
            assert np.all(rel <= 1e-10), (o.p, rel)
            assert np.allclose(info["resid"], o.resid, rtol=1e-6, atol=1e-12), (o.p, info["resid"], o.resid)
            if o.p >= 2:
                big = np.abs(o.E) > 1e-6 * np.abs(o.E).max()
                assert np.allclose(info["E"][big], o.E[big], rtol=1e-10, atol=0), (o.p, info["E"], o.E)
                assert np.all(np.abs(info["E"] - o.E) <= 1e-10 * np.abs(o.E).max())
    finally:
        S.sppc_destroy(h)


def test_c2_leading_block_correction_matches_oracle():
    """After three SPPC orders the first continuation step appends
    T = r_j / (diag(H) - theta_j) (clamped) on rows >= 77,670 and the deflated
    leading-block MINRES solution on rows < 77,670.  The oracle forms the same
    block from the GPU's Ritz pairs (Z = Q Y from the returned basis and
    projected matrix); columns are compared up to the Ritz vector's sign."""
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix("c2")
    k, n1, n = w.k, w.small_dim, w.n
    nl = int(w.level_offsets[LEAD_LEVELS])
    opts = S.sppc_default_opts(p_max=15, hybrid=1, switch_order=ORDERS, precond=2, precond_iters=LEAD_ITERS,
                               precond_levels=LEAD_LEVELS)
    h = S.sppc_create(rp, c, v, w.level_offsets, n1, k, opts)
    try:
        S.sppc_start(h, k)
        for _ in range(ORDERS):
            S.sppc_correct(h)
            th, _ = S.sppc_rayleigh_ritz(h, k)
        m = k * (ORDERS + 1)
        Q = S.sppc_get_state(h, 1, (n, m))
        Ht = S.sppc_get_state(h, 3, (m, m))
        S.sppc_refine_step(h, k)
        T = S.sppc_get_state(h, 8, (n, k))
    finally:
        S.sppc_destroy(h)
    ev, Y = np.linalg.eigh(0.5 * (Ht + Ht.T))
    assert np.allclose(ev[:k], th, rtol=1e-12, atol=0)
    Z = Q @ Y[:, :k]
    R = csr_spmm(rp, c, v, Z) - Z * th
    diag = np.zeros(n)
    rows = np.repeat(np.arange(n), np.diff(rp))
    on = rows == c
    diag[rows[on]] = v[on]
    den = diag[:, None] - th[None, :]
    small = np.abs(den) < 1e-2
    den[small] = np.where(den[small] >= 0, 1e-2, -1e-2)
    Tref = R / den
    HL = _leading(rp, c, v, nl)
    for j in range(k):
        Tref[:nl, j] = lead_block_correction(HL, Z[:nl, j], R[:nl, j], th[j], LEAD_ITERS)
    for j in range(k):
        sgn = 1.0 if np.dot(T[:, j], Tref[:, j]) >= 0 else -1.0
        d = np.abs(sgn * T[:, j] - Tref[:, j])
        scale_lead = np.abs(Tref[:nl, j]).max()
        scale_rest = np.abs(Tref[nl:, j]).max()
        assert d[:nl].max() <= 1e-9 * scale_lead, (j, d[:nl].max() / scale_lead)
        assert d[nl:].max() <= 1e-9 * scale_rest, (j, d[nl:].max() / scale_rest)
