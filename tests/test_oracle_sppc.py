"""Pins for the oracle (CPU only): closed forms, textbook special cases,
invariants and brute force.  None of these re-types an oracle formula; each
checks it against something the paper or the mathematics fixes."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads as W
from conftest import dense, make_matrix
from oracle.lanczos import block_lanczos
from oracle.minres import minres
from oracle.spmm import csr_spmm

TINY = W.Workload("tiny", [60, 100, 120, 120], 30, 3, seed=5)


def _split(A, n1):
    """H0 = diag(H0_hat, 0) and V = H - H0 (Eq. split2)."""
    H0 = np.zeros_like(A)
    H0[:n1, :n1] = A[:n1, :n1]
    return H0, A - H0


# ---------------------------------------------------------------- MINRES
@pytest.mark.parametrize("kind", ["spd", "indefinite"])
def test_minres_matches_dense_solve(kind):
    rng = np.random.Generator(np.random.PCG64(3))
    n = 80
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.linspace(0.5, 9.0, n) if kind == "spd" else np.concatenate([-np.linspace(0.3, 4, 7), np.linspace(0.2, 9, n - 7)])
    A = (Qm * ev) @ Qm.T
    b = rng.standard_normal(n)
    x, it, r = minres(lambda v: A @ v, b, tol=1e-13, maxit=10 * n)
    xt = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xt) <= 1e-11 * np.linalg.norm(xt)
    assert abs(r - np.linalg.norm(A @ x - b)) <= 1e-12 * np.linalg.norm(b)


def test_minres_zero_rhs_and_projected_singular_system():
    x, it, r = minres(lambda v: 2 * v, np.zeros(5))
    assert it == 0 and not x.any()
    rng = np.random.Generator(np.random.PCG64(4))
    n = 50
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.linspace(-3, 6, n)
    ev[10] = 0.0                      # exactly singular along u = Qm[:, 10]
    A = (Qm * ev) @ Qm.T
    u = Qm[:, 10]
    b = rng.standard_normal(n)
    b = b - u * (u @ b)
    x, it, r = minres(lambda v: (lambda y: y - u * (u @ y))(A @ v), b, tol=1e-13, maxit=10 * n)
    x = x - u * (u @ x)
    inv = np.zeros(n)
    inv[ev != 0] = 1.0 / ev[ev != 0]
    xt = Qm @ (inv * (Qm.T @ b))          # spectral pseudo-inverse
    assert np.linalg.norm(x - xt) <= 1e-10 * np.linalg.norm(xt)


# ----------------------------------------------------------- identities
@pytest.fixture(scope="module")
def small_run():
    w, rp, c, v = make_matrix("small")
    r = oracle.sppc(rp, c, v, w.small_dim, w.k, fixed_orders=6, vpsi="both", keep=True)
    return w, rp, c, v, r


def test_small_space_eigenpairs(small_run):
    w, rp, c, v, r = small_run
    A = dense(rp, c, v)
    H11 = A[: w.small_dim, : w.small_dim]
    res = H11 @ r.psi_hat - r.psi_hat * r.E0
    assert np.abs(res).max() <= 1e-12 * np.abs(r.E0).max()
    assert np.allclose(r.psi_hat.T @ r.psi_hat, np.eye(w.k), atol=1e-13)
    assert np.all(np.diff(r.E0) >= 0)


def test_first_order_closed_forms(small_run):
    """Eq. (first_PC): E^(1) = 0 and Psi^(1) = (H Psi^(0) - E^(0) Psi^(0)) / E^(0);
    then E^(2) = (V Psi^(0))^T (V Psi^(0)) / E^(0) follows from Eq. (exp_seq)."""
    w, rp, c, v, r = small_run
    A = dense(rp, c, v)
    Psi0 = r.Psi[0]
    assert np.abs(r.E[1]).max() <= 1e-13 * np.abs(r.E0).max()
    expect = (A @ Psi0 - Psi0 * r.E0) / r.E0
    assert np.abs(r.Psi[1] - expect).max() <= 1e-12 * np.abs(expect).max()
    H0, V = _split(A, w.small_dim)
    VP = V @ Psi0
    assert np.allclose(r.E[2], np.einsum("ij,ij->j", VP, VP) / r.E0, rtol=1e-12, atol=0)


def test_recycled_h_psi_equals_direct_product(small_run):
    """Eq. (HPsip): H Psi^(p-1) from stored H Q equals a fresh product."""
    w, rp, c, v, r = small_run
    assert len(r.HPsi_direct) == len(r.HPsi_recycled) == 6
    for d, rc in zip(r.HPsi_direct, r.HPsi_recycled):
        assert np.abs(d - rc).max() <= 1e-12 * np.abs(d).max()


def test_correction_energy_symmetric_form(small_run):
    """Eq. (exp_seq): E^(p) = (Psi^(p-1))^T V Psi^(0) = psi_hat^T (V Psi^(p-1))_1."""
    w, rp, c, v, r = small_run
    A = dense(rp, c, v)
    H0, V = _split(A, w.small_dim)
    for p in range(2, 7):
        alt = np.einsum("ij,ij->j", r.Psi[0], V @ r.Psi[p - 1])
        assert np.allclose(r.E[p], alt, rtol=1e-10, atol=1e-12 * np.abs(alt).max())


def test_intermediate_normalisation(small_run):
    """Deflating psi_hat_k (Eq. sm_lin_proj) keeps Psi_k^(p) orthogonal to Psi_k^(0)."""
    w, rp, c, v, r = small_run
    for p in range(1, 7):
        d = np.einsum("ij,ij->j", r.Psi[0], r.Psi[p])
        assert np.abs(d).max() <= 1e-12 * np.abs(r.Psi[p]).max()


def test_projected_matrix_and_basis(small_run):
    """Order 0: Q^T H Q = diag(E^(0)) since V11 = 0; the bordered matrix of
    Eq. (proj) equals Q^T H Q recomputed from scratch; Q is orthonormal."""
    w, rp, c, v, r = small_run
    A = dense(rp, c, v)
    Q = r.Q
    k = w.k
    full = Q.T @ A @ Q
    assert np.abs(full[:k, :k] - np.diag(r.E0)).max() <= 1e-12 * np.abs(r.E0).max()
    assert np.abs(r.Ht - full).max() <= 1e-11 * np.abs(full).max()
    assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() <= 1e-13


# ------------------------------------------------ perturbation series
def test_rayleigh_schroedinger_series():
    """For H(c) = H0 + cV (Eq. Hc) the partial sums of Eq. (exp) built from the
    oracle's E^(p) and Psi^(p) approach the exact eigenpairs of H(c) with error
    O(c^(P+1)); halving c divides the error by about 2^(P+1)."""
    w, rp, c, v = make_matrix(TINY)
    A = dense(rp, c, v)
    n1, k, P = w.small_dim, w.k, 4
    r = oracle.sppc(rp, c, v, n1, k, fixed_orders=P + 1, keep=True)
    H0, V = _split(A, n1)
    errs_e, errs_v = [], []
    for cc in (0.02, 0.01):
        lam, U = np.linalg.eigh(H0 + cc * V)
        S = sum(cc ** p * r.E[p] for p in range(P + 1))
        errs_e.append(np.abs(S - lam[:k]))
        # eigenvector with intermediate normalisation Psi^(0)^T Psi(c) = 1
        Uk = U[:, :k] / np.einsum("ij,ij->j", r.Psi[0], U[:, :k])
        Sv = sum(cc ** p * r.Psi[p] for p in range(P + 1))
        errs_v.append(np.linalg.norm(Sv - Uk, axis=0))
        bound = 2 * np.abs(r.E[P + 1]) * cc ** (P + 1) + 1e-13
        assert np.all(errs_e[-1] <= bound)
    ratio_e = errs_e[0] / errs_e[1]
    ratio_v = errs_v[0] / errs_v[1]
    assert np.all((ratio_e > 2 ** (P + 1) * 0.6) & (ratio_e < 2 ** (P + 1) * 1.6)), ratio_e
    assert np.all((ratio_v > 2 ** (P + 1) * 0.6) & (ratio_v < 2 ** (P + 1) * 1.6)), ratio_v


# ------------------------------------------------------- special cases
def _krylov_ritz(A, S, steps, k):
    """Lowest k Ritz values of the block Krylov space K_(steps+1)(A, S): a
    Lanczos basis with full reorthogonalisation, written out for the test."""
    B, _ = np.linalg.qr(S)
    basis = [B]
    out = []
    for j in range(steps + 1):
        Qk = np.hstack(basis)
        out.append(np.linalg.eigvalsh(Qk.T @ A @ Qk)[:k])
        Wn = A @ basis[-1]
        for _ in range(2):
            Wn = Wn - Qk @ (Qk.T @ Wn)
        Bn, _ = np.linalg.qr(Wn)
        basis.append(Bn)
    return out


@pytest.mark.parametrize("n1,k", [(1, 1), (3, 3)])
def test_reduces_to_krylov_when_small_space_is_the_start_block(n1, k):
    """n1 = k: x1 lies in span(psi_hat) after deflation, x2 extends the block
    Krylov space, so M^(p) = K_(p+1)(H, [I_k; 0]) and the Ritz values equal
    those of (block) Lanczos from the first k unit vectors."""
    w, rp, c, v = make_matrix(TINY)
    A = dense(rp, c, v)
    P = 5
    r = oracle.sppc(rp, c, v, n1, k, fixed_orders=P)
    S = np.zeros((A.shape[0], k))
    S[:k, :k] = np.eye(k)
    kr = _krylov_ritz(A, S, P, k)
    for p in range(P + 1):
        assert np.allclose(r.orders[p].theta, kr[p], rtol=1e-10, atol=0), p


def test_exact_at_order_zero_without_coupling():
    """V12 = 0 and the lower block's spectrum above E^(0): Psi^(0) are exact
    eigenvectors, so order 0 already has zero residual."""
    w, rp, c, v = make_matrix(TINY)
    n1 = w.small_dim
    rows = np.repeat(np.arange(w.n), np.diff(rp))
    keep = ~(((rows < n1) & (c >= n1)) | ((rows >= n1) & (c < n1)))
    nrp = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=w.n))]).astype(np.int64)
    c2, v2 = c[keep], v[keep]
    A = dense(nrp, c2, v2)
    lam = np.linalg.eigvalsh(A)[: w.k]
    assert np.linalg.eigvalsh(A[n1:, n1:])[0] > lam[-1]
    r = oracle.sppc(nrp, c2, v2, n1, w.k, p_max=3, tol=1e-12)
    assert len(r.orders) == 1 and r.converged
    assert np.allclose(r.theta, lam, rtol=1e-13)


def test_exact_when_small_space_is_everything():
    w, rp, c, v = make_matrix(TINY)
    lam = np.linalg.eigvalsh(dense(rp, c, v))[: w.k]
    r = oracle.sppc(rp, c, v, w.n, w.k, p_max=2, tol=1e-12)
    assert len(r.orders) == 1 and np.allclose(r.theta, lam, rtol=1e-13)


# ---------------------------------------------------------- invariants
def test_ritz_values_are_decreasing_upper_bounds_and_obey_kato_temple(small_matrix):
    """Nested subspaces (Eq. Qp): Ritz values are upper bounds of the true
    eigenvalues (Courant-Fischer) that never increase with p; the lowest obeys
    the Kato-Temple bound theta1 - ||r1||^2/(lambda2 - theta1) <= lambda1."""
    w, rp, c, v = small_matrix
    A = dense(rp, c, v)
    lam = np.linalg.eigvalsh(A)[: w.k + 1]
    r = oracle.sppc(rp, c, v, w.small_dim, w.k, fixed_orders=15)
    prev = None
    for o in r.orders:
        assert np.all(o.theta >= lam[: w.k] - 1e-12)
        if prev is not None:
            assert np.all(o.theta <= prev + 1e-12)
        prev = o.theta
        r1 = o.resid[0] * abs(o.theta[0])
        if o.theta[0] < lam[1]:
            assert o.theta[0] - r1 ** 2 / (lam[1] - o.theta[0]) <= lam[0] + 1e-12
    assert r.orders[-1].theta[0] - lam[0] < 1e-3 * (r.orders[0].theta[0] - lam[0])


def test_brute_force_convergence_to_dense_eigenvalues():
    """On a tiny matrix 30 orders make M^(P) rich enough to hold the k lowest
    eigenvectors to ~1e-6 residual (the corrections then stagnate, angle
    ~1e-13); the Ritz values, quadratic in that error, meet dense eigh."""
    w, rp, c, v = make_matrix(TINY)
    lam = np.linalg.eigvalsh(dense(rp, c, v))[: w.k]
    r = oracle.sppc(rp, c, v, w.small_dim, w.k, fixed_orders=30)
    assert np.all(r.resid < 1e-5)
    assert np.allclose(r.theta, lam, rtol=1e-11)


def test_minres_mode_matches_exact_small_solves(small_matrix):
    w, rp, c, v = small_matrix
    a = oracle.sppc(rp, c, v, w.small_dim, w.k, fixed_orders=5, solver="pinv")
    b = oracle.sppc(rp, c, v, w.small_dim, w.k, fixed_orders=5, solver="minres", minres_tol=1e-13)
    for oa, ob in zip(a.orders, b.orders):
        assert np.allclose(oa.theta, ob.theta, rtol=1e-10, atol=0)
        assert np.allclose(oa.E, ob.E, rtol=1e-8, atol=1e-10)


# --------------------------------------------------------- truth / spmm
def test_block_lanczos_truth(small_matrix):
    w, rp, c, v = small_matrix
    lam = np.linalg.eigvalsh(dense(rp, c, v))[: w.k]
    X0 = W.random_block(w.n, 2 * w.k, 1)
    th, Z, res, spmv = block_lanczos(rp, c, v, w.k, X0, tol=1e-11, max_blocks=150)
    assert np.all(res <= 1e-11)
    assert np.allclose(th, lam, rtol=1e-11)


def test_c_spmm_matches_dense_product(c1_matrix):
    w, rp, c, v = c1_matrix
    X = W.random_block(w.n, 6, 2)
    Yc = csr_spmm(rp, c, v, X, use_c=True)
    Ys = csr_spmm(rp, c, v, X, use_c=False)
    assert np.abs(Yc - Ys).max() <= 1e-13 * np.abs(Ys).max()
    A = dense(rp[:201], c, v, w.n)
    assert np.abs(Yc[:200] - A[:200] @ X).max() <= 1e-13 * np.abs(Ys).max()


# ------------------------------------- closed-form correction energies
def _rs_closed_form(a, b, v, w, V22):
    """E^(2), E^(3), E^(4) of the lowest state for H0 = diag(a, b, 0, ..., 0)
    (H0_hat = diag(a, b), a < b, a != 0) and V with V11 = 0, rows v (state a)
    and w (state b) of V12, lower block V22: Rayleigh-Schroedinger theory
    worked out by hand, in exact rationals.

    With intermediate normalisation the lower block of H0 is zero, so its
    resolvent is 1/a; the second state enters through 1/(a - b):
      Psi1 = (0, 0, v/a)            E2 = s/a,             s = v.v
      Psi2 = (0, (w.v)/(a(a-b)), V22 v/a^2)   E3 = t/a^2, t = v.V22 v
      E4 = (w.v)^2/(a^2 (a-b)) + (u - s^2)/a^3,          u = v.V22^2 v
    """
    Fr = Fraction
    v = [Fr(x) for x in v]
    w = [Fr(x) for x in w]
    a, b = Fr(a), Fr(b)
    dot = lambda x, y: sum(p * q for p, q in zip(x, y))
    mv = lambda M, x: [sum(Fr(M[i][j]) * x[j] for j in range(len(x))) for i in range(len(M))]
    s = dot(v, v)
    V22v = mv(V22, v)
    t = dot(v, V22v)
    u = dot(V22v, V22v)
    wv = dot(w, v)
    return [s / a, t / a ** 2, wv ** 2 / (a ** 2 * (a - b)) + (u - s ** 2) / a ** 3]


@pytest.mark.parametrize("solver", ["pinv", "minres"])
@pytest.mark.parametrize("case", ["one_state", "two_states"])
def test_correction_energies_match_hand_derived_series(solver, case):
    """Eq. (exp)'s energies E^(1..4) on small integer matrices against the
    hand-derived Rayleigh-Schroedinger closed forms (Eqs. split2, sm_lin):
    E^(1) = 0 because V's leading block is zero; a wrong resolvent sign, a
    dropped E^(q) Psi^(p-q) term or a missing second state changes E^(3) or
    E^(4).  For n1 = 1, H = [[-3, 1, 2], [1, 1, 1], [2, 1, -1]] gives
    E = -3, 0, -5/3, 1/9, 5/9."""
    if case == "one_state":
        a, b = -3, None
        v, w = [1, 2], [0, 0]
        V22 = [[1, 1], [1, -1]]
    else:
        a, b = -3, 2
        v, w = [1, 2, 0, -1], [2, -1, 1, 1]
        V22 = [[1, 1, 0, 2], [1, -1, 1, 0], [0, 1, 2, -1], [2, 0, -1, 0]]
    n1 = 1 if b is None else 2
    m = len(v)
    A = np.zeros((n1 + m, n1 + m))
    A[0, 0] = a
    A[0, n1:] = A[n1:, 0] = v
    if b is not None:
        A[1, 1] = b
        A[1, n1:] = A[n1:, 1] = w
    A[n1:, n1:] = V22
    M = sp.csr_matrix(A)
    r = oracle.sppc(M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data, n1, 1,
                    fixed_orders=4, keep=True, solver=solver)
    want = _rs_closed_form(a, b if b is not None else 0, v, w, V22)
    if case == "one_state":
        assert want == [Fraction(-5, 3), Fraction(1, 9), Fraction(5, 9)]
    assert r.E[0][0] == a and r.E[1][0] == 0.0
    tol = 1e-13 if solver == "pinv" else 1e-10
    assert len(r.E) >= 5
    for p, e in enumerate(want, start=2):
        assert abs(r.E[p][0] - float(e)) <= tol * max(1.0, abs(float(e))), (p, r.E[p][0], e)


# ------------------------------------------- scale covariance, Eq. (rrn)
def test_scale_covariance_and_reported_residual(small_run):
    """H -> 3H scales every energy and Ritz value by 3 and leaves Psi^(p) and the
    scaled residuals (Eq. rrn) unchanged: every step of Algorithm 2 is
    homogeneous, so a dropped scale (an unscaled residual, an E^(0) squared, a
    constant shift) breaks it.  The reported residual equals
    ||H z - theta z|| / |theta| formed with the dense matrix and the returned
    Ritz vectors."""
    w, rp, c, v, r = small_run
    r3 = oracle.sppc(rp, c, 3.0 * v, w.small_dim, w.k, fixed_orders=6, vpsi="both", keep=True)
    for o, o3 in zip(r.orders, r3.orders):
        assert np.allclose(o3.theta, 3.0 * o.theta, rtol=1e-12, atol=0)
        assert np.allclose(o3.resid, o.resid, rtol=1e-8, atol=1e-14)
    scale = max(np.abs(e).max() for e in r.E)
    for e, e3 in zip(r.E, r3.E):
        assert np.abs(e3 - 3.0 * e).max() <= 1e-10 * 3.0 * scale
    for ps, ps3 in zip(r.Psi, r3.Psi):
        assert np.abs(ps3 - ps).max() <= 1e-9 * max(1.0, np.abs(ps).max())
    A = dense(rp, c, v)
    direct = np.linalg.norm(A @ r.Z - r.Z * r.theta, axis=0) / np.abs(r.theta)
    assert np.allclose(r.resid, direct, rtol=1e-8, atol=1e-13)
