"""Pins for the SPPC + block continuation oracle (CPU only)."""
import numpy as np

import oracle
import workloads as W
from conftest import dense, make_matrix
from test_oracle_sppc import TINY, _krylov_ritz


def test_identity_preconditioner_continues_the_block_krylov_space():
    """n1 = k makes SPPC's basis the block Krylov space of [I_k; 0]; extending it
    by the Ritz residuals (no preconditioner) adds exactly the next Krylov block,
    so the Ritz values stay those of block Lanczos."""
    w, rp, c, v = make_matrix(TINY)
    A = dense(rp, c, v)
    k = 3
    th, rs, conv, rec = oracle.sppc_hybrid(rp, c, v, k, k, switch_order=2, tol=1e-300, max_blocks=50, maxit=4,
                                           precond="none")
    S = np.zeros((w.n, k))
    S[:k, :k] = np.eye(k)
    kr = _krylov_ritz(A, S, 2 + 4, k)
    dav = [r for r in rec if r.phase == "davidson"]
    assert len(dav) == 4
    for r in dav:
        assert np.allclose(r.theta, kr[2 + r.step], rtol=1e-10, atol=0), r.step


def test_hybrid_converges_to_dense_eigenvalues_within_kato_temple(small_matrix):
    w, rp, c, v = small_matrix
    lam = np.linalg.eigvalsh(dense(rp, c, v))[: w.k + 1]
    th, rs, conv, rec = oracle.sppc_hybrid(rp, c, v, w.small_dim, w.k, switch_order=4, tol=1e-8, max_blocks=8)
    assert conv and np.all(rs <= 1e-8)
    gap = np.abs(np.diff(lam)).min()
    bound = (rs * np.abs(th)) ** 2 / gap
    assert np.all(np.abs(th - lam[: w.k]) <= 10 * bound + 1e-12)
    assert np.all(th >= lam[: w.k] - 1e-12)
    # the records are monotone: SPPC orders, then Davidson steps, SpMV count grows by k
    sp = [r.spmv for r in rec]
    assert all(b - a == w.k for a, b in zip(sp, sp[1:]))


def test_thick_restart_keeps_converging():
    w, rp, c, v = make_matrix(TINY)
    lam = np.linalg.eigvalsh(dense(rp, c, v))[: w.k]
    th, rs, conv, rec = oracle.sppc_hybrid(rp, c, v, w.small_dim, w.k, switch_order=2, tol=1e-9, max_blocks=4)
    assert conv and max(r.m for r in rec) <= 4 * w.k
    assert np.allclose(th, lam, rtol=1e-12)


def test_single_projection_is_enough_when_the_norm_survives():
    """The second projection changes only rounding when the first one kept at
    least half of each column's norm: with reorth="cond" and reorth="twice" the
    eigenvalues of every step agree to rounding, and the basis stays orthonormal
    to working accuracy either way."""
    w, rp, c, v = make_matrix(TINY)
    kw = dict(switch_order=2, tol=1e-300, max_blocks=50, maxit=6)
    a = oracle.sppc_hybrid(rp, c, v, w.small_dim, w.k, reorth="twice", **kw)[3]
    b = oracle.sppc_hybrid(rp, c, v, w.small_dim, w.k, reorth="cond", **kw)[3]
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert np.allclose(x.theta, y.theta, rtol=1e-12, atol=0), x.step


def test_perturbation_hook_is_rounding_sized_early():
    """perturb multiplies T by 1 + perturb*N(0,1): with 1e-15 the first steps of a
    run differ from the unperturbed one at rounding level only, and perturb=0 is
    the unperturbed run bit for bit."""
    w, rp, c, v = make_matrix(TINY)
    kw = dict(switch_order=1, tol=1e-300, max_blocks=6, maxit=8, precond="none")
    a = oracle.sppc_hybrid(rp, c, v, w.small_dim, w.k, **kw)[3]
    b = oracle.sppc_hybrid(rp, c, v, w.small_dim, w.k, perturb=1e-15, **kw)[3]
    z = oracle.sppc_hybrid(rp, c, v, w.small_dim, w.k, perturb=0.0, perturb_seed=5, **kw)[3]
    assert all(np.array_equal(x.theta, y.theta) for x, y in zip(a, z))
    diff = max(np.max(np.abs(x.theta - y.theta) / np.abs(x.theta)) for x, y in zip(a, b))
    assert 0 < diff < 1e-12


def test_lead_block_correction_solves_the_deflated_system():
    """With as many MINRES steps as unknowns the leading-block correction is the
    minimum-norm solution of P (H11 - theta) P t = P r (P = I - z z^T), which a
    dense least-squares solve gives independently; it is always orthogonal to z,
    and zero steps give zero."""
    from oracle.hybrid import lead_block_correction, _leading_block
    w, rp, c, v = make_matrix(TINY)
    n1 = w.small_dim
    H11 = _leading_block(rp, c, v, n1)
    A = H11.toarray()
    rng = np.random.Generator(np.random.PCG64(3))
    z = rng.standard_normal(n1)
    r = rng.standard_normal(n1)
    theta = float(np.linalg.eigvalsh(A)[1]) + 0.37
    t = lead_block_correction(H11, z, r, theta, 3 * n1)
    zh = z / np.linalg.norm(z)
    P = np.eye(n1) - np.outer(zh, zh)
    M = P @ (A - theta * np.eye(n1)) @ P
    ref = np.linalg.lstsq(M, P @ r, rcond=None)[0]
    assert abs(zh @ t) <= 1e-12 * np.linalg.norm(t)
    assert np.allclose(t, ref, rtol=0, atol=1e-9 * np.linalg.norm(ref))
    assert np.array_equal(lead_block_correction(H11, z, r, theta, 0), np.zeros(n1))


def test_lead_preconditioner_converges_to_dense_eigenvalues(small_matrix):
    w, rp, c, v = small_matrix
    lam = np.linalg.eigvalsh(dense(rp, c, v))[: w.k + 1]
    th, rs, conv, rec = oracle.sppc_hybrid(rp, c, v, w.small_dim, w.k, switch_order=3, tol=1e-8, max_blocks=8,
                                           precond="lead", lead_iters=20)
    assert conv and np.all(rs <= 1e-8)
    gap = np.abs(np.diff(lam)).min()
    assert np.all(np.abs(th - lam[: w.k]) <= 10 * (rs * np.abs(th)) ** 2 / gap + 1e-12)


def test_lead_block_over_more_levels_converges_to_the_same_eigenvalues():
    """precond="lead" with a leading block of two levels (lead_rows) reaches the
    same eigenpairs as with the small space alone, in no more steps here."""
    w, rp, c, v = make_matrix("c1")
    kw = dict(switch_order=2, tol=1e-9, max_blocks=7, precond="lead", maxit=300, lead_iters=20)
    th1, rs1, cv1, rec1 = oracle.sppc_hybrid(rp, c, v, w.small_dim, w.k, **kw)
    th2, rs2, cv2, rec2 = oracle.sppc_hybrid(rp, c, v, w.small_dim, w.k, lead_rows=int(w.level_offsets[2]), **kw)
    assert cv1 and cv2
    assert np.allclose(th1, th2, rtol=1e-12, atol=0)
    assert len(rec2) <= len(rec1)


def test_continuation_residual_and_scale_covariance(small_matrix):
    """The continuation's reported residuals equal ||H z - theta z|| / |theta|
    formed with the dense matrix and the final Ritz vectors (Eq. rrn), and
    H -> 3H scales its Ritz values by 3 and leaves those residuals unchanged
    (no preconditioner: every step is homogeneous)."""
    w, rp, c, v = small_matrix
    kw = dict(switch_order=2, tol=1e-300, max_blocks=8, maxit=5, precond="none")
    out = {}
    th, rs, conv, rec = oracle.sppc_hybrid(rp, c, v, w.small_dim, w.k, out=out, **kw)
    A = dense(rp, c, v)
    Z = out["Z"]
    direct = np.linalg.norm(A @ Z - Z * th, axis=0) / np.abs(th)
    assert np.allclose(rs, direct, rtol=1e-8, atol=1e-13)
    assert np.allclose(Z.T @ Z, np.eye(w.k), atol=1e-12)
    th3, rs3, _, _ = oracle.sppc_hybrid(rp, c, 3.0 * v, w.small_dim, w.k, **kw)
    assert np.allclose(th3, 3.0 * th, rtol=1e-11, atol=0)
    assert np.allclose(rs3, rs, rtol=1e-6, atol=1e-14)
