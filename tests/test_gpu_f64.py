"""The native FP64 path (opts.precision = -1) through the C ABI.  GPU only.

Its value slots hold IEEE doubles and its kernels accumulate with DFMA, so a
product with one stored entry per row rounds once, exactly as numpy's FP64
multiply does: a diagonal H gives Y = diag(H) * X bit for bit (the
double-float path cannot, its values carry about 48 bits).  The basis is
orthonormal to FP64 rounding, and the whole method (SPPC + the preconditioned
continuation, the bench's options) lands on the dense eigenvalues and agrees
with the double-float path.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from conftest import dense, make_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SMALL8 = W.Workload("small8", [300, 500, 900, 1300], 40, 8, seed=7)


@pytest.mark.parametrize("ncols", [1, 4, 5, 8])
def test_diagonal_product_is_exact_fp64(ncols):
    import paper_2407_08901_gb300 as S
    n = 70_001  # several slices of 16 rows and a ragged last one
    rng = np.random.Generator(np.random.PCG64(3))
    v = rng.standard_normal(n) * np.exp(rng.uniform(-20, 20, n))
    rp = np.arange(n + 1, dtype=np.int64)
    c = np.arange(n, dtype=np.int32)
    h = S.sppc_create(rp, c, v, np.array([0, 1000, n], dtype=np.int64), 1000, 2,
                      S.sppc_default_opts(p_max=1, precision=-1))
    try:
        X = rng.standard_normal((n, ncols)) * np.exp(rng.uniform(-20, 20, (n, ncols)))
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.empty_like(Xd)
        S.sppc_spmm(h, Xd, Yd)
        torch.cuda.synchronize()
        assert np.array_equal(Yd.cpu().numpy(), v[:, None] * X)
    finally:
        S.sppc_destroy(h)


def test_basis_is_orthonormal_to_fp64_rounding():
    """The appended blocks (CGS2 + CholeskyQR2 in FP64) are orthonormal to FP64
    rounding.  Block 0 holds the small eigensolve's eigenvectors psi_hat, whose
    mutual orthogonality is that of inverse iteration on the projected matrix
    (about eps ||H0_hat|| / gap, 1e-13 here), so it is held to 1e-12."""
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix("c1")
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts(p_max=6, precision=-1))
    try:
        S.sppc_solve(h, w.k, tol=1e-300, p_max=6)
        m = w.k * 7
        Q = S.sppc_get_state(h, 1, (w.n, m))
    finally:
        S.sppc_destroy(h)
    G = Q.T @ Q - np.eye(m)
    k = w.k
    assert np.abs(G[:k, :k]).max() <= 1e-12
    assert np.abs(G[k:, :]).max() <= 1e-14, np.abs(G[k:, :]).max()


def test_method_converges_to_dense_eigenvalues_and_matches_double_float():
    """The timed method's options on a k = 8 problem: 4 SPPC orders, then the
    continuation with the two-level leading-block preconditioner, to 1e-10."""
    import paper_2407_08901_gb300 as S
    rp, c, v = W.generate(SMALL8)
    lam = np.linalg.eigvalsh(dense(rp, c, v))[: SMALL8.k]
    out = {}
    for prec in (-1, 0):
        o = S.sppc_default_opts(p_max=6, hybrid=1, switch_order=4, precond=2, precond_iters=20, precond_levels=2,
                                tol=1e-10, precision=prec)
        h = S.sppc_create(rp, c, v, SMALL8.level_offsets, SMALL8.small_dim, SMALL8.k, o)
        try:
            conv, th, rs, st = S.sppc_solve(h, SMALL8.k, tol=1e-10)
            assert conv, (prec, rs)
            out[prec] = np.asarray(th)
        finally:
            S.sppc_destroy(h)
    assert np.allclose(out[-1], lam, rtol=1e-12, atol=0), (out[-1] - lam) / np.abs(lam)
    assert np.allclose(out[-1], out[0], rtol=1e-12, atol=0)


def test_noalloc_and_host_products_follow_the_format():
    """sppc_spmm, sppc_spmm_host and sppc_spmm_noalloc on an FP64 handle give the
    same bytes (one product, one format)."""
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix("c1")
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts(p_max=1, precision=-1))
    try:
        X = np.ascontiguousarray(W.random_block(w.n, 8, 4))
        Xd = torch.from_numpy(X).cuda()
        Y1 = torch.empty_like(Xd)
        Y2 = torch.full_like(Xd, float("nan"))
        S.sppc_spmm(h, Xd, Y1)
        S.sppc_spmm_noalloc(h, Xd, Y2)
        Yh = np.zeros_like(X)
        S.sppc_spmm_host(h, X, Yh)
        torch.cuda.synchronize()
        assert torch.equal(Y1, Y2)
        assert np.array_equal(Y1.cpu().numpy(), Yh)
        ref = oracle.csr_spmm(rp, c, v, X)
        mag = oracle.csr_spmm(rp, c, np.abs(v), np.abs(X))
        assert np.all(np.abs(Yh - ref) <= 1e-13 * mag)
    finally:
        S.sppc_destroy(h)


def test_incompatible_options_are_rejected():
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix("small")
    for kw in (dict(hybrid=2), dict(hybrid=1, proposal=1)):
        with pytest.raises(S.SppcError) as err:
            S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts(precision=-1, **kw))
        assert err.value.status == 1
