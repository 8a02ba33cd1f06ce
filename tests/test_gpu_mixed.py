"""Mixed precision (opts.precision = 1; 2 with BF16 off-diagonal values): H rounded to FP32, the solve's products
with H in FP32, everything else double-float, Ritz values and residuals
recomputed with double-float products at the end.  GPU only.

References (the matrix is the FP32-rounded H): dense eigh of the rounded matrix,
or the FP64 path of this library on the rounded matrix; the solver's target is
1e-8 relative in eigenvalues and the tolerance in (double-float) residuals.  The
shift against the unrounded H is the quantisation error, reported separately."""
import numpy as np
import pytest

import workloads as W
from conftest import dense, make_matrix
from oracle.spmm import csr_spmm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SMALL8 = W.Workload("small8", [300, 500, 900, 1300], 40, 8, seed=7)


def _rounded(v):
    return v.astype(np.float32).astype(np.float64)


def _bf16(f32):
    """FP32 -> nearest BF16 (ties to even), as FP32 (bit arithmetic on the words)."""
    u = np.ascontiguousarray(f32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _rounded_bf16(rp, c, v):
    """Off-diagonal values to FP32 then BF16, the diagonal to FP32."""
    rows = np.repeat(np.arange(rp.shape[0] - 1), np.diff(rp))
    f = v.astype(np.float32)
    return np.where(rows == c, f, _bf16(f)).astype(np.float64)


def test_bf16_rounding_pins():
    """Round to nearest, ties to even, at BF16's 8-bit significand."""
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -3.140625, 0.1], dtype=np.float32)
    got = _bf16(x)
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, 1.0, -3.140625, 0.10009765625], dtype=np.float32)
    assert np.array_equal(got, want), got


@pytest.mark.parametrize("name,chunk,ncols", [("c1", 0, 8), ("c2mini", 0, 8), ("c2mini", 9000, 8),
                                               ("c1", 0, 4), ("c2mini", 9000, 4)])
def test_fp32_spmm_within_its_error_bound(name, chunk, ncols):
    """FP32 accumulation of a row of m products: error <= (m + 4) 2^-24 sum |a||x|
    (m roundings of the running sum, X rounded to FP32, tile partial sums);
    8-column (32-byte gathers) and 4-column (16-byte gathers) kernels."""
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix(name)
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, ncols,
                      S.sppc_default_opts(precision=1, spmm_chunk_cols=chunk))
    try:
        X = W.random_block(w.n, ncols, 21)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.full_like(Xd, float("nan"))
        S.sppc_spmm(h, Xd, Yd)
        Y = Yd.cpu().numpy()
    finally:
        S.sppc_destroy(h)
    vr = _rounded(v)
    ref = csr_spmm(rp, c, vr, X)
    mag = csr_spmm(rp, c, np.abs(vr), np.abs(X))
    m = np.diff(rp).astype(np.float64)[:, None]
    assert np.all(np.abs(Y - ref) <= (m + 4) * 2.0 ** -24 * mag + 1e-300)


@pytest.mark.parametrize("name,chunk", [("c1", 0), ("c2mini", 9000)])
def test_bf16_spmm_within_its_error_bound(name, chunk):
    """BF16 values are exact in FP32, so the bound is the FP32 one on the
    BF16-rounded matrix (diagonal FP32, applied once per row)."""
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix(name)
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, 8 if w.k < 7 else w.k,
                      S.sppc_default_opts(precision=2, spmm_chunk_cols=chunk))
    try:
        X = W.random_block(w.n, 8, 22)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.full_like(Xd, float("nan"))
        S.sppc_spmm(h, Xd, Yd)
        Y = Yd.cpu().numpy()
    finally:
        S.sppc_destroy(h)
    vr = _rounded_bf16(rp, c, v)
    ref = csr_spmm(rp, c, vr, X)
    mag = csr_spmm(rp, c, np.abs(vr), np.abs(X))
    m = np.diff(rp).astype(np.float64)[:, None]
    assert np.all(np.abs(Y - ref) <= (m + 4) * 2.0 ** -24 * mag + 1e-300)


def test_bf16_solve_matches_dense_eigenvalues_of_the_rounded_matrix():
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix(SMALL8)
    vr = _rounded_bf16(rp, c, v)
    lam = np.linalg.eigvalsh(dense(rp, c, vr))[: w.k]
    opts = S.sppc_default_opts(p_max=6, hybrid=1, switch_order=3, precond=2, precision=2, tol=1e-8)
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, opts)
    try:
        conv, th, rs, st = S.sppc_solve(h, w.k, tol=1e-8)
    finally:
        S.sppc_destroy(h)
    assert conv and np.all(rs <= 1e-8), rs
    assert np.allclose(th, lam, rtol=1e-8, atol=0), (th - lam) / np.abs(lam)
    # quantisation error against the unrounded matrix: reported, ~1e-4 relative
    lam0 = np.linalg.eigvalsh(dense(rp, c, v))[: w.k]
    assert np.max(np.abs(lam - lam0) / np.abs(lam0)) < 1e-2


@pytest.mark.parametrize("k", [8, 4])
def test_mixed_solve_matches_dense_eigenvalues_of_the_rounded_matrix(k):
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix(W.Workload(f"small{k}", [300, 500, 900, 1300], 40, k, seed=7))
    vr = _rounded(v)
    lam = np.linalg.eigvalsh(dense(rp, c, vr))[: w.k]
    opts = S.sppc_default_opts(p_max=6, hybrid=1, switch_order=3, precond=2, precision=1, tol=1e-8)
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, opts)
    try:
        conv, th, rs, st = S.sppc_solve(h, w.k, tol=1e-8)
    finally:
        S.sppc_destroy(h)
    assert conv and np.all(rs <= 1e-8), rs
    assert np.allclose(th, lam, rtol=1e-8, atol=0), (th - lam) / np.abs(lam)


def test_mixed_solve_matches_the_fp64_path_on_the_rounded_matrix():
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix("c2mini")
    vr = _rounded(v)
    kw = dict(p_max=15, hybrid=1, switch_order=15, precond=2, precond_iters=10, tol=1e-6)
    out = {}
    vb = _rounded_bf16(rp, c, v)
    for prec, vals in ((1, v), (0, vr), (0, v), (2, v), (0, vb)):
        h = S.sppc_create(rp, c, vals, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts(precision=prec, **kw))
        try:
            conv, th, rs, st = S.sppc_solve(h, w.k, tol=1e-6)
        finally:
            S.sppc_destroy(h)
        assert conv and np.all(rs <= 1e-6), (prec, rs)
        out[(prec, "raw" if vals is v else ("f32" if vals is vr else "bf16"))] = np.asarray(th)
    mixed, fp64_rounded, fp64 = out[(1, "raw")], out[(0, "f32")], out[(0, "raw")]
    bf, fp64_bf = out[(2, "raw")], out[(0, "bf16")]
    assert np.allclose(bf, fp64_bf, rtol=1e-8, atol=0), (bf - fp64_bf) / np.abs(fp64_bf)
    assert np.allclose(mixed, fp64_rounded, rtol=1e-8, atol=0), (mixed - fp64_rounded) / np.abs(fp64_rounded)
    # quantisation of the values to FP32 moves the eigenvalues by ~1e-7 relative
    assert np.max(np.abs(fp64_rounded - fp64) / np.abs(fp64)) < 1e-5
