"""The tensor-core block Gram product (tcgen05, exact FP16 digit products of a
fixed-point split) against exact integer sums and the FP64 Gram, through the C
ABI (sppc_block_gram), and the solve with opts.tensor_gram.  GPU only.

Pins:
* inputs on a fixed-point grid whose digit products all fall in the kept levels
  (a = k 2^-30, b = k' 2^-10, |k|, |k'| < 2^20): the result equals the exact
  integer sum (numpy int64 matmul), bit for bit;
* orthonormal A (QR of a Gaussian matrix) and B with columns of very different
  scales, a zero column and a ragged row count: within one FP64 rounding of the
  fixed-point bound of the exactly rounded Gram, in both slot formats;
* more than 16 blocks (two launches), one row, no rows;
* |a| >= 2 or a NaN is reported as SPPC_ERR_NAN;
* a c2mini solve gives the same Ritz values with the tensor-core Gram as with
  the CUDA-core one, in FP64 and double-float.
"""
import numpy as np
import pytest

from conftest import make_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _S():
    import paper_2407_08901_gb300 as S
    return S


def _orthonormal(nb, n, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    X = torch.randn(n, 8 * nb, generator=g, dtype=torch.float64)
    if n >= 8 * nb:
        Q, _ = torch.linalg.qr(X)
    else:  # too few rows for orthonormal columns: unit columns
        Q = X / torch.linalg.norm(X, dim=0, keepdim=True)
    return Q.reshape(n, nb, 8).permute(1, 0, 2).contiguous()


def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _split(x):
    c = 134217729.0 * x  # 2^27 + 1 (Veltkamp)
    h = c - (c - x)
    return h, x - h


def _two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def _dd_gram(A, B):
    """A^T B in double-double (Dekker products, pairwise error-free sums): the
    exact Gram to about 2^-100 relative, rounded to FP64."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    out = np.zeros((A.shape[0] * 8, 8))
    for a in range(A.shape[0]):
        p, e = _two_prod(A[a][:, :, None], B[:, None, :])
        errs = [e.sum(axis=0)]
        while p.shape[0] > 1:
            if p.shape[0] % 2:
                p = np.concatenate([p, np.zeros((1,) + p.shape[1:])])
            p, e = _two_sum(p[0::2], p[1::2])
            errs.append(e.sum(axis=0))
        lo = np.zeros((8, 8))
        for e in errs:
            lo = lo + e
        out[a * 8:(a + 1) * 8] = (p[0] + lo) if p.shape[0] else lo
    return out


@pytest.mark.parametrize("n", [64, 1000, 4099, 40000])
def test_grid_inputs_are_exact(n):
    S = _S()
    rng = np.random.default_rng(n)
    nb = 5
    ka = rng.integers(-(1 << 20) + 1, 1 << 20, size=(nb, n, 8), dtype=np.int64)
    kb = rng.integers(-(1 << 20) + 1, 1 << 20, size=(n, 8), dtype=np.int64)
    kb[:, 3] = 0                                   # a zero column
    kb[: n // 2, 5] //= 4096                        # a column with mixed magnitudes
    exact = np.einsum("anr,nj->arj", ka, kb).reshape(nb * 8, 8)   # |sum| < n 2^40 < 2^56: int64 exact
    assert np.all(np.abs(exact) < (1 << 53))  # so that the FP64 result is exact too
    want = np.ldexp(exact.astype(np.float64), -40)
    A = torch.from_numpy(np.ldexp(ka.astype(np.float64), -30)).cuda()
    B = torch.from_numpy(np.ldexp(kb.astype(np.float64), -10)).cuda()
    G = S.sppc_block_gram(A, B, tensor=True).cpu().numpy()
    assert np.array_equal(G, want)
    G0 = S.sppc_block_gram(A, B, tensor=False).cpu().numpy()
    assert np.array_equal(G0, want)


def _tol(A, B):
    """Bound on |G_tc - G|: the fixed-point rounding and dropped digit levels
    (about 2^-60 max|b_j| per row) plus FP64 rounding of the sum."""
    n = A.shape[1]
    absg = np.einsum("anr,nj->arj", np.abs(A), np.abs(B)).reshape(-1, 8)
    bmax = np.max(np.abs(B), axis=0)
    return 4 * n * 2.0 ** -60 * bmax[None, :] + 8 * 2.0 ** -53 * absg


@pytest.mark.parametrize("df", [False, True])
@pytest.mark.parametrize("nb,n", [(1, 1), (3, 1000), (16, 4099), (20, 30011), (16, 100003)])
def test_orthonormal_basis_against_fp64(nb, n, df):
    S = _S()
    Q = _orthonormal(nb, n, seed=nb * 1000 + n)
    g = torch.Generator(device="cpu").manual_seed(n + 7)
    B = torch.randn(n, 8, generator=g, dtype=torch.float64)
    B = B * torch.tensor([1e-3, 1.0, 1e5, 0.0, 3.0, 1e-12, 7.0, 1e12], dtype=torch.float64)
    B[:, 6] = Q[0, :, 2] * 5.0 + 1e-9 * B[:, 6]   # nearly in the span: large cancellation in G
    Ah, Bh = Q.numpy(), B.numpy()
    ref = _dd_gram(Ah, Bh)
    G = S.sppc_block_gram(Q.cuda(), B.cuda(), tensor=True, df=df).cpu().numpy()
    tol = _tol(Ah, Bh)
    if df:
        tol = tol + 2.0 ** -46 * np.einsum("anr,nj->arj", np.abs(Ah), np.abs(Bh)).reshape(-1, 8)
    err = np.abs(G - ref)
    assert np.all(err <= tol), float(np.max(err / np.maximum(tol, 1e-300)))
    assert np.all(G[:, 3] == 0.0)


def test_empty_rows_give_zero():
    S = _S()
    A = torch.zeros(2, 0, 8, dtype=torch.float64, device="cuda")
    B = torch.zeros(0, 8, dtype=torch.float64, device="cuda")
    G = S.sppc_block_gram(A, B, tensor=True).cpu().numpy()
    assert G.shape == (16, 8) and np.all(G == 0.0)


@pytest.mark.parametrize("case", ["big", "nan_a", "inf_b"])
def test_out_of_range_is_reported(case):
    S = _S()
    Q = _orthonormal(2, 3000, seed=5).cuda()
    B = torch.randn(3000, 8, dtype=torch.float64, device="cuda")
    if case == "big":
        Q[1, 1234, 3] = 2.5
    elif case == "nan_a":
        Q[0, 17, 0] = float("nan")
    else:
        B[2999, 7] = float("inf")
    with pytest.raises(S.SppcError) as err:
        S.sppc_block_gram(Q, B, tensor=True)
    assert err.value.status == 11
    # the library stays usable
    G = S.sppc_block_gram(_orthonormal(1, 100, 3).cuda(), torch.ones(100, 8, dtype=torch.float64, device="cuda"),
                          tensor=True)
    assert torch.isfinite(G).all()


@pytest.mark.parametrize("prec", [-1, 0])
def test_solve_with_tensor_gram_matches(prec):
    S = _S()
    w, rp, c, v = make_matrix("c2mini")
    out = []
    for tg in (0, 1):
        opts = S.sppc_default_opts(p_max=10, hybrid=1, switch_order=5, precond=2, precond_levels=3, tol=1e-9,
                                   precision=prec, tensor_gram=tg)
        h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, opts)
        try:
            conv, th, rs, st = S.sppc_solve(h, w.k, tol=1e-9)
            out.append((np.asarray(th), np.asarray(rs), conv))
        finally:
            S.sppc_destroy(h)
    (t0, r0, c0), (t1, r1, c1) = out
    assert c0 and c1
    assert np.max(np.abs(t1 - t0) / np.abs(t0)) < 1e-11
