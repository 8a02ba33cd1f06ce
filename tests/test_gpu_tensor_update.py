"""The tensor-core block update Y = alpha X + sum_a Q_a C_a (tcgen05, exact FP16
digit products of a fixed-point split) against exact sums and a double-double
reference, through the C ABI (sppc_block_update).  GPU only.

Pins:
* inputs on a fixed-point grid whose digit products all fall in the kept levels
  (q = k 2^-30, C = k' 2^-10, X = k'' 2^-20, alpha = 1.5): the result equals the
  exact value (numpy int64 sums), bit for bit, on the tensor and CUDA cores;
* orthonormal Q (QR of a Gaussian matrix), C with columns of very different
  scales and a zero column, ragged row counts, more than 16 blocks (two
  launches), Y written over X, X absent: within the fixed-point bound plus one
  FP64 rounding, in both slot formats;
* a non-finite coefficient is reported as SPPC_ERR_NAN;
* ties: Y = 2^12 + t 2^-41 rounds to nearest, ties to even, on both cores.
"""
import numpy as np
import pytest

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
    else:
        Q = X / torch.linalg.norm(X, dim=0, keepdim=True)
    return Q.reshape(n, nb, 8).permute(1, 0, 2).contiguous()


def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _split(x):
    c = 134217729.0 * x
    h = c - (c - x)
    return h, x - h


def _two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def _dd_update(A, C, alpha, X):
    """alpha X + sum_a A_a C_a in double-double, rounded to FP64."""
    n = A.shape[1]
    hi = np.zeros((n, 8))
    lo = np.zeros((n, 8))
    if X is not None:
        al = np.ones(8) if alpha is None else alpha
        hi, lo = _two_prod(X, al[None, :])
    for a in range(A.shape[0]):
        for i in range(8):
            p, e = _two_prod(A[a][:, i:i + 1], C[8 * a + i][None, :])
            hi, e2 = _two_sum(hi, p)
            lo = lo + e + e2
    return hi + lo


def _tol(A, C, alpha, X, df):
    absa = np.abs(A).transpose(1, 0, 2).reshape(A.shape[1], -1)
    absc = np.abs(C)
    mag = absa @ absc
    if X is not None:
        mag = mag + np.abs(X) * (np.ones(8) if alpha is None else np.abs(alpha))[None, :]
    cmax = np.max(absc, axis=0)
    g = np.where(cmax > 0, 2.0 ** np.ceil(np.log2(np.maximum(cmax, 1e-300)) + 1), 1.0)
    tol = 2.0 ** -61 * absc.sum(axis=0)[None, :] + 2.0 ** -61 * g[None, :] * absa.sum(axis=1)[:, None] + 8 * 2.0 ** -53 * mag
    if df:
        tol = tol + 2.0 ** -46 * mag
    return tol


@pytest.mark.parametrize("n", [64, 1000, 4099])
def test_grid_inputs_are_exact(n):
    S = _S()
    rng = np.random.default_rng(n + 11)
    nb = 5
    ka = rng.integers(-(1 << 20) + 1, 1 << 20, size=(nb, n, 8), dtype=np.int64)
    kc = rng.integers(-(1 << 20) + 1, 1 << 20, size=(8 * nb, 8), dtype=np.int64)
    kc[:, 3] = 0
    kx = rng.integers(-(1 << 20) + 1, 1 << 20, size=(n, 8), dtype=np.int64)
    # exact: sum_i ka kc 2^-40 + 1.5 kx 2^-20 = (sum_i ka kc + 1.5 * 2^20 kx) 2^-40
    exact = np.einsum("anr,arj->nj", ka, kc.reshape(nb, 8, 8)) + 3 * (kx << 19)
    assert np.all(np.abs(exact) < (1 << 53))
    want = np.ldexp(exact.astype(np.float64), -40)
    A = torch.from_numpy(np.ldexp(ka.astype(np.float64), -30)).cuda()
    C = torch.from_numpy(np.ldexp(kc.astype(np.float64), -10)).cuda()
    X = torch.from_numpy(np.ldexp(kx.astype(np.float64), -20)).cuda()
    alpha = torch.full((8,), 1.5, dtype=torch.float64, device="cuda")
    for tc in (True, False):
        Y = S.sppc_block_update(A, C, alpha, X, tensor=tc).cpu().numpy()
        assert np.array_equal(Y, want), tc


@pytest.mark.parametrize("df", [False, True])
@pytest.mark.parametrize("nb,n", [(1, 1), (3, 1000), (16, 4099), (20, 30011), (7, 100003)])
def test_orthonormal_basis_against_double_double(nb, n, df):
    S = _S()
    Q = _orthonormal(nb, n, seed=nb * 77 + n)
    g = torch.Generator(device="cpu").manual_seed(n + 5)
    C = torch.randn(8 * nb, 8, generator=g, dtype=torch.float64)
    C = C * torch.tensor([1e-3, 1.0, 1e5, 0.0, 3.0, 1e-12, 7.0, 1e12], dtype=torch.float64)
    X = torch.randn(n, 8, generator=g, dtype=torch.float64)
    alpha = torch.randn(8, generator=g, dtype=torch.float64)
    Ah, Ch, Xh, ah = Q.numpy(), C.numpy(), X.numpy(), alpha.numpy()
    ref = _dd_update(Ah, Ch, ah, Xh)
    Y = S.sppc_block_update(Q.cuda(), C.cuda(), alpha.cuda(), X.cuda(), tensor=True, df=df).cpu().numpy()
    tol = _tol(Ah, Ch, ah, Xh, df)
    err = np.abs(Y - ref)
    assert np.all(err <= tol), float(np.max(err / np.maximum(tol, 1e-300)))


@pytest.mark.parametrize("df", [False, True])
def test_in_place_and_without_x(df):
    S = _S()
    nb, n = 4, 5003
    Q = _orthonormal(nb, n, seed=9)
    g = torch.Generator(device="cpu").manual_seed(3)
    C = torch.randn(8 * nb, 8, generator=g, dtype=torch.float64)
    X = torch.randn(n, 8, generator=g, dtype=torch.float64)
    Ah, Ch, Xh = Q.numpy(), C.numpy(), X.numpy()
    # Y = X - Q C written over X (the Gram-Schmidt subtraction, alpha = 1)
    Xd = X.cuda()
    S.sppc_block_update(Q.cuda(), (-C).cuda(), None, Xd, Y=Xd, tensor=True, df=df)
    ref = _dd_update(Ah, -Ch, None, Xh)
    assert np.all(np.abs(Xd.cpu().numpy() - ref) <= _tol(Ah, -Ch, None, Xh, df))
    # Y = Q C (no X term)
    Y = S.sppc_block_update(Q.cuda(), C.cuda(), None, None, tensor=True, df=df).cpu().numpy()
    ref = _dd_update(Ah, Ch, None, None)
    assert np.all(np.abs(Y - ref) <= _tol(Ah, Ch, None, None, df))


@pytest.mark.parametrize("df", [False, True])
def test_tensor_and_cuda_cores_agree_at_scale(df):
    # 2e5 rows: every CTA runs several 128-row tiles through the pipeline
    S = _S()
    nb, n = 6, 200_003
    Q = _orthonormal(nb, n, seed=21).cuda()
    g = torch.Generator(device="cuda").manual_seed(4)
    C = torch.randn(8 * nb, 8, generator=g, dtype=torch.float64, device="cuda")
    X = torch.randn(n, 8, generator=g, dtype=torch.float64, device="cuda")
    for alpha in (None, torch.randn(8, generator=g, dtype=torch.float64, device="cuda")):
        Y1 = S.sppc_block_update(Q, C, alpha, X, tensor=True, df=df)
        Y0 = S.sppc_block_update(Q, C, alpha, X, tensor=False, df=df)
        # the CUDA-core update rounds once per multiply-add (8 nb of them, on top
        # of alpha X); the tensor path rounds the exact sum once
        a = torch.ones(8, dtype=torch.float64, device="cuda") if alpha is None else alpha.abs()
        mag = X.abs() * a + Q.abs().permute(1, 0, 2).reshape(n, -1) @ C.abs()
        u = 2.0 ** -46 if df else 2.0 ** -53
        assert bool(((Y1 - Y0).abs() <= (8 * nb + 4) * u * mag).all())


def test_non_finite_coefficient_is_reported():
    S = _S()
    Q = _orthonormal(2, 3000, seed=2).cuda()
    C = torch.ones(16, 8, dtype=torch.float64, device="cuda")
    C[5, 3] = float("nan")
    with pytest.raises(S.SppcError) as err:
        S.sppc_block_update(Q, C, tensor=True)
    assert err.value.status == 11


def test_rounding_ties_to_even():
    """The exact sum is rounded once, to nearest with ties to even: Y = 2^12 +
    t 2^-41 (half an ulp of 2^12 per unit of t) from q = 1 against c = 2^12 and
    q = t 2^-30 against c = 2^-11, on the tensor and the CUDA cores."""
    from fractions import Fraction
    S = _S()
    ts = [1, 2, 3, 5, -1, -3, 0, 7]
    n = len(ts)
    A = np.zeros((1, n, 8))
    A[0, :, 0] = 1.0
    A[0, :, 1] = np.ldexp(np.array(ts, dtype=np.float64), -30)
    C = np.zeros((8, 8))
    C[0, 0] = 2.0 ** 12
    C[1, 0] = 2.0 ** -11
    want = np.array([float(Fraction(2) ** 12 + t * Fraction(1, 2 ** 41)) for t in ts])  # Fraction -> nearest double
    for tc in (True, False):
        Y = S.sppc_block_update(torch.from_numpy(A).cuda(), torch.from_numpy(C).cuda(), tensor=tc).cpu().numpy()
        assert np.array_equal(Y[:, 0], want), (tc, Y[:, 0] - want)
        assert np.all(Y[:, 1:] == 0.0)
