"""The projected eigensolve (sppc_small_syev) against LAPACK on random and on
clustered spectra, with the Householder steps in double-float and in FP64.
GPU only.  Eigenvalues to 1e-12 of ||S|| (FP64: 1e-13); eigenvectors by their
residual ||S v - theta v|| and orthonormality (vectors of a degenerate
eigenvalue are only defined as a subspace)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _check(S, nev, f64=False):
    import paper_2407_08901_gb300 as lib
    th, V = lib.sppc_small_syev(torch.from_numpy(S).cuda(), nev, f64=f64)
    th, V = th.cpu().numpy(), V.cpu().numpy()
    ref = np.linalg.eigvalsh(S)[:nev]
    nrm = np.abs(np.linalg.eigvalsh(S)).max()
    tol_val, tol_res, tol_orth = (1e-13, 1e-12, 1e-12) if f64 else (1e-12, 1e-11, 1e-11)
    assert np.all(np.diff(th) >= -1e-13 * nrm)
    assert np.allclose(th, ref, rtol=0, atol=tol_val * nrm), np.max(np.abs(th - ref)) / nrm
    res = np.linalg.norm(S @ V - V * th, axis=0)
    assert np.all(res <= tol_res * nrm), res.max() / nrm
    assert np.allclose(V.T @ V, np.eye(nev), rtol=0, atol=tol_orth)


@pytest.mark.parametrize("f64", [False, True])
@pytest.mark.parametrize("m", [1, 2, 3, 8, 9, 17, 33, 64, 127, 144])
def test_random_symmetric(m, f64):
    rng = np.random.Generator(np.random.PCG64(m))
    A = rng.standard_normal((m, m))
    S = (A + A.T) / 2 + np.diag(np.linspace(-3, 3, m))
    _check(S, min(16, m), f64)
    if m >= 9:
        _check(S, 3, f64)  # fewer vectors than CTAs in the cluster


@pytest.mark.parametrize("f64", [False, True])
def test_scaled_and_reducible(f64):
    """Large and small scales (the FP64 Sturm counts rescale their minors, whose
    magnitudes reach 1e+-320 here) and a tridiagonal form that splits (zero
    off-diagonals)."""
    rng = np.random.Generator(np.random.PCG64(5))
    m = 40
    A = rng.standard_normal((m, m))
    S = (A + A.T) / 2
    for scale in (1e-8, 1e8):
        _check(S * scale, 8, f64)
    D = np.diag(np.concatenate([np.linspace(-2, 2, 20), np.linspace(-1.5, 2.5, 20)]))
    D[5, 6] = D[6, 5] = 0.3
    _check(D, 10, f64)


@pytest.mark.parametrize("f64", [False, True])
@pytest.mark.parametrize("gaps", [(1e-6, 1e-9), (1e-12, 0.0), (1e-8, 1e-8)])
def test_clustered_spectrum(gaps, f64):
    """Eigenvalue pairs and a triple closer than FP32 can resolve, and an exactly
    degenerate pair, inside the 16 lowest: the crowded path (FP64 brackets,
    FP64 inverse-iteration steps, Gram-Schmidt in the group)."""
    m = 96
    rng = np.random.Generator(np.random.PCG64(11))
    lam = np.sort(rng.uniform(-5, 5, m))
    lam[3] = lam[2] + gaps[0]
    lam[8] = lam[7] + gaps[1]
    lam[12] = lam[11] + 2e-8
    lam[13] = lam[12] + 3e-8
    lam = np.sort(lam)
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    S = (Q * lam) @ Q.T
    S = (S + S.T) / 2
    _check(S, 16, f64)


def test_bad_sizes_are_rejected():
    import paper_2407_08901_gb300 as lib
    with pytest.raises(lib.SppcError):
        lib.sppc_small_syev(torch.zeros(145, 145, dtype=torch.float64, device="cuda"), 8)
    with pytest.raises(lib.SppcError):
        lib.sppc_small_syev(torch.zeros(10, 10, dtype=torch.float64, device="cuda"), 17)
