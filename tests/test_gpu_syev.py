"""The projected eigensolve (sppc_small_syev) against LAPACK on random and on
clustered spectra.  GPU only.  Eigenvalues to 1e-12 of ||S||; eigenvectors by
their residual ||S v - theta v|| and orthonormality (vectors of a degenerate
eigenvalue are only defined as a subspace)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _check(S, nev, tol_res=1e-11):
    import paper_2407_08901_gb300 as lib
    th, V = lib.sppc_small_syev(torch.from_numpy(S).cuda(), nev)
    th, V = th.cpu().numpy(), V.cpu().numpy()
    ref = np.linalg.eigvalsh(S)[:nev]
    nrm = np.abs(np.linalg.eigvalsh(S)).max()
    assert np.all(np.diff(th) >= -1e-13 * nrm)
    assert np.allclose(th, ref, rtol=0, atol=1e-12 * nrm), np.max(np.abs(th - ref)) / nrm
    res = np.linalg.norm(S @ V - V * th, axis=0)
    assert np.all(res <= tol_res * nrm), res.max() / nrm
    assert np.allclose(V.T @ V, np.eye(nev), rtol=0, atol=1e-11)


@pytest.mark.parametrize("m", [1, 2, 3, 8, 33, 64, 127, 144])
def test_random_symmetric(m):
    rng = np.random.Generator(np.random.PCG64(m))
    A = rng.standard_normal((m, m))
    S = (A + A.T) / 2 + np.diag(np.linspace(-3, 3, m))
    _check(S, min(16, m))


@pytest.mark.parametrize("gaps", [(1e-6, 1e-9), (1e-12, 0.0), (1e-8, 1e-8)])
def test_clustered_spectrum(gaps):
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
    _check(S, 16)


def test_bad_sizes_are_rejected():
    import paper_2407_08901_gb300 as lib
    with pytest.raises(lib.SppcError):
        lib.sppc_small_syev(torch.zeros(145, 145, dtype=torch.float64, device="cuda"), 8)
    with pytest.raises(lib.SppcError):
        lib.sppc_small_syev(torch.zeros(10, 10, dtype=torch.float64, device="cuda"), 17)
