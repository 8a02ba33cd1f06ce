"""The allocation-free SpMM entry point (sppc_spmm_noalloc), through the C ABI.

It serves callers that cannot allocate device memory while they multiply, for
example a framework that owns all device memory through its own allocator and
budget.  Its scratch sits in a fixed 32 MiB device array shared by every call,
so these tests check two calls in a row against the allocating sppc_spmm and
against the oracle, on the column-tiled path too (the second call must not see
stale data from the first), for every value format, and that an oversized
request is refused before anything runs.  The file sorts last so that a run
stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

import workloads as W
from oracle.spmm import csr_spmm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_spmm_matches_spmm_on_two_calls_in_a_row():
    import paper_2407_08901_gb300 as S
    w = W.config("c1")
    rp, c, v = W.generate(w)
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k)
    try:
        for call, ncols in enumerate((8, 5)):
            X = torch.from_numpy(W.random_block(w.n, ncols, 100 + call)).cuda()
            Yref = torch.empty_like(X)
            Y = torch.full_like(X, float("nan"))
            S.sppc_spmm(h, X, Yref)
            S.sppc_spmm_noalloc(h, X, Y)
            torch.cuda.synchronize()
            y, yref = Y.cpu().numpy(), Yref.cpu().numpy()
            # the tolerance the SpMM tests use: 1e-12 of sum_j |H_ij x_j| per entry
            mag = csr_spmm(rp, c, np.abs(v), np.abs(X.cpu().numpy()))
            assert np.all(np.abs(y - yref) <= 1e-12 * mag), call
    finally:
        S.sppc_destroy(h)


@pytest.mark.parametrize("prec", [0, -1])
def test_noalloc_tiled_products_match_oracle_on_two_calls(prec):
    """Column tiles (1,000 columns, 20 tiles on c1): a row's first tile writes
    its sum into the shared array and later tiles add to it, so nothing there
    may depend on what the previous call left.  Two calls in a row with
    different widths, each against the oracle's CSR product at the SpMM tests'
    bound (1e-12 of sum_j |H_ij x_j|; FP64 handles as well)."""
    import paper_2407_08901_gb300 as S
    w = W.config("c1")
    rp, c, v = W.generate(w)
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k,
                      S.sppc_default_opts(p_max=1, spmm_chunk_cols=1000, precision=prec))
    try:
        assert S.sppc_get_layout(h)["n_chunks"] == 20
        for call, ncols in enumerate((8, 3)):
            X = W.random_block(w.n, ncols, 200 + call)
            Xd = torch.from_numpy(X).cuda()
            Y = torch.full_like(Xd, float("nan"))
            S.sppc_spmm_noalloc(h, Xd, Y)
            torch.cuda.synchronize()
            ref = csr_spmm(rp, c, v, X)
            mag = csr_spmm(rp, c, np.abs(v), np.abs(X))
            assert np.all(np.abs(Y.cpu().numpy() - ref) <= 1e-12 * mag), (prec, call)
    finally:
        S.sppc_destroy(h)


def test_noalloc_follows_fp32_products_of_mixed_precision_handles():
    """On a handle with FP32 values (precision 1) the allocation-free product is
    the FP32 product sppc_spmm runs (its FP32 copy of X also lives in the fixed
    array): identical bytes on two calls in a row."""
    import paper_2407_08901_gb300 as S
    w = W.config("small")
    rp, c, v = W.generate(w)
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts(p_max=1, precision=1))
    try:
        for call in range(2):
            X = torch.from_numpy(W.random_block(w.n, 4, 300 + call)).cuda()
            Yref = torch.empty_like(X)
            Y = torch.full_like(X, float("nan"))
            S.sppc_spmm(h, X, Yref)
            S.sppc_spmm_noalloc(h, X, Y)
            torch.cuda.synchronize()
            assert torch.equal(Y, Yref), call
    finally:
        S.sppc_destroy(h)


def test_noalloc_spmm_rejects_requests_beyond_its_scratch():
    import paper_2407_08901_gb300 as S
    n = 300_000  # 2 * n * 8 * 8 bytes = 38.4 MB > 32 MiB
    rp = np.arange(n + 1, dtype=np.int64)
    c = np.arange(n, dtype=np.int32)
    v = np.linspace(1.0, 2.0, n)
    h = S.sppc_create(rp, c, v, np.array([0, 1000, n], dtype=np.int64), 1000, 2, S.sppc_default_opts(p_max=1))
    try:
        X = torch.ones((n, 8), dtype=torch.float64, device="cuda")
        Y = torch.zeros_like(X)
        with pytest.raises(S.SppcError) as ei:
            S.sppc_spmm_noalloc(h, X, Y)
        assert ei.value.status == 1 and "scratch" in str(ei.value)
        # two columns fit (2 * n * 2 * 8 bytes = 9.6 MB): H is diagonal, so Y = diag(H)
        X2 = X[:, :2].contiguous()
        Y2 = torch.zeros_like(X2)
        S.sppc_spmm_noalloc(h, X2, Y2)
        torch.cuda.synchronize()
        ref = np.stack([v, v], axis=1)
        assert np.all(np.abs(Y2.cpu().numpy() - ref) <= 1e-12 * np.abs(ref))
    finally:
        S.sppc_destroy(h)
