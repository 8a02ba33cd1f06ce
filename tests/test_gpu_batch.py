"""Batched solves (many independent problems of uneven sizes, k = 4): the
concurrent runner against one-by-one solves (identical results) and against
dense eigenvalues."""
import numpy as np
import pytest

import workloads as W
from conftest import dense

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _problems():
    """Six matrices of the batched law (3-6 levels x2.2, ~80 entries per row,
    k = 4) at sizes a dense eigensolve still handles."""
    rng = np.random.Generator(np.random.PCG64(5))
    out = []
    for m in range(6):
        n = int(rng.integers(1500, 4000))
        L = int(rng.integers(3, 7))
        w = W.Workload(f"b{m}", W.level_sizes_geometric(n, L, 2.2), 80, 4, seed=100 + m)
        out.append((w,) + W.generate(w))
    return out


def _opts(S, precision=0):
    return S.sppc_default_opts(p_max=8, hybrid=1, switch_order=4, precond=2, precond_iters=10, tol=1e-8,
                               hybrid_maxit=500, precision=precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_one_by_one_and_dense(precision):
    import paper_2407_08901_gb300 as S
    probs = _problems()
    hs = [S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, _opts(S, precision)) for w, rp, c, v in probs]
    try:
        st, th, rs, cv, stats = S.sppc_solve_batch(hs, 4, tol=1e-8, workers=3)
    finally:
        for h in hs:
            S.sppc_destroy(h)
    assert st == S.SPPC_OK and cv.all()
    for i, (w, rp, c, v) in enumerate(probs):
        h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, _opts(S, precision))
        try:
            conv, th1, rs1, st1 = S.sppc_solve(h, w.k, tol=1e-8)
        finally:
            S.sppc_destroy(h)
        assert conv
        assert np.array_equal(th[i], th1) and np.array_equal(rs[i], rs1)
        assert stats[i]["spmv_h"] == st1["spmv_h"]
        vals = v if precision == 0 else v.astype(np.float32).astype(np.float64)
        lam = np.linalg.eigvalsh(dense(rp, c, vals))[: w.k]
        assert np.allclose(th[i], lam, rtol=1e-8, atol=0), (i, (th[i] - lam) / np.abs(lam))


def test_batch_rejects_small_kmax():
    import paper_2407_08901_gb300 as S
    w, rp, c, v = _problems()[0]
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, _opts(S))
    try:
        with pytest.raises(S.SppcError):
            S.sppc_solve_batch([h], 2, tol=1e-8, workers=1)
    finally:
        S.sppc_destroy(h)


@pytest.mark.parametrize("ncols", [8, 4, 3])
def test_batched_spmm_equals_per_handle_products(ncols):
    """One persistent launch over six matrices (work queue over their slices),
    replayed from a CUDA graph: bit-identical to per-handle products."""
    import paper_2407_08901_gb300 as S
    probs = _problems()
    hs = [S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts()) for w, rp, c, v in probs]
    plan = None
    try:
        Xs = [torch.from_numpy(W.random_block(w.n, ncols, 40 + i)).cuda() for i, (w, *_r) in enumerate(probs)]
        Ys = [torch.full_like(X, float("nan")) for X in Xs]
        plan = S.sppc_spmm_batch_plan(hs, Xs, Ys)
        for _ in range(2):                       # graph replays give the same products
            S.sppc_spmm_batch_run(plan)
            torch.cuda.synchronize()
            for h, X, Y in zip(hs, Xs, Ys):
                Yr = torch.empty_like(X)
                S.sppc_spmm(h, X, Yr)
                torch.cuda.synchronize()
                assert torch.equal(Y, Yr)
            for Y in Ys:
                Y.fill_(float("nan"))
    finally:
        S.sppc_spmm_batch_destroy(plan)
        for h in hs:
            S.sppc_destroy(h)
