"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.  GPU only.

Both value formats are covered: double-float (two fp32, ~48-bit significand,
error-free transformations; opts.precision = 0) and native FP64 (DFMA;
opts.precision = -1).  An SpMM row sum of m terms carries an error below
~m * 2^-46 * sum_j |H_ij x_j| in double-float (accumulation bound of the
lazily renormalised accumulator) and ~m * 2^-53 * sum_j |H_ij x_j| in FP64, so
entries are compared against 1e-12 (double-float) or 1e-13 (FP64) times that
row magnitude.  Eigenvalues must match the oracle to 1e-10 relative at the same
order (the target of the FP64 path); scaled residuals (a difference of nearly
equal vectors) to 1e-6 relative plus 1e-12 absolute.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from conftest import make_matrix
from oracle.spmm import csr_spmm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lib():
    import paper_2407_08901_gb300 as S
    return S


def _abs_spmm(rp, c, v, X):
    return csr_spmm(rp, c, np.abs(v), np.abs(X))


def _create(name_or_w, opts=None, **kw):
    S = _lib()
    w, rp, c, v = make_matrix(name_or_w)
    o = opts or S.sppc_default_opts(**kw)
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, o)
    return S, w, rp, c, v, h


SPMM_TOL = {0: 1e-12, -1: 1e-13}


@pytest.mark.parametrize("prec", [0, -1])
@pytest.mark.parametrize("name", ["small", "c1"])
@pytest.mark.parametrize("ncols", [1, 2, 5, 8])
def test_spmm_matches_oracle(name, ncols, prec):
    S, w, rp, c, v, h = _create(name, precision=prec)
    try:
        X = W.random_block(w.n, ncols, 11 + ncols)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.empty_like(Xd)
        S.sppc_spmm(h, Xd, Yd)
        torch.cuda.synchronize()
        Y = Yd.cpu().numpy()
        ref = csr_spmm(rp, c, v, X)
        mag = _abs_spmm(rp, c, v, X)
        assert np.all(np.abs(Y - ref) <= SPMM_TOL[prec] * mag + 1e-300), np.max(np.abs(Y - ref) / mag)
        # host-buffer entry point gives the same bytes
        Yh = np.zeros_like(X)
        S.sppc_spmm_host(h, np.ascontiguousarray(X), Yh)
        assert np.array_equal(Yh, Y)
    finally:
        S.sppc_destroy(h)


@pytest.mark.parametrize("ncols,kernel", [(3, 0), (8, 0), (8, 1)])
def test_spmm_empty_and_ragged_rows(ncols, kernel):
    """A matrix with empty rows (no stored entry at all) and a level whose size is
    not a multiple of the 16-row slice; 8 columns run the TMA-gather kernel
    (kernel 0) or the register-gather one (kernel 1), including slices of width 0."""
    S = _lib()
    n = 203
    rng = np.random.Generator(np.random.PCG64(9))
    A = np.zeros((n, n))
    for i in range(n):
        if i % 7 == 3:
            continue
        js = rng.integers(0, n, 5)
        A[i, js] = rng.standard_normal(5)
    A = A + A.T
    for i in range(n):
        if i % 7 == 3:
            A[i, :] = 0
            A[:, i] = 0
    rows, cols = np.nonzero(A)
    rp = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]).astype(np.int64)
    c = cols.astype(np.int32)
    v = A[rows, cols]
    lev = np.array([0, 37, 101, n], dtype=np.int64)
    h = S.sppc_create(rp, c, v, lev, 37, 2, S.sppc_default_opts(spmm_kernel=kernel))
    try:
        X = W.random_block(n, ncols, 1)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.full_like(Xd, 7.0)
        S.sppc_spmm(h, Xd, Yd)
        Y = Yd.cpu().numpy()
        ref = A @ X
        assert np.allclose(Y, ref, rtol=0, atol=1e-12 * (np.abs(A) @ np.abs(X)).max() + 1e-300)
        assert np.all(Y[3::7] == 0.0)
    finally:
        S.sppc_destroy(h)


def _sell_reference(rp, c, ncols, seg, chunk_cols=0, sigma=1024, sh=16):
    """The SELL-16 layout: columns cut into chunks; per chunk and per level the
    rows with entries in the chunk (plus, in chunk 0, rows with no entry at all)
    are sorted by decreasing count inside windows of sigma rows (stable) and cut
    into slices of 16 rows."""
    nrows = seg[-1]
    C = chunk_cols if 0 < chunk_cols < ncols else ncols
    nch = -(-ncols // C)
    lens = np.zeros((nrows, nch), dtype=np.int64)
    for r in range(nrows):
        cc = c[rp[r]:rp[r + 1]]
        cc = cc[cc < ncols]
        lens[r] = np.bincount(cc // C, minlength=nch)[:nch]
    empty = lens.sum(axis=1) == 0
    slice_rows, slice_ptr, chunk_slice = [], [0], []
    for q in range(nch):
        chunk_slice.append(len(slice_rows))
        for a, b in zip(seg[:-1], seg[1:]):
            part = np.array([r for r in range(a, b) if lens[r, q] > 0 or (q == 0 and empty[r])], dtype=np.int64)
            for w0 in range(0, len(part), sigma):
                idx = part[w0:w0 + sigma]
                part[w0:w0 + sigma] = idx[np.argsort(-lens[idx, q], kind="stable")]
            for s0 in range(0, len(part), sh):
                rows = part[s0:s0 + sh]
                pad = np.full(sh, -1)
                pad[: len(rows)] = rows
                slice_rows.append(pad)
                slice_ptr.append(slice_ptr[-1] + sh * int(lens[rows, q].max()))
    chunk_slice.append(len(slice_rows))
    return (np.array(slice_ptr, dtype=np.int64), np.concatenate(slice_rows).astype(np.int32),
            np.array(chunk_slice, dtype=np.int64))


@pytest.mark.parametrize("name,chunk,sigma", [("small", -1, 0), ("small", 700, 0), ("c1", -1, 0), ("c1", 4096, 0),
                                              ("small", 700, 16), ("c1", -1, 64), ("c1", 4096, 256)])
def test_layout_is_bit_exact(name, chunk, sigma):
    S, w, rp, c, v, h = _create(name, spmm_chunk_cols=chunk, sell_sigma=sigma)
    try:
        L = S.sppc_get_layout(h)
        assert S.sppc_sell_sigma(h)[0] == (sigma or 1024)
    finally:
        S.sppc_destroy(h)
    sp, sr, cs = _sell_reference(rp, c, w.n, list(w.level_offsets), chunk, sigma=sigma or 1024)
    assert L["n_chunks"] == len(cs) - 1
    assert np.array_equal(L["chunk_slice"], cs)
    assert np.array_equal(L["slice_ptr"], sp) and np.array_equal(L["slice_rows"], sr)
    sp11, sr11, _ = _sell_reference(rp, c, w.small_dim, [0, w.small_dim])
    assert np.array_equal(L["h11_slice_ptr"], sp11) and np.array_equal(L["h11_slice_rows"], sr11)


def test_sigma_autotune_picks_a_candidate_and_stays_exact():
    """opts.sell_sigma = -2: the three windows are timed, one of them is kept,
    and the layout (and so the product) is the one of that window."""
    S, w, rp, c, v, h = _create("c1", sell_sigma=-2)
    try:
        sigma, ms = S.sppc_sell_sigma(h)
        assert sigma in (64, 256, 1024) and np.all(ms > 0)
        L = S.sppc_get_layout(h)
        X = W.random_block(w.n, 8, 4)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.empty_like(Xd)
        S.sppc_spmm(h, Xd, Yd)
        Y = Yd.cpu().numpy()
    finally:
        S.sppc_destroy(h)
    sp, sr, _ = _sell_reference(rp, c, w.n, list(w.level_offsets), 0, sigma=sigma)
    assert np.array_equal(L["slice_ptr"], sp) and np.array_equal(L["slice_rows"], sr)
    ref = csr_spmm(rp, c, v, X)
    assert np.all(np.abs(Y - ref) <= SPMM_TOL[0] * _abs_spmm(rp, c, v, X))


@pytest.mark.parametrize("prec", [0, -1])
@pytest.mark.parametrize("chunk", [257, 1000, 5000])
def test_chunked_spmm_matches_oracle(chunk, prec):
    """Column tiling: every chunk adds its partial row sums to Y; the row's first
    chunk writes, its last one finishes."""
    S, w, rp, c, v, h = _create("c1", spmm_chunk_cols=chunk, precision=prec)
    try:
        X = W.random_block(w.n, 8, 3)
        Xd = torch.from_numpy(X).cuda()
        Yd = torch.full_like(Xd, float("nan"))
        S.sppc_spmm(h, Xd, Yd)
        Y = Yd.cpu().numpy()
        ref = csr_spmm(rp, c, v, X)
        mag = _abs_spmm(rp, c, v, X)
        assert np.all(np.abs(Y - ref) <= SPMM_TOL[prec] * mag), np.max(np.abs(Y - ref) / mag)
    finally:
        S.sppc_destroy(h)


@pytest.mark.parametrize("name,chunk", [("small", -1), ("small", 700), ("c1", 4096), ("c2mini", 0),
                                        ("c2mini", 3000)])
def test_tma_and_register_gather_kernels_agree_bit_for_bit(name, chunk):
    """The TMA-gather SpMM (8 columns) accumulates every row in the same order and
    with the same renormalisation as the register-gather kernel: identical bits,
    and both within the accumulation bound of the oracle."""
    S = _lib()
    out = []
    for kernel in (0, 1):
        _, w, rp, c, v, h = _create(name, spmm_chunk_cols=chunk, spmm_kernel=kernel)
        try:
            X = W.random_block(w.n, 8, 5)
            Xd = torch.from_numpy(X).cuda()
            Yd = torch.full_like(Xd, float("nan"))
            S.sppc_spmm(h, Xd, Yd)
            out.append(Yd.cpu().numpy())
        finally:
            S.sppc_destroy(h)
    assert np.array_equal(out[0], out[1])
    ref = csr_spmm(rp, c, v, X)
    mag = _abs_spmm(rp, c, v, X)
    assert np.all(np.abs(out[0] - ref) <= 1e-12 * mag + 1e-300), np.max(np.abs(out[0] - ref) / mag)


def _compare_orders(S, h, ref, k, rtol_theta=1e-10):
    for o in ref.orders:
        info = S.sppc_order_info(h, o.p, k)
        assert np.allclose(info["theta"], o.theta, rtol=rtol_theta, atol=0), (o.p, info["theta"] - o.theta)
        assert np.allclose(info["resid"], o.resid, rtol=1e-6, atol=1e-12), (o.p, info["resid"], o.resid)
        if o.p >= 2:
            # E^(p) to 1e-10 relative wherever it is not tiny against the order's
            # largest; all entries to 1e-10 of that largest
            big = np.abs(o.E) > 1e-6 * np.abs(o.E).max()
            assert np.allclose(info["E"][big], o.E[big], rtol=1e-10, atol=0), (o.p, info["E"], o.E)
            assert np.all(np.abs(info["E"] - o.E) <= 1e-10 * np.abs(o.E).max()), (o.p, info["E"], o.E)
        if o.p == 1:
            assert np.all(np.abs(info["E"]) <= 1e-12 * np.abs(ref.E0).max())


SMALL8 = W.Workload("small8", [300, 500, 900, 1300], 40, 8, seed=7)


@pytest.mark.parametrize("prec", [0, -1])
@pytest.mark.parametrize("name,orders", [("small", 8), ("c1", 2), (SMALL8, 8), ("c2mini", 3)])
def test_sppc_matches_oracle_order_by_order(name, orders, prec):
    """k = 8 workloads exercise the deflated small solves (opts.minres_deflate)."""
    S, w, rp, c, v, h = _create(name, p_max=max(orders, 2), precision=prec)
    try:
        conv, th, rs, st = S.sppc_solve(h, w.k, tol=1e-300, p_max=orders)
        ref = oracle.sppc(rp, c, v, w.small_dim, w.k, fixed_orders=orders)
        E0 = S.sppc_get_state(h, 5, (w.k,))
        assert np.allclose(E0, ref.E0, rtol=1e-12, atol=0)
        _compare_orders(S, h, ref, w.k)
        assert st["orders"] == orders and st["spmv_h"] == w.k * (orders + 1)
        assert np.allclose(th, ref.theta, rtol=1e-10, atol=0)
    finally:
        S.sppc_destroy(h)


def test_stepwise_api_equals_solve():
    S, w, rp, c, v, h = _create("small", p_max=4)
    try:
        th0, rs0 = S.sppc_start(h, w.k)
        seq = [th0]
        for _ in range(3):
            S.sppc_correct(h)
            th, rs = S.sppc_rayleigh_ritz(h, w.k)
            seq.append(th)
        conv, thS, rsS, st = S.sppc_solve(h, w.k, tol=1e-300, p_max=3)
        assert np.array_equal(thS, seq[-1])
        with pytest.raises(S.SppcError):
            S.sppc_rayleigh_ritz(h, w.k)  # no correction pending
    finally:
        S.sppc_destroy(h)


@pytest.mark.parametrize("prec", [0, -1])
def test_ritz_vectors_and_basis(prec):
    """Returned Z: H Z - Z theta reproduces the reported residuals; Q^T Q = I;
    the projected matrix equals Q^T H Q recomputed on the CPU."""
    S, w, rp, c, v, h = _create("small", p_max=5, precision=prec)
    try:
        Z = torch.zeros((w.n, w.k), dtype=torch.float64, device="cuda")
        conv, th, rs, st = S.sppc_solve(h, w.k, tol=1e-300, p_max=5, Z=Z)
        Zh = Z.cpu().numpy()
        HZ = csr_spmm(rp, c, v, Zh)
        r = np.linalg.norm(HZ - Zh * th, axis=0) / np.abs(th)
        assert np.allclose(r, rs, rtol=1e-5, atol=1e-12)
        m = w.k * 6
        Q = S.sppc_get_state(h, 1, (w.n, m))
        assert np.abs(Q.T @ Q - np.eye(m)).max() <= 1e-12
        Ht = S.sppc_get_state(h, 3, (m, m))
        full = Q.T @ csr_spmm(rp, c, v, Q)
        assert np.abs(Ht - 0.5 * (full + full.T)).max() <= 1e-11 * np.abs(full).max()
    finally:
        S.sppc_destroy(h)


@pytest.mark.parametrize("prec", [0, -1])
def test_small_space_eigenpairs(prec):
    S, w, rp, c, v, h = _create("c1", precision=prec)
    try:
        S.sppc_start(h, w.k)
        psi = S.sppc_get_state(h, 0, (w.small_dim, w.k))
        E0 = S.sppc_get_state(h, 5, (w.k,))
    finally:
        S.sppc_destroy(h)
    n1 = w.small_dim
    H11 = np.zeros((n1, n1))
    for i in range(n1):
        cc = c[rp[i]:rp[i + 1]]
        m = cc < n1
        H11[i, cc[m]] = v[rp[i]:rp[i + 1]][m]
    lam = np.linalg.eigvalsh(H11)[: w.k]
    assert np.allclose(E0, lam, rtol=1e-12)
    assert np.abs(H11 @ psi - psi * E0).max() <= 1e-11
    assert np.abs(psi.T @ psi - np.eye(w.k)).max() <= 1e-12


def test_autotuned_tiling():
    """spmm_chunk_cols = -2: the candidates that fit are timed and one is kept;
    the product equals the one of a handle built with that tile directly."""
    S = _lib()
    w, rp, c, v = make_matrix("c2mini")
    h1 = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts(spmm_chunk_cols=-2))
    try:
        cc, ms = S.sppc_spmm_tiling(h1)
        assert cc == -1 and ms[0] > 0     # 50,000 columns: only the untiled layout is a candidate
        h2 = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts(spmm_chunk_cols=cc))
        try:
            X = torch.from_numpy(W.random_block(w.n, 8, 5)).cuda()
            Y1, Y2 = torch.empty_like(X), torch.empty_like(X)
            S.sppc_spmm(h1, X, Y1)
            S.sppc_spmm(h2, X, Y2)
            torch.cuda.synchronize()
            assert torch.equal(Y1, Y2)
        finally:
            S.sppc_destroy(h2)
    finally:
        S.sppc_destroy(h1)
