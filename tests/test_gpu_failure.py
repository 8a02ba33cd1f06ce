"""Failure detection on the GPU without a fault (GPU only).

A grid barrier of the persistent MINRES kernel is given a spin cap of one poll
(`opts.spin_cap = 1`), so a CTA that has to wait gives up at once: it raises the
kernel's error flag and leaves, the other CTAs leave at their next wait, and the
call returns SPPC_ERR_TIMEOUT.  Every wait stays bounded and no access depends
on the abandoned values, so nothing faults or hangs.  The context stays usable:
a fresh handle on the same device then runs the same orders and matches the
oracle.
"""
import numpy as np
import pytest

import oracle
from conftest import make_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_minres_barrier_time_out_returns_status():
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix("c1")  # n1 = 2,000 rows: 32 MINRES CTAs
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts(p_max=3, spin_cap=1))
    try:
        with pytest.raises(S.SppcError) as err:
            S.sppc_solve(h, w.k, tol=1e-300, p_max=3)
        assert err.value.status == 8, err.value  # SPPC_ERR_TIMEOUT
    finally:
        S.sppc_destroy(h)
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts(p_max=3))
    try:
        conv, th, rs, st = S.sppc_solve(h, w.k, tol=1e-300, p_max=3)
        assert st["orders"] == 3
        ref = oracle.sppc(rp, c, v, w.small_dim, w.k, fixed_orders=3)
        np.testing.assert_allclose(th, ref.theta, rtol=1e-10, atol=0)
    finally:
        S.sppc_destroy(h)


def test_tma_pipeline_wait_time_out_returns_status():
    """The TMA-gather SpMM (spmm_kernel = 0) with spin_cap = 1: every mbarrier wait
    runs out at once (no poll allowed), so each warp gives up at its first stage,
    waits for the copies it issued and leaves; the handle's flag turns the call
    into SPPC_ERR_TIMEOUT.  A fresh handle then multiplies correctly, and the
    flag of the first handle does not leak into it."""
    import workloads as W
    from oracle.spmm import csr_spmm
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix("c1")
    X = np.ascontiguousarray(W.random_block(w.n, 8, 21))
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k,
                      S.sppc_default_opts(p_max=3, spmm_kernel=0, spin_cap=1))
    try:
        Y = np.zeros_like(X)
        with pytest.raises(S.SppcError) as err:
            S.sppc_spmm_host(h, X, Y)
        assert err.value.status == 8, err.value  # SPPC_ERR_TIMEOUT
    finally:
        S.sppc_destroy(h)
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts(p_max=3, spmm_kernel=0))
    try:
        Y = np.zeros_like(X)
        S.sppc_spmm_host(h, X, Y)
        ref = csr_spmm(rp, c, v, X)
        mag = csr_spmm(rp, c, np.abs(v), np.abs(X))
        assert np.all(np.abs(Y - ref) <= 1e-12 * mag)
    finally:
        S.sppc_destroy(h)
