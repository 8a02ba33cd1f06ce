"""The small solves of Eq. sm_lin_proj by FP32 MINRES with iterative refinement
(opts.minres_fp32), through the C ABI.  GPU only.

Each sweep solves for the current residual in FP32 and the residual is
recomputed in double-float, so the refined solution meets the same tolerance
(1e-12 relative) as the double-float MINRES: the SPPC orders must match the
oracle (dense spectral solve) to 1e-10 in the Ritz values, with FP64 and with
FP32-rounded values (precision 1), and take more than one sweep.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from conftest import make_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SMALL8 = W.Workload("small8", [300, 500, 900, 1300], 40, 8, seed=7)


@pytest.mark.parametrize("name,orders", [("c1", 3), (SMALL8, 6), ("c2mini", 3)])
def test_refined_fp32_minres_orders_match_oracle(name, orders):
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix(name)
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k,
                      S.sppc_default_opts(p_max=orders, minres_fp32=1))
    try:
        conv, th, rs, st = S.sppc_solve(h, w.k, tol=1e-300, p_max=orders)
        ref = oracle.sppc(rp, c, v, w.small_dim, w.k, fixed_orders=orders)
        for o in ref.orders:
            info = S.sppc_order_info(h, o.p, w.k)
            assert np.allclose(info["theta"], o.theta, rtol=1e-10, atol=0), (o.p, info["theta"] - o.theta)
            if o.p >= 2:
                assert np.all(info["minres_iters"] > 0)
    finally:
        S.sppc_destroy(h)


def test_refined_fp32_minres_in_the_mixed_path():
    """precision 1 (FP32 values): the whole method with refined FP32 small solves
    equals the one with double-float small solves to 1e-10 (same rounded matrix,
    same tolerance)."""
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix("c2mini")
    out = []
    for fp32 in (0, 1):
        o = S.sppc_default_opts(p_max=6, hybrid=1, switch_order=4, precond=2, precond_levels=3, tol=1e-9,
                                precision=1, minres_fp32=fp32)
        h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, o)
        try:
            conv, th, rs, st = S.sppc_solve(h, w.k, tol=1e-9)
            assert conv
            out.append(np.asarray(th))
        finally:
            S.sppc_destroy(h)
    assert np.allclose(out[0], out[1], rtol=1e-10, atol=0)
