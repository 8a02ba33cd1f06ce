"""Matrices that never visit the host: the device generator and sppc_create from
a device CSR, through the C ABI.  GPU only.

* The device generator (workloads/gen_device.cu) writes the same CSR as the
  host generator, bit for bit (row pointers, columns and every value), on the
  small workloads and on c2 (4.0e8 entries).
* sppc_create from a device CSR reads only the row pointers and the leading
  rows on the host; it must build the same layout and give the same Ritz values,
  bit for bit, as from the host copy, in every value format, and reject the same
  bad input.
"""
import numpy as np
import pytest

import workloads as W
from conftest import make_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("name", ["small", "c1", "c2mini", "c2"])
def test_device_generator_is_bit_identical_to_host(name):
    w, rp, c, v = make_matrix(name)
    drp, dc, dv = W.generate_device(w)
    torch.cuda.synchronize()
    assert np.array_equal(drp.cpu().numpy(), rp)
    assert np.array_equal(dc.cpu().numpy(), c)
    assert np.array_equal(dv.cpu().numpy().view(np.uint64), v.view(np.uint64))


@pytest.mark.parametrize("prec", [0, -1, 1, 2])
def test_create_from_device_csr_equals_host_csr(prec):
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix("c2mini")
    drp, dc, dv = (torch.from_numpy(a).cuda() for a in (rp, c, v))
    opts = dict(p_max=6, hybrid=1, switch_order=3, precond=2, precond_levels=3, tol=1e-9, precision=prec)
    out = []
    for dev in (False, True):
        args = (drp, dc, dv) if dev else (rp, c, v)
        h = S.sppc_create(*args, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts(**opts), on_device=dev)
        try:
            L = S.sppc_get_layout(h)
            conv, th, rs, st = S.sppc_solve(h, w.k, tol=1e-9)
            out.append((L, np.asarray(th), np.asarray(rs), st["spmv_h"]))
        finally:
            S.sppc_destroy(h)
    (L0, t0, r0, s0), (L1, t1, r1, s1) = out
    for key in ("slice_ptr", "slice_rows", "chunk_slice", "h11_slice_ptr", "h11_slice_rows"):
        assert np.array_equal(L0[key], L1[key]), key
    assert np.array_equal(t0, t1) and np.array_equal(r0, r1) and s0 == s1


@pytest.mark.parametrize("case,status", [("nan", 11), ("unsorted", 1), ("col_range", 1), ("asym", 2)])
def test_device_csr_bad_input_is_rejected(case, status):
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix("small")
    c, v = c.copy(), v.copy()
    r = 200  # a row past the small space: its entries are checked on the device only
    lo = rp[r]
    if case == "nan":
        v[lo + 1] = np.nan
    elif case == "unsorted":
        c[lo], c[lo + 1] = c[lo + 1], c[lo]
    elif case == "col_range":
        c[lo + 2] = w.n + 5
    elif case == "asym":
        v[lo + 1] += 1e-3
    drp, dc, dv = (torch.from_numpy(a).cuda() for a in (rp, c, v))
    with pytest.raises(S.SppcError) as err:
        S.sppc_create(drp, dc, dv, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts(check_symmetry=1),
                      on_device=True)
    assert err.value.status == status, str(err.value)
