"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and rejects malformed input before touching the device."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT, make_matrix


def _header_symbols():
    src = open(os.path.join(ROOT, "include", "sppc.h")).read()
    return set(re.findall(r"^\s*(?:sppc_status|void|const char\*|int64_t)\s+(sppc_\w+)\s*\(", src, re.M))


def test_library_exports_every_declared_symbol():
    import ctypes
    import paper_2407_08901_gb300 as S
    lib = ctypes.CDLL(S.LIB)
    declared = _header_symbols()
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(S.EXPORTED_SYMBOLS)


def test_default_opts():
    import paper_2407_08901_gb300 as S
    o = S.sppc_default_opts()
    assert o.p_max == 15 and o.tol == 1e-6 and o.minres_tol == 1e-12 and o.check_symmetry == 0
    assert o.spmm_kernel == 1 and o.reorth == 0 and o.precond == 1 and o.precond_iters == 20


def _small():
    w, rp, c, v = make_matrix("small")
    return w, rp.copy(), c.copy(), v.copy()


@pytest.mark.parametrize("case,status", [
    ("n1_not_level", 3), ("k_zero", 1), ("k_nine", 1), ("levels_bad", 3), ("unsorted", 1), ("col_range", 1),
    ("nan", 11), ("asym", 2), ("rowptr", 1), ("spmm_kernel", 1), ("reorth", 1), ("precond", 1), ("precision", 1),
    ("precision_k", 1), ("precond_levels", 1), ("switch_stall", 1), ("hybrid", 1), ("rmm_mixed", 1),
    ("spin_cap", 1), ("precision_neg", 1), ("f64_rmm", 1), ("f64_proposal", 1),
    ("sigma_odd", 1), ("sigma_big", 1), ("sigma_neg", 1),
])
def test_create_rejects_bad_input(case, status):
    import paper_2407_08901_gb300 as S
    w, rp, c, v = _small()
    lev = w.level_offsets.copy()
    n1, k = w.small_dim, w.k
    opts = S.sppc_default_opts(check_symmetry=1, spmm_kernel=2 if case == "spmm_kernel" else 1,
                               reorth=-1 if case == "reorth" else 0, precond=3 if case == "precond" else 1,
                               precision={"precision": 3, "precision_k": 2, "precision_neg": -2, "f64_rmm": -1,
                                          "f64_proposal": -1}.get(case, 0),
                               precond_levels=99 if case == "precond_levels" else 1,
                               switch_stall=-0.5 if case == "switch_stall" else 0.0,
                               hybrid={"hybrid": 3, "rmm_mixed": 2, "f64_rmm": 2, "f64_proposal": 1}.get(case, 0))
    if case == "f64_proposal":
        opts.proposal = 1
    if case == "rmm_mixed":
        opts.precision = 1
        k = 8
    if case == "spin_cap":
        opts.spin_cap = -1
    if case.startswith("sigma_"):
        opts.sell_sigma = {"sigma_odd": 24, "sigma_big": 2048, "sigma_neg": -1}[case]
    if case == "n1_not_level":
        n1 = n1 + 1
    elif case == "k_zero":
        k = 0
    elif case == "k_nine":
        k = 9
    elif case == "precision_k":
        k = 5      # 6-column blocks: no FP32 product kernel
    elif case == "levels_bad":
        lev[2] = lev[1]
    elif case == "unsorted":
        lo = rp[5]
        c[lo], c[lo + 1] = c[lo + 1], c[lo]
    elif case == "col_range":
        c[10] = w.n + 3
    elif case == "nan":
        v[7] = np.nan
    elif case == "asym":
        v[3] += 1e-3
    elif case == "rowptr":
        rp[-1] += 1
    with pytest.raises(S.SppcError) as ei:
        S.sppc_create(rp, c, v, lev, n1, k, opts)
    assert ei.value.status == status, str(ei.value)
    assert S.sppc_last_error(None)


def test_small_syev_rejects_bad_sizes_before_any_device_call():
    import ctypes
    import paper_2407_08901_gb300 as S
    lib = ctypes.CDLL(S.LIB)
    lib.sppc_small_syev.restype = ctypes.c_int32
    lib.sppc_small_syev.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_void_p]
    buf = ctypes.c_void_p(1)  # never dereferenced: the size check fails first
    assert lib.sppc_small_syev(buf, 200, 200, 8, buf, buf, 8, 0, None) == 1
    assert lib.sppc_small_syev(buf, 10, 10, 0, buf, buf, 8, 0, None) == 1
    assert lib.sppc_small_syev(None, 10, 10, 4, buf, buf, 4, 0, None) == 1
    assert lib.sppc_small_syev(buf, 10, 10, 4, buf, buf, 4, 2, None) == 1  # unknown flag bit


def test_binding_refuses_to_import_without_the_library(tmp_path):
    """The binding has no fallback: a copy of the package whose libsppc.so was
    never built raises ImportError on import, naming the missing library."""
    import shutil
    import subprocess
    import sys
    src = os.path.join(ROOT, "paper_2407_08901_gb300")
    dst = tmp_path / "paper_2407_08901_gb300"
    dst.mkdir()
    for f in os.listdir(src):
        if f.endswith(".py"):
            shutil.copy(os.path.join(src, f), dst / f)
    r = subprocess.run([sys.executable, "-c", "import paper_2407_08901_gb300"], cwd=tmp_path,
                       env={**os.environ, "PYTHONPATH": str(tmp_path)}, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "libsppc.so is missing" in r.stderr


def test_product_path_shares_nothing_with_the_oracle():
    """The package (binding, CUDA sources, header) neither imports, includes nor
    links anything under oracle/, and the oracle imports nothing from the package."""
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b|#\s*include\s+[<\"][^>\"]*oracle)", re.M)
    for d in ("paper_2407_08901_gb300", os.path.join("paper_2407_08901_gb300", "csrc"), "include"):
        for f in os.listdir(os.path.join(ROOT, d)):
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(ROOT, d, f)).read()
                assert not pat.search(src), os.path.join(d, f)
                assert "_oracle_spmm" not in src, os.path.join(d, f)
    back = re.compile(r"^\s*(from\s+paper_2407_08901_gb300\b|import\s+paper_2407_08901_gb300\b)", re.M)
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            assert not back.search(open(os.path.join(ROOT, "oracle", f)).read()), f
