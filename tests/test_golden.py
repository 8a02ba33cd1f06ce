"""The oracle against the stored values in tests/golden/ (written by
tests/golden/make_golden.py from the oracle alone): a change to the oracle's
arithmetic fails here until the fixture is regenerated on purpose."""
import json
import os

import numpy as np

import oracle
import workloads as W
from conftest import ROOT, make_matrix


def test_oracle_reproduces_the_stored_small_workload_orders():
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "sppc_small_orders.json")))
    w, rp, c, v = make_matrix("small")
    gw = g["workload"]
    assert (gw["level_sizes"], gw["nnz_per_row"], gw["k"], gw["seed"], gw["n1"]) == \
        (list(w.level_sizes), w.nnz_per_row, w.k, w.seed, w.small_dim)
    orders = len(g["theta"]) - 1
    r = oracle.sppc(rp, c, v, w.small_dim, w.k, fixed_orders=orders, keep=True)
    assert len(r.orders) == orders + 1
    for p, o in enumerate(r.orders):
        assert np.allclose(o.theta, g["theta"][p], rtol=1e-11, atol=0), p
        assert np.allclose(o.resid, g["resid"][p], rtol=1e-7, atol=1e-13), p
    scale = max(np.abs(np.asarray(e)).max() for e in g["E"])
    for p, e in enumerate(r.E):
        assert np.abs(e - np.asarray(g["E"][p])).max() <= 1e-10 * scale, p
    assert W.config("small").name == gw["name"]
