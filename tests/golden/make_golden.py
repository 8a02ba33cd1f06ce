"""Writes the stored expected values under tests/golden/ from the CPU oracle
alone (and the seeded input generator); nothing here touches the CUDA path.

    python tests/golden/make_golden.py

sppc_small_orders.json: Algorithm 2 on the "small" synthetic workload (2,000
rows in 4 levels, n1 = 300, k = 4, seed 7) for 6 correction orders with exact
small solves: per order the Ritz values (Eq. tilde_H), the scaled residuals
(Eq. rrn) and the correction energies E^(p) (Eq. exp_seq).  The test beside it
re-runs the oracle and compares, so any change to the oracle's arithmetic shows
up there and has to be regenerated here, with the passage that justifies it
named in the change's description.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

ORDERS = 6


def small_orders():
    w = W.config("small")
    rp, c, v = W.generate(w)
    r = oracle.sppc(rp, c, v, w.small_dim, w.k, fixed_orders=ORDERS, keep=True)
    return {
        "cite": "Algorithm 2; Eqs. exp_seq, exp_seq2, sm_lin_proj, blkGS, QR, proj, tilde_H, rrn",
        "workload": {"name": w.name, "level_sizes": list(map(int, w.level_sizes)), "nnz_per_row": int(w.nnz_per_row),
                     "k": int(w.k), "seed": int(w.seed), "n1": int(w.small_dim)},
        "call": f"oracle.sppc(..., n1, k, fixed_orders={ORDERS}, keep=True)  (solver='pinv')",
        "theta": [o.theta.tolist() for o in r.orders],
        "resid": [o.resid.tolist() for o in r.orders],
        "E": [e.tolist() for e in r.E],
    }


if __name__ == "__main__":
    out = os.path.join(HERE, "sppc_small_orders.json")
    with open(out, "w") as f:
        json.dump(small_orders(), f, indent=1)
    print(out)
