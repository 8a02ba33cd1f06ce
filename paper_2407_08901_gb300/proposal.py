"""Learned correction proposal: training-set collection and training on the GPU.

Not part of the paper.  The network (see ``include/sppc.h``) is trained on
(residual, exact correction) pairs that plain SPPC (Algorithm 2) produces on
smaller synthetic matrices of the 2,000,000-row workload's law (7 levels x2.2,
~200 entries per row): for each training matrix the exact eigenvectors come
from a tight solve (SPPC + block continuation to scaled residual 1e-10), then
plain SPPC runs to a seeded order p and ``sppc_proposal_samples`` turns that
order's Ritz pairs into samples.  Every step of the arithmetic runs in the
library's kernels (features, targets, moments, standardisation, forward,
backward, Adam); this module only moves buffers and draws the seeded sample
orders.

    python -m paper_2407_08901_gb300.proposal --matrices 200 --out proposal_net.npz
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import (NET_FEATURES, NET_PARAMS, sppc_create, sppc_default_opts, sppc_destroy, sppc_feature_moments,
               sppc_mlp_train_epoch, sppc_proposal_samples, sppc_rayleigh_ritz, sppc_correct, sppc_solve,
               sppc_standardize, sppc_start)

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_NET = os.path.join(HERE, "proposal_net.npz")
NH = 64


def init_params(seed: int) -> np.ndarray:
    """Seeded start: weights uniform in +-1/sqrt(fan_in), biases zero, output layer
    zero (the proposal starts as the plain Jacobi block)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.uniform(-1, 1, (NH, NET_FEATURES)) / np.sqrt(NET_FEATURES)
    W2 = rng.uniform(-1, 1, (NH, NH)) / np.sqrt(NH)
    p = np.concatenate([W1.ravel(), np.zeros(NH), W2.ravel(), np.zeros(NH), np.zeros(NH), [0.0]])
    assert p.size == NET_PARAMS
    return p.astype(np.float32)


def training_workload(seed: int, n: int = 50_000):
    import workloads as W
    return W.Workload(f"c5train_{seed}", W.level_sizes_geometric(n, 7, 2.2), 200, 8, seed=seed)


def collect(seeds, n: int = 50_000, keep_fraction: float = 0.125, order_lo: int = 2, order_hi: int = 14,
            sample_seed: int = 0, device: str = "cuda", log=print):
    """Samples (raw features F (N x 6), rhat (N), y (N), CUDA float32) from plain
    SPPC on the training matrices `seeds`; a seeded fraction of each matrix's
    samples is kept."""
    import torch
    import workloads as W
    rng = np.random.Generator(np.random.PCG64(sample_seed))
    gen = torch.Generator(device=device)
    gen.manual_seed(sample_seed)
    Fs, Rs, Ys = [], [], []
    t0 = time.time()
    for m, seed in enumerate(seeds):
        w = training_workload(int(seed), n)
        rp, c, v = W.generate(w)
        k = w.k
        # exact eigenvectors: SPPC + preconditioned continuation to 1e-10
        ho = sppc_default_opts(p_max=15, hybrid=1, switch_order=15, precond=2, precond_iters=10, tol=1e-10,
                               hybrid_maxit=2000)
        h = sppc_create(rp, c, v, w.level_offsets, w.small_dim, k, ho)
        psi = torch.empty(w.n, k, dtype=torch.float64, device=device)
        try:
            conv, _, _, _ = sppc_solve(h, k, tol=1e-10, Z=psi)
        finally:
            sppc_destroy(h)
        if not conv:
            log(f"matrix seed {seed}: exact solve did not reach 1e-10, skipped")
            continue
        # plain SPPC to a seeded order, then the samples of that order's Ritz pairs
        p = int(rng.integers(order_lo, order_hi + 1))
        h = sppc_create(rp, c, v, w.level_offsets, w.small_dim, k, sppc_default_opts(p_max=15))
        try:
            sppc_start(h, k)
            for _ in range(p):
                sppc_correct(h)
                sppc_rayleigh_ritz(h, k)
            cnt = (w.n - w.small_dim) * k
            F = torch.empty(cnt, NET_FEATURES, dtype=torch.float32, device=device)
            rh = torch.empty(cnt, dtype=torch.float32, device=device)
            y = torch.empty(cnt, dtype=torch.float32, device=device)
            got = sppc_proposal_samples(h, psi, F, rh, y)
            assert got == cnt
        finally:
            sppc_destroy(h)
        keep = torch.randperm(cnt, generator=gen, device=device)[: max(1, int(cnt * keep_fraction))]
        Fs.append(F[keep])
        Rs.append(rh[keep])
        Ys.append(y[keep])
        if (m + 1) % 20 == 0 or m == 0:
            log(f"  {m + 1}/{len(seeds)} matrices, order {p}, {time.time() - t0:.1f} s")
    return torch.cat(Fs), torch.cat(Rs), torch.cat(Ys)


def train(F, rhat, y, epochs: int = 4, batch: int = 4096, lr: float = 1e-3, seed: int = 0, log=print):
    """Standardise, then minibatch Adam on the GPU.  Returns (params, mu, sd,
    per-epoch mean batch losses, loss of the m = 0 network and of the trained
    network on one random subset of the samples)."""
    import torch
    from . import sppc_mlp_loss_grad
    mu, sd = sppc_feature_moments(F)
    sd = np.where(sd > 0, sd, 1.0)
    X = torch.empty_like(F)
    sppc_standardize(F, mu, sd, X)
    params = torch.from_numpy(init_params(seed)).to(F.device)
    mom = torch.zeros_like(params)
    vel = torch.zeros_like(params)
    gen = torch.Generator(device=F.device)
    gen.manual_seed(seed)
    step, losses = 0, []
    for ep in range(epochs):
        perm = torch.randperm(F.shape[0], generator=gen, device=F.device)
        step, loss = sppc_mlp_train_epoch(params, mom, vel, X, rhat, y, perm, batch, step, lr)
        losses.append(loss)
        log(f"  epoch {ep + 1}: mean batch loss {loss:.6g}")
    # loss of the plain Jacobi block (m = 0) and of the trained network on the
    # same random subset of the samples
    sub = torch.randperm(F.shape[0], generator=gen, device=F.device)[:262_144]
    Xs, rs, ys = X[sub].contiguous(), rhat[sub].contiguous(), y[sub].contiguous()
    g0 = torch.empty_like(params)
    l0 = torch.empty(1, dtype=torch.float32, device=F.device)
    sppc_mlp_loss_grad(torch.zeros_like(params), Xs, rs, ys, g0, l0)
    loss_m0 = float(l0.item())
    sppc_mlp_loss_grad(params, Xs, rs, ys, g0, l0)
    loss_net = float(l0.item())
    log(f"  loss on a {Xs.shape[0]}-sample subset: m = 0 {loss_m0:.6g}, trained {loss_net:.6g}")
    return params.cpu().numpy(), mu.astype(np.float32), sd.astype(np.float32), losses, loss_m0, loss_net


def save(path: str, params, mu, sd, meta: dict) -> None:
    np.savez(path, params=np.asarray(params, np.float32), mu=np.asarray(mu, np.float32),
             sd=np.asarray(sd, np.float32), meta=json.dumps(meta))


def load(path: str = DEFAULT_NET):
    """(params, mu, sd, meta) of a saved network."""
    z = np.load(path)
    return z["params"], z["mu"], z["sd"], json.loads(str(z["meta"]))


def evaluate(seeds, net_path: str = DEFAULT_NET, n: int = 2_000_000, tol: float = 1e-6, precond_levels: int = 3,
             precond_iters: int = 20, log=print):
    """Solve matrices of the 2,000,000-row law (seeds `seeds`) with SPPC (15
    orders) + preconditioned continuation, with and without the network's
    proposal; per matrix the CUDA-event time, H-vector products, continuation
    steps, proposals kept, and plain SPPC's largest scaled residual after its
    15 orders."""
    import torch
    import workloads as W
    from . import sppc_order_info, sppc_set_proposal
    params, mu, sd, _ = load(net_path)
    rows = []
    for seed in seeds:
        w = W.Workload(f"c2law_{seed}", W.level_sizes_geometric(n, 7, 2.2), 200, 8, seed=int(seed))
        rp, c, v = W.generate(w)
        rec = {"seed": int(seed)}
        for name, prop in (("without", 0), ("learned", 1)):
            o = sppc_default_opts(p_max=15, hybrid=1, switch_order=15, precond=2, precond_iters=precond_iters,
                                  precond_levels=precond_levels, tol=tol, proposal=prop)
            h = sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, o)
            try:
                if prop:
                    sppc_set_proposal(h, params, mu, sd)
                for rep in range(2):   # the second solve is timed
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    conv, th, rs, st = sppc_solve(h, w.k, tol=tol)
                    e1.record()
                    torch.cuda.synchronize()
                if not prop:
                    rec["plain_sppc_resid_after_15"] = float(np.max(sppc_order_info(h, 15, w.k)["resid"]))
                    th0 = np.asarray(th)
            finally:
                sppc_destroy(h)
            rec[name] = {"s": e0.elapsed_time(e1) / 1e3, "converged": bool(conv), "spmv_h": int(st["spmv_h"]),
                         "steps": int(st["refine_steps"]), "kept": int(st["proposals_kept"]),
                         "tried": int(st["proposals_tried"])}
            if prop:
                rec[name]["max_rel_theta_diff"] = float(np.max(np.abs(np.asarray(th) - th0) / np.abs(th0)))
        log(json.dumps(rec))
        rows.append(rec)
    return rows


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--matrices", type=int, default=200, help="training matrices (seeds 1..N)")
    ap.add_argument("--n", type=int, default=50_000, help="rows per training matrix")
    ap.add_argument("--keep", type=float, default=0.125, help="fraction of each matrix's samples kept")
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default=DEFAULT_NET)
    ap.add_argument("--evaluate", type=int, nargs="*", default=None,
                    help="instead of training: evaluate the saved network on these seeds of the 2,000,000-row law")
    a = ap.parse_args(argv)
    if a.evaluate is not None:
        evaluate(a.evaluate or [1000, 1001, 1002, 1003], net_path=a.out)
        return
    t0 = time.time()
    F, rh, y = collect(range(1, a.matrices + 1), n=a.n, keep_fraction=a.keep)
    t1 = time.time()
    print(f"{F.shape[0]} samples from {a.matrices} matrices in {t1 - t0:.1f} s")
    params, mu, sd, losses, base, trained = train(F, rh, y, epochs=a.epochs, batch=a.batch, lr=a.lr)
    t2 = time.time()
    meta = {"matrices": a.matrices, "n": a.n, "samples": int(F.shape[0]), "epochs": a.epochs, "batch": a.batch,
            "lr": a.lr, "losses": losses, "loss_m0": base, "loss_trained": trained, "collect_s": t1 - t0,
            "train_s": t2 - t1}
    save(a.out, params, mu, sd, meta)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
