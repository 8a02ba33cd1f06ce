#!/usr/bin/env python3
"""Benchmark: time to the k lowest eigenpairs at scaled residual 1e-6.

Workload (one "step" = one whole solve): the synthetic hierarchical Hamiltonian
with n = 2,000,000 rows in 7 levels growing x2.2 (small space n1 = 9,660 =
level 0), ~200 nonzeros per row (4.02e8), FP64 values, seed 0; k = 8.  Method:
SPPC (Algorithm 2) for 15 correction orders, then the preconditioned block
continuation until every scaled residual ||Hz - theta z|| / |theta| <= 1e-6
(preconditioner: the diagonal of H shifted by each Ritz value, with the leading
block's rows from 10 MINRES steps on the shifted leading block deflated by the
Ritz vector).
The matrix is resident in HBM when a timed step starts (sppc_create is done
before); L2 is flushed (a 512 MB write) before every step.  Each step is timed
with CUDA events on the library's stream.

The JSON line also carries
  e2e:       the same solve through the C ABI from host CSR buffers, with the
             matrix upload (sppc_create) and the Ritz-vector download in the
             timed region;
  roofline:  the SpMM kernel (k SpMVs with H per step of the method): algorithmic
             bytes per launch over its average CUDA-event duration inside the
             timed solves, against the measured HBM copy bandwidth;
  cpu_baseline: the CPU oracle on a bounded sample of the same workload.

--impl reference times the CPU oracle (the reference arm of this project) on
the host cores, each step one bounded sample, scaled to the metric's unit.
Multi-GPU (torchrun): the path does not shard; every rank solves its own
replica and the line reports the slowest rank.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s to k eigenpairs at scaled resid 1e-6 vs FP64 SPPC; SpMM HBM GB/s vs peak"
SWITCH_ORDER = 15
TOL = 1e-6
PRECOND = 2          # continuation: shifted diagonal + deflated leading-block solve
PRECOND_ITERS = 20   # MINRES steps of the leading-block solve
PRECOND_LEVELS = 3   # the leading block spans levels 0-2 (77,670 rows of c2)


def solve_opts(S, n_levels: int = 7, **kw):
    """The timed method's options: SPPC for SWITCH_ORDER orders, then the block
    continuation with the leading-block preconditioner; keyword overrides."""
    base = dict(p_max=SWITCH_ORDER, hybrid=1, switch_order=SWITCH_ORDER, tol=TOL, precond=PRECOND,
                precond_iters=PRECOND_ITERS, precond_levels=min(PRECOND_LEVELS, max(1, n_levels - 1)))
    base.update(kw)
    if base["switch_order"] > base["p_max"]:
        base["p_max"] = base["switch_order"]
    return S.sppc_default_opts(**base)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparator", action="store_true", help="skip the block Lanczos comparator solve")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision solve")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal solve")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched 64-matrix workload")
    ap.add_argument("--no-c3", action="store_true", help="skip the n = 2e7 mixed-precision workload (config 3)")
    ap.add_argument("--tensor-gram", type=int, default=1, choices=[0, 1],
                    help="Gram products against the basis on the tensor cores (opts.tensor_gram)")
    ap.add_argument("--precision", type=int, default=-1, choices=[-1, 0],
                    help="value format of the --profile spmm / solve / minres runs: -1 native FP64, 0 double-float")
    ap.add_argument("--profile", default="none",
                    choices=["none", "spmm", "spmm32", "spmm16", "solve", "minres", "learned", "dense"],
                    help="run the workload's SpMM twice (spmm; spmm32 / spmm16: the FP32- / BF16-value kernels), "
                         "one solve with the bench options (solve), or three plain SPPC orders (minres: two "
                         "small-space MINRES solves, few GB held) or one solve with the learned proposal (learned) "
                         "and exit, for profilers; prints no JSON line")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# Nominal FP64 (DFMA) rate of one GB300: 152 SMs x 2.07 GHz x 2 FMA per clock per
# SM x 2 FLOP = 1.26 TFLOP/s (the rate the GPU's tables give, 1.25 TFLOP/s).
FP64_PEAK_TFLOPS = 1.25


def bench_config(w, nnz: int) -> dict:
    """The workload and method, identical in both arms (no run-dependent keys)."""
    return {"workload": f"{w.name}: n={w.n}, {len(w.level_sizes)} levels x2.2, n1={w.small_dim}, nnz={nnz}, "
                        f"k={w.k}, FP64 values, seed {w.seed}",
            "method": f"SPPC {SWITCH_ORDER} orders + block continuation preconditioned by the shifted diagonal and "
                      f"{PRECOND_ITERS} MINRES steps on the deflated leading block (levels 0-{PRECOND_LEVELS - 1}), "
                      f"to scaled residual {TOL:g}",
            "l2": "flushed by a 512 MB write before every step"}


def read_traffic(name: str):
    """DRAM bytes per launch from a committed one-pass ncu summary
    (profiles/<name>_traffic.json), or None."""
    path = os.path.join(ROOT, "profiles", f"{name}_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f).get("dram_bytes_per_launch")


def spmm_algorithmic_bytes(n: int, nnz: int, kp: int) -> int:
    """Compulsory bytes of one SpMM Y = H X (kp double-float columns): matrix
    values (8 B) and column indices (4 B) once, one row-pointer word per row,
    X read once and Y written once."""
    return nnz * (8 + 4) + (n + 1) * 8 + 2 * n * kp * 8


def _small_start(w, rp, c, v):
    """The oracle's small-space start: the k + 8 lowest eigenpairs of H0_hat by
    ARPACK (all that its MINRES mode needs)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    n1 = w.small_dim
    rows = np.repeat(np.arange(n1), np.diff(rp[: n1 + 1]))
    cc = c[: rp[n1]]
    m = cc < n1
    H11 = sp.csr_matrix((v[: rp[n1]][m], (rows[m], cc[m])), shape=(n1, n1))
    ev, U = sla.eigsh(H11, k=w.k + 8, which="SA", tol=1e-13)
    o = np.argsort(ev)
    return ev[o], U[:, o]


def cpu_oracle_method(w, rp, c, v, switch_order: int = SWITCH_ORDER, max_steps: int = 1000):
    """The timed method on the CPU oracle, as it stands: ARPACK start, SPPC
    (Algorithm 2, MINRES small solves) for switch_order orders, then the
    continuation preconditioned by the shifted diagonal and the deflated
    leading-block MINRES (oracle.hybrid) until every scaled residual is <= TOL
    or max_steps steps.  Returns (seconds, phases, theta, converged, records,
    threads); phases holds the start and the end time of every order and step,
    records the Ritz values of every order and step."""
    import oracle
    from oracle import spmm as ospmm
    threads = os.cpu_count() or 1
    ospmm.set_threads(threads)
    t0 = time.perf_counter()
    small = _small_start(w, rp, c, v)
    marks = [("start", 0, time.perf_counter() - t0)]
    th, rs, conv, rec = oracle.sppc_hybrid(
        rp, c, v, w.small_dim, w.k, switch_order=switch_order, tol=TOL, max_blocks=switch_order + 1,
        maxit=max_steps, precond="lead", solver="minres", lead_iters=PRECOND_ITERS,
        lead_rows=int(w.level_offsets[min(PRECOND_LEVELS, len(w.level_sizes) - 1)]), small_eig=small,
        on_step=lambda ph, i: marks.append((ph, i, time.perf_counter() - t0)))
    return time.perf_counter() - t0, marks, np.asarray(th), bool(conv), rec, threads


def cpu_oracle_modelled(w, rp, c, v, orders: int, steps: int):
    """A bounded sample of the oracle's method: ARPACK start, SPPC orders 0..2,
    one continuation step.  The solve's time is modelled from its pieces: the
    start, orders 0 and 1 (order 1 has no small solve, Eq. first_PC), order 2's
    time for each of the other orders, and the continuation step's time for
    each step.  Returns (modelled seconds, sample seconds, pieces, threads)."""
    t, marks, _, _, _, threads = cpu_oracle_method(w, rp, c, v, switch_order=2, max_steps=1)
    at = {(ph, i): x for ph, i, x in marks}
    pieces = {"start": at[("start", 0)], "order0": at[("sppc", 0)] - at[("start", 0)],
              "order1": at[("sppc", 1)] - at[("sppc", 0)], "order2": at[("sppc", 2)] - at[("sppc", 1)],
              "step1": at[("davidson", 1)] - at[("sppc", 2)]}
    model = (pieces["start"] + pieces["order0"] + pieces["order1"] + (orders - 1) * pieces["order2"]
             + steps * pieces["step1"])
    return model, t, pieces, threads


def slowest_rank(value: float, dist=None, device: str = "cuda") -> float:
    """Replicas under torchrun: every rank solves its own copy of the workload; the
    job's time per step is the slowest rank's (max over ranks)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# The counts of the timed method on c2 (the GPU solve: 15 SPPC orders, then 11
# continuation steps), used by the reference arm, which runs without a GPU.
METHOD_ORDERS = SWITCH_ORDER
METHOD_STEPS = int(os.environ.get("SPPC_BENCH_STEPS", "11"))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import workloads as W
    w = W.config(args.workload)
    rp, c, v = W.generate(w)
    models, samples, pieces = [], [], None
    threads = os.cpu_count() or 1
    for it in range(args.warmup + args.steps):
        model, t, pieces, threads = cpu_oracle_modelled(w, rp, c, v, METHOD_ORDERS, METHOD_STEPS)
        if it >= args.warmup:
            models.append(model)
            samples.append(t)
    value = float(np.mean(models))
    sample = (f"{w.name}: per step, the oracle's method (ARPACK start, SPPC in MINRES mode, lead-preconditioned "
              f"continuation) run to order 2 and one continuation step ({np.mean(samples):.2f} s); the solve "
              f"modelled as start + orders 0-1 + {METHOD_ORDERS - 1} x order 2 + {METHOD_STEPS} x the step "
              f"(last sample's pieces, s: " + ", ".join(f"{k} {x:.2f}" for k, x in pieces.items()) + ")")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(samples)) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(w, int(c.shape[0])),
            "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_c3(S, W, torch, stream, flush):
    """Config 3: n = 2e7 in 9 levels x2.2, ~250 entries per row (5.0e9), k = 8,
    built on the GPU by the device generator (its host CSR would be 60 GB).  The
    method with FP32 values, then with BF16 off-diagonal values (FP32
    accumulation, double-float projection); each eigenvalue's error against an
    FP64 solve of the same rounded matrix (the solver's error) and against the
    FP64 solve of the unrounded H (the rounding of H's values)."""
    w3 = W.config("c3")
    nlev = len(w3.level_sizes)
    t0 = time.perf_counter()
    rp3, c3, v3 = W.generate_device(w3)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    n3, nnz3, k3 = w3.n, int(c3.numel()), w3.k
    out = {"workload": f"c3: n={n3}, {nlev} levels x2.2, n1={w3.small_dim}, nnz={nnz3}, k={k3}, seed {w3.seed}, "
                       "generated on the device", "generate_s": t_gen}

    def solve(prec=-1, rounding=0):
        o = solve_opts(S, nlev, timing=1, precision=prec, value_rounding=rounding)
        hh = S.sppc_create(rp3, c3, v3, w3.level_offsets, w3.small_dim, k3, o, stream=stream, on_device=True)
        try:
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                conv_, th_, rs_, st_ = S.sppc_solve(hh, k3, tol=TOL, stream=stream)
                e1.record(stream)
            e1.synchronize()
        finally:
            S.sppc_destroy(hh)
        return e0.elapsed_time(e1) / 1e3, bool(conv_), np.asarray(th_), np.asarray(rs_), st_

    t64, cv64, th64, rs64, st64 = solve(-1, 0)
    out["f64"] = {"value": t64, "unit": "s", "converged": cv64, "spmv_h": st64["spmv_h"],
                  "max_scaled_resid": float(np.max(rs64)),
                  "spmm_ms_per_product": st64["spmm_ms"] / max(st64["spmm_launches"], 1)}
    peak, peak_kind = peaks()
    for prec, key, bytes_val in ((1, "fp32", 4), (2, "bf16", 2)):
        tm, cvm, thm, rsm, stm = solve(prec, 0)
        tr, cvr, thr, rsr, _ = solve(-1, prec)
        spmm_ms = stm["spmm_ms"] / max(stm["spmm_launches"], 1)
        alg = nnz3 * (bytes_val + 4) + (n3 + 1) * 8 + n3 * 8 * 4 + n3 * 8 * 8
        out[key] = {
            "method": ("H values rounded to FP32" if prec == 1 else "off-diagonal values rounded to BF16 (diagonal "
                       "FP32)") + "; FP32 products with H until the residual estimates reach 1e-6, then "
                       "double-float products; Gram, CholeskyQR2, projected eigensolve and MINRES in double-float",
            "value": tm, "unit": "s", "speedup_vs_f64": t64 / tm, "converged": cvm, "spmv_h": stm["spmv_h"],
            "max_scaled_resid": float(np.max(rsm)),
            "max_rel_theta_err_vs_f64_same_rounded_matrix": float(np.max(np.abs(thm - thr) / np.abs(thr))),
            "f64_same_rounded_matrix": {"value": tr, "converged": cvr, "max_scaled_resid": float(np.max(rsr))},
            "max_rel_theta_diff_vs_f64_unrounded": float(np.max(np.abs(thm - th64) / np.abs(th64))),
            "spmm": {"kernel": f"k_spmm_sell_f32r (FP32 X, {'FP32' if prec == 1 else 'BF16'} values)",
                     "ms_per_product": spmm_ms, "algorithmic_bytes": alg,
                     "achieved_GBps": alg / (spmm_ms * 1e-3) / 1e9,
                     "frac": alg / (spmm_ms * 1e-3) / 1e9 / peak, "peak": peak, "peak_kind": peak_kind}}
    del rp3, c3, v3
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch

    import paper_2407_08901_gb300 as S
    import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = W.config(args.workload)
    rp, c, v = W.generate(w)
    n, nnz, k = w.n, int(c.shape[0]), w.k
    kp = (k + 1) // 2 * 2
    stream = torch.cuda.Stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed_solve(hh, **kw):
        """One solve on `stream` after a 512 MB L2 flush, timed with CUDA events."""
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = S.sppc_solve(hh, k, tol=TOL, stream=stream, **kw)
            e1.record(stream)
        e1.synchronize()
        return (e0.elapsed_time(e1),) + tuple(out)

    # the headline: the method in native FP64 (every value an IEEE double, DFMA)
    opts = solve_opts(S, len(w.level_sizes), timing=1, precision=-1, tensor_gram=args.tensor_gram)
    h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k, opts, stream=stream)
    for _ in range(args.warmup):
        timed_solve(h)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = S.sppc_kernel_launches()
    times, stats = [], []
    for _ in range(args.steps):
        ms, conv, th, rs, st = timed_solve(h)
        times.append(ms)
        stats.append(st)
    launches = S.sppc_kernel_launches() - launches0
    th_last = np.asarray(th)
    barrier()
    clk = clocks.stop()
    ms_step = slowest_rank(float(np.mean(times)), dist, "cuda")
    # plain SPPC's own result: the largest scaled residual after its last order;
    # the Ritz values of every SPPC order (parity with the oracle below)
    plain_resid = float(np.max(S.sppc_order_info(h, int(st["switched_at"]), k)["resid"]))
    order_theta = [np.asarray(S.sppc_order_info(h, p, k)["theta"]) for p in range(int(st["switched_at"]) + 1)]
    S.sppc_destroy(h)

    # end to end through the C ABI from host buffers
    e2e_times = []
    Zh = torch.empty((n, k), dtype=torch.float64, pin_memory=True)
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        he = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k, opts, stream=stream)
        Zd = torch.empty((n, k), dtype=torch.float64, device="cuda")
        S.sppc_solve(he, k, tol=TOL, Z=Zd, stream=stream)
        with torch.cuda.stream(stream):
            Zh.copy_(Zd, non_blocking=True)
        stream.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        S.sppc_destroy(he)
        del Zd
    h2d = rp.nbytes + c.nbytes + v.nbytes + w.level_offsets.nbytes
    d2h = n * k * 8 + 2 * k * 8

    peak, peak_kind = peaks()
    st = stats[-1]
    spmm_ms = sum(s_["spmm_ms"] for s_ in stats)
    spmm_n = sum(s_["spmm_launches"] for s_ in stats)
    avg_ms = spmm_ms / max(spmm_n, 1)
    alg = spmm_algorithmic_bytes(n, nnz, kp)
    flops = 2 * nnz * kp
    line = {
        "metric": METRIC, "value": ms_step / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(w, nnz),
        "solve": {"orders": st["orders"], "refine_steps": st["refine_steps"], "spmv_h": st["spmv_h"],
                  "converged": bool(st["converged"]), "max_scaled_resid": float(np.max(rs)),
                  "parallelism": "replicas" if world > 1 else "1 GPU"},
        "e2e": {"value": float(np.mean(e2e_times)), "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "roofline": {"kernel": "k_spmm_sell<8, FP64>", "bound": "alu",
                     "achieved": flops / (avg_ms * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                     "peak_kind": "nominal FP64 (DFMA) rate, 152 SMs x 2.07 GHz x 2 FMA/clk x 2 FLOP",
                     "unit": "TFLOP/s", "frac": flops / (avg_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                     "traffic": read_traffic("spmm_f64_c2"), "flops_per_launch": flops,
                     "avg_launch_ms": avg_ms, "launches": spmm_n,
                     "hbm": {"algorithmic_bytes": alg, "achieved": alg / (avg_ms * 1e-3) / 1e9, "peak": peak,
                             "peak_kind": peak_kind, "unit": "GB/s",
                             "frac": alg / (avg_ms * 1e-3) / 1e9 / peak},
                     "launch_unit": "one 8-column product H X (all column tiles)"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "breakdown_ms_per_step": {kk: float(np.mean([s_[kk] for s_ in stats]))
                                  for kk in ("spmm_ms", "minres_ms", "small_eig_ms", "dense_ms", "total_ms")},
    }
    if rank == 0 and world == 1:
        # the same method in double-float (two fp32 words, ~48 bits, on the FP32
        # pipes): time, agreement with the FP64 run, and its SpMM against HBM
        hd = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k,
                           solve_opts(S, len(w.level_sizes), timing=1, tensor_gram=args.tensor_gram), stream=stream)
        timed_solve(hd)
        dts, dstats = [], []
        for _ in range(3):
            ms_d, dconv, dth, drs, dst = timed_solve(hd)
            dts.append(ms_d)
            dstats.append(dst)
        S.sppc_destroy(hd)
        d_ms = sum(x["spmm_ms"] for x in dstats) / max(sum(x["spmm_launches"] for x in dstats), 1)
        line["df64"] = {
            "method": "the same method with double-float values and arithmetic (fp32 pairs, ~48 significant "
                      "bits, error-free transformations on the FP32 pipes)",
            "value": float(np.mean(dts)) / 1e3, "unit": "s", "speedup_vs_f64": ms_step / float(np.mean(dts)),
            "spmv_h": dstats[-1]["spmv_h"], "converged": bool(dconv), "max_scaled_resid": float(np.max(drs)),
            "max_rel_theta_diff_vs_f64": float(np.max(np.abs(np.asarray(dth) - th_last) / np.abs(th_last))),
            "breakdown_ms_per_step": {kk: float(np.mean([x[kk] for x in dstats]))
                                      for kk in ("spmm_ms", "minres_ms", "small_eig_ms", "dense_ms")},
            "roofline": {"kernel": "k_spmm_sell<8>", "bound": "hbm", "achieved": alg / (d_ms * 1e-3) / 1e9,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": alg / (d_ms * 1e-3) / 1e9 / peak, "traffic": read_traffic("spmm_df64_c2"),
                         "algorithmic_bytes": alg, "avg_launch_ms": d_ms,
                         "gather_bytes": nnz * kp * 8,
                         "gather_GBps": nnz * kp * 8 / (d_ms * 1e-3) / 1e9}}
        df_th = np.asarray(dth)
    if rank == 0 and world == 1 and not args.no_mixed:
        # mixed precision (H rounded to FP32, or off-diagonals to BF16; FP32 products
        # with H during the solve, double-float elsewhere, double-float products at
        # the end): one solve timed with CUDA events.  Eigenvalues against an FP64
        # solve of the same rounded matrix (the solver error) and against this run's
        # FP64 solve of the unrounded H (the quantisation of H's values).
        rows = np.repeat(np.arange(n), np.diff(rp))
        f32 = v.astype(np.float32)
        u = f32.view(np.uint32).astype(np.uint64)
        bf = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32)
        rounded = {1: f32.astype(np.float64), 2: np.where(rows == c, f32, bf).astype(np.float64)}
        del rows, u, bf
        for prec, key, desc in ((1, "mixed_precision", "H values rounded to FP32"),
                                (2, "mixed_precision_bf16", "off-diagonal values rounded to BF16 (diagonal FP32)")):
            mopts = solve_opts(S, timing=1, precision=prec)
            hm = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k, mopts, stream=stream)
            mt = []
            for _ in range(2):
                with torch.cuda.stream(stream):
                    flush.fill_(1.0)
                    m0 = torch.cuda.Event(enable_timing=True)
                    m1 = torch.cuda.Event(enable_timing=True)
                    m0.record(stream)
                    mconv, mth, mrs, mst = S.sppc_solve(hm, k, tol=TOL, stream=stream)
                    m1.record(stream)
                torch.cuda.synchronize()
                mt.append(m0.elapsed_time(m1) / 1e3)
            S.sppc_destroy(hm)
            ropts = solve_opts(S, len(w.level_sizes), precision=-1)
            hr = S.sppc_create(rp, c, rounded[prec], w.level_offsets, w.small_dim, k, ropts, stream=stream)
            _, rth, _, _ = S.sppc_solve(hr, k, tol=TOL, stream=stream)
            S.sppc_destroy(hr)
            mth, rth, th0 = np.asarray(mth), np.asarray(rth), np.asarray(th_last)
            line[key] = {
                "method": desc + "; FP32 products with H (FP32 X, FP32 accumulation) until the residual "
                          "estimates reach 1e-6, then a restart with double-float products; Gram, CholeskyQR2, "
                          "projected eigensolve and MINRES in double-float",
                "value": mt[-1], "unit": "s", "speedup_vs_f64": ms_step / 1e3 / mt[-1], "spmv_h": mst["spmv_h"],
                "converged": bool(mconv), "max_scaled_resid": float(np.max(mrs)), "spmm_ms": mst["spmm_ms"],
                "max_rel_theta_err_vs_fp64_same_rounded_matrix": float(np.max(np.abs(mth - rth) / np.abs(rth))),
                "max_rel_theta_diff_vs_fp64_unrounded": float(np.max(np.abs(mth - th0) / np.abs(th0)))}
        del rounded
    if rank == 0 and world == 1 and not args.no_mixed:
        # the small solves by FP32 MINRES with iterative refinement in double-float,
        # against the double-float MINRES, in the double-float and FP32-value paths
        fr = {}
        for prec, key in ((0, "df64_values"), (1, "fp32_values")):
            res = {}
            for fp32 in (0, 1):
                hf = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k,
                                   solve_opts(S, timing=1, precision=prec, minres_fp32=fp32), stream=stream)
                try:
                    timed_solve(hf)
                    ms_f, fconv, fth, frs, fst = timed_solve(hf)
                finally:
                    S.sppc_destroy(hf)
                res["fp32_refined" if fp32 else "double_float"] = {
                    "value": ms_f / 1e3, "unit": "s", "minres_ms": fst["minres_ms"],
                    "minres_iters": fst["minres_iters"], "converged": bool(fconv),
                    "max_rel_theta_diff_vs_f64": float(np.max(np.abs(np.asarray(fth) - th_last) / np.abs(th_last)))}
            fr[key] = res
        line["minres_fp32_refinement"] = fr
    if rank == 0 and world == 1 and not args.no_c3:
        line["c3"] = run_c3(S, W, torch, stream, flush)
    if rank == 0 and world == 1 and not args.no_learned:
        # learned correction proposal: the same solve with the trained network's
        # block in each continuation step (kept iff the largest scaled residual
        # drops), network from the committed training run
        from paper_2407_08901_gb300 import proposal as PR
        if os.path.exists(PR.DEFAULT_NET):
            params, mu, sd, meta = PR.load(PR.DEFAULT_NET)
            lopts = solve_opts(S, timing=1, proposal=1)
            hl = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k, lopts, stream=stream)
            S.sppc_set_proposal(hl, params, mu, sd)
            lt = []
            for _ in range(2):
                with torch.cuda.stream(stream):
                    flush.fill_(1.0)
                    l0 = torch.cuda.Event(enable_timing=True)
                    l1 = torch.cuda.Event(enable_timing=True)
                    l0.record(stream)
                    lconv, lth, lrs, lst = S.sppc_solve(hl, k, tol=TOL, stream=stream)
                    l1.record(stream)
                torch.cuda.synchronize()
                lt.append(l0.elapsed_time(l1) / 1e3)
            S.sppc_destroy(hl)
            line["learned_proposal"] = {
                "method": "per-row network (6 features, 2x64 GELU, BF16 inference) proposing each continuation "
                          "step's block as (r / (diag(H) - theta)) (1 + m); kept iff the largest scaled residual "
                          "drops, else the plain preconditioned block",
                "training": {kk: meta.get(kk) for kk in ("matrices", "n", "samples", "epochs", "losses", "loss_m0",
                                                          "loss_trained")},
                "value": lt[-1], "unit": "s", "spmv_h": lst["spmv_h"], "steps": lst["refine_steps"],
                "proposals_kept": lst["proposals_kept"], "proposals_tried": lst["proposals_tried"],
                "converged": bool(lconv), "max_scaled_resid": float(np.max(lrs)),
                "vs_without": {"what": "the same method in double-float without the network",
                               "value": line["df64"]["value"], "spmv_h": dstats[-1]["spmv_h"],
                               "steps": dstats[-1]["refine_steps"]},
                "vs_f64": {"value": ms_step / 1e3, "spmv_h": st["spmv_h"]},
                "plain_sppc_after_15_orders_max_scaled_resid": plain_resid,
                "max_rel_theta_diff_vs_fp64": float(np.max(np.abs(np.asarray(lth) - np.asarray(th_last))
                                                           / np.abs(np.asarray(th_last))))}
            # held-out matrices of the same law (seeds 1000-1003, n = 2e6, built on the
            # device): the method with and without the network, one solve each
            held = {}
            for seed in (1000, 1001, 1002, 1003):
                wt = W.Workload(f"c2_seed{seed}", w.level_sizes, w.nnz_per_row, k, seed=seed)
                trp, tc, tv = W.generate_device(wt)
                res = {}
                for key, kw in (("plain", {}), ("learned", {"proposal": 1})):
                    ht = S.sppc_create(trp, tc, tv, wt.level_offsets, wt.small_dim, k, solve_opts(S, timing=1, **kw),
                                       stream=stream, on_device=True)
                    if kw:
                        S.sppc_set_proposal(ht, params, mu, sd)
                    try:
                        ms_t, tconv, tth, trs, tst = timed_solve(ht)
                    finally:
                        S.sppc_destroy(ht)
                    res[key] = {"value": ms_t / 1e3, "spmv_h": tst["spmv_h"], "steps": tst["refine_steps"],
                                "converged": bool(tconv)}
                    if kw:
                        res[key]["proposals_kept"] = tst["proposals_kept"]
                        res[key]["proposals_tried"] = tst["proposals_tried"]
                held[str(seed)] = res
                del trp, tc, tv
            line["learned_proposal"]["held_out_seeds"] = held
        else:
            line["learned_proposal"] = {"unavailable": "no trained network at " + os.path.relpath(PR.DEFAULT_NET, ROOT)}
    if rank == 0 and world == 1 and not args.no_batched:
        # batched workload: 64 independent matrices, n log-uniform in [5e3, 2e5],
        # 3-6 levels, ~80 entries per row, k = 4, FP32 products with H and
        # double-float projection; all solved by the concurrent batch runner,
        # wall clock around the whole batch (one worker = one by one)
        ws = W.c4_batch(64, seed=0)
        mats = [W.generate(wb) for wb in ws]
        res = {}
        for nwork in (1, 8, 16):
            hs = [S.sppc_create(rpb, cb, vb, wb.level_offsets, wb.small_dim, wb.k,
                                solve_opts(S, len(wb.level_sizes), precision=1, hybrid_maxit=2000))
                  for wb, (rpb, cb, vb) in zip(ws, mats)]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bst, bth, brs, bcv, bstats = S.sppc_solve_batch(hs, 4, tol=TOL, workers=nwork)
            torch.cuda.synchronize()
            res[nwork] = (time.perf_counter() - t0, bcv, bstats, brs)
            for hb in hs:
                S.sppc_destroy(hb)
        t1, cv1, st1, rs1 = res[1]
        best = min((8, 16), key=lambda q: res[q][0])
        t8, cv8, st8, rs8 = res[best]
        line["batched"] = {
            "workload": "64 matrices, n log-uniform in [5e3, 2e5] (total " + str(sum(wb.n for wb in ws)) +
                        " rows, " + str(int(sum(m[1].shape[0] for m in mats))) + " entries), 3-6 levels x2.2, "
                        "~80 entries/row, k=4, seeds 0..63",
            "method": f"concurrent batch runner, {best} host threads x 1 CUDA stream each, largest first; each "
                      "problem SPPC + preconditioned continuation, FP32 products with H",
            "value": t8, "unit": "s", "matrices_per_s": 64 / t8, "one_by_one_s": t1,
            "workers_s": {str(q): res[q][0] for q in res},
            "converged": int(cv8.sum()), "max_scaled_resid": float(np.max(rs8)),
            "spmv_h": int(sum(x["spmv_h"] for x in st8))}
        # the batch's products Y_m = H_m X_m (4 columns): 64 sppc_spmm calls
        # against one graph replay of the batched persistent launch
        hs = [S.sppc_create(rpb, cb, vb, wb.level_offsets, wb.small_dim, wb.k, S.sppc_default_opts(p_max=1))
              for wb, (rpb, cb, vb) in zip(ws, mats)]
        Xs = [torch.from_numpy(W.random_block(wb.n, 4, 7)).cuda() for wb in ws]
        Ys = [torch.empty_like(X) for X in Xs]
        plan = S.sppc_spmm_batch_plan(hs, Xs, Ys)
        def timed(fn, reps=5):
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) / reps
        t_loop = timed(lambda: [S.sppc_spmm(hb, X, Y) for hb, X, Y in zip(hs, Xs, Ys)])
        t_graph = timed(lambda: S.sppc_spmm_batch_run(plan))
        S.sppc_spmm_batch_destroy(plan)
        for hb in hs:
            S.sppc_destroy(hb)
        nnz_all = int(sum(m[1].shape[0] for m in mats))
        line["batched"]["spmm"] = {
            "what": "the 64 products Y_m = H_m X_m with 4 columns, double-float",
            "per_matrix_calls_ms": t_loop * 1e3, "one_graph_replay_ms": t_graph * 1e3,
            "graph_algorithmic_GBps": (nnz_all * 12 + sum(wb.n * 4 * 8 * 2 for wb in ws)) / t_graph / 1e9}
        del mats
    if rank == 0 and world == 1 and not args.no_comparator:
        # the SpMM layout chosen by the library's autotuners: the column tile
        # (spmm_chunk_cols = -2), then the SELL sort window at that tile
        # (sell_sigma = -2), in both value formats
        tune = {}
        for prec, key in ((0, "double_float"), (-1, "f64")):
            ht = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k,
                               S.sppc_default_opts(p_max=1, spmm_chunk_cols=-2, sell_sigma=-2, precision=prec),
                               stream=stream)
            tc, tms = S.sppc_spmm_tiling(ht)
            sg, sms = S.sppc_sell_sigma(ht)
            S.sppc_destroy(ht)
            tune[key] = {
                "chosen_columns_per_tile": tc,
                "ms_per_product": {name: float(x) for name, x in zip(("untiled", "2621440", "1310720", "655360",
                                                                      "327680"), tms) if x > 0},
                "chosen_sigma": sg,
                "ms_per_product_by_sigma": {str(s_): float(x) for s_, x in zip((64, 256, 1024), sms)}}
        line["spmm_tile_autotune"] = tune
    if rank == 0 and world == 1 and not args.no_comparator:
        # the paper's own hybrid: SPPC for 15 orders, then per-pair RMM-DIIS
        # (Jacobi preconditioner, DIIS depth 8), capped at 600 iterations
        hr_ = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k,
                            S.sppc_default_opts(p_max=SWITCH_ORDER, hybrid=2, switch_order=SWITCH_ORDER, tol=TOL,
                                                hybrid_maxit=600), stream=stream)
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            r0 = torch.cuda.Event(enable_timing=True)
            r1 = torch.cuda.Event(enable_timing=True)
            r0.record(stream)
            rconv, rth, rrs, rst = S.sppc_solve(hr_, k, tol=TOL, stream=stream)
            r1.record(stream)
        torch.cuda.synchronize()
        S.sppc_destroy(hr_)
        line["sppc_rmm_diis"] = {
            "method": "the paper's hybrid: SPPC 15 orders, then per-pair RMM-DIIS (Jacobi preconditioner, DIIS "
                      "depth 8, step 1), one 8-column product per iteration, at most 600 iterations",
            "value": r0.elapsed_time(r1) / 1e3, "unit": "s", "converged": bool(rconv),
            "pairs_converged": int(np.sum(np.asarray(rrs) <= TOL)), "max_scaled_resid": float(np.max(rrs)),
            "iterations": rst["refine_steps"], "spmv_h": rst["spmv_h"]}
    if rank == 0 and world == 1 and not args.no_comparator:
        # sensitivity to the switch point: the same method switching to the
        # continuation after fewer SPPC orders (the paper switches at stagnation,
        # about order 15; the timed method keeps that)
        sw = {}
        for so in (6, 3, "stall"):
            so_opts = (solve_opts(S, switch_stall=0.9) if so == "stall" else solve_opts(S, switch_order=so))
            hs_ = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k, so_opts, stream=stream)
            for _ in range(2):
                with torch.cuda.stream(stream):
                    flush.fill_(1.0)
                    s0 = torch.cuda.Event(enable_timing=True)
                    s1 = torch.cuda.Event(enable_timing=True)
                    s0.record(stream)
                    sconv, sth, srs, sst = S.sppc_solve(hs_, k, tol=TOL, stream=stream)
                    s1.record(stream)
                torch.cuda.synchronize()
            S.sppc_destroy(hs_)
            key = ("switch_when_a_residual_drops_less_than_10pct" if so == "stall"
                   else f"switch_after_{so}_orders")
            sw[key] = {"value": s0.elapsed_time(s1) / 1e3, "unit": "s", "spmv_h": sst["spmv_h"],
                       "steps": sst["refine_steps"], "switched_at": sst["switched_at"], "converged": bool(sconv)}
        line["switch_sensitivity"] = sw
    if rank == 0 and world == 1 and not args.no_comparator:
        # C2's comparator: block Lanczos from Psi^(0) (the same loop, no SPPC orders,
        # no preconditioner), one untimed-loop solve timed with CUDA events
        copts = S.sppc_default_opts(p_max=SWITCH_ORDER, hybrid=1, switch_order=0, tol=TOL, precond=0,
                                    hybrid_maxit=5000)
        hc = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k, copts, stream=stream)
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            cconv, cth, crs, cst = S.sppc_solve(hc, k, tol=TOL, stream=stream)
            c1.record(stream)
        torch.cuda.synchronize()
        line["comparator"] = {"method": "block Lanczos from Psi^(0), full reorthogonalisation, thick restart",
                              "value": c0.elapsed_time(c1) / 1e3, "unit": "s", "spmv_h": cst["spmv_h"],
                              "steps": cst["refine_steps"], "converged": bool(cconv),
                              "max_rel_theta_diff": float(np.max(np.abs(np.asarray(cth) - np.asarray(th_last))
                                                                 / np.abs(np.asarray(th_last))))}
        S.sppc_destroy(hc)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's whole method, once, on the host cores; its eigenvalues
        # against the GPU's FP64 solve; and the reference arm's bounded-sample
        # model of the same solve, to show how far the two agree
        t, marks, cth_, cconv_, crec, threads = cpu_oracle_method(w, rp, c, v)
        sppc_rel = [float(np.max(np.abs(order_theta[r.step] - r.theta) / np.abs(r.theta)))
                    for r in crec if r.phase == "sppc" and r.step < len(order_theta)]
        at = {(ph, i): x for ph, i, x in marks}
        t_sppc = at.get(("sppc", SWITCH_ORDER), t) - at[("start", 0)]
        model, tsample, pieces, _ = cpu_oracle_modelled(w, rp, c, v, SWITCH_ORDER, int(st["refine_steps"]))
        line["cpu_baseline"] = {
            "value": t, "unit": "s", "cores": threads, "kind": "oracle",
            "sample": f"{w.name}: full solve, the oracle's method as it stands (ARPACK start, SPPC {SWITCH_ORDER} "
                      f"orders in MINRES mode, lead-preconditioned continuation to {TOL:g}), one timed run",
            "phases_s": {"start": at[("start", 0)], "sppc_orders": t_sppc,
                         "continuation": t - at[("start", 0)] - t_sppc},
            "converged": cconv_, "spmv_h": int(crec[-1].spmv),
            "max_rel_theta_diff_vs_gpu_f64": float(np.max(np.abs(cth_ - th_last) / np.abs(th_last))),
            "reference_arm_model_s": model, "reference_arm_sample_s": tsample}
        # parity of the timed FP64 solve with the oracle, order by order over the
        # SPPC phase (the continuation's trajectories part at rounding level)
        line["parity_vs_oracle"] = {
            "what": "max relative difference of the k Ritz values, GPU FP64 solve vs the CPU oracle, per SPPC order",
            "orders": len(sppc_rel), "max_rel_theta_per_order": sppc_rel, "max_rel_theta": max(sppc_rel),
            "bound": 1e-10, "ok": bool(max(sppc_rel) <= 1e-10)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_profile(args):
    """Fixed, short invocations of the library for profilers (ncu launch lists and
    counter captures): two 8-column SpMM products with H, or one whole solve with
    the options the timed steps use."""
    import torch

    import paper_2407_08901_gb300 as S
    import workloads as W

    if args.profile == "dense":
        # the tensor-core Gram and update kernels alone on n = 5e5 rows (A = 512 MB
        # of FP64 values, 1 GB of digit tiles at 16 blocks), 1 and 16 blocks
        n = 500_000
        g = torch.Generator(device="cuda").manual_seed(1)
        A = torch.randn(16, n, 8, device="cuda", dtype=torch.float64, generator=g) / n ** 0.5
        B = torch.randn(n, 8, device="cuda", dtype=torch.float64, generator=g)
        for nb in (1, 16):
            C = torch.randn(8 * nb, 8, device="cuda", dtype=torch.float64, generator=g)
            S.sppc_block_gram(A[:nb].contiguous(), B, tensor=True, df=args.precision == 0)
            S.sppc_block_update(A[:nb].contiguous(), C, None, B, tensor=True, df=args.precision == 0)
        torch.cuda.synchronize()
        print(f"profile dense: n {n}, blocks 1 and 16, precision {args.precision}", flush=True)
        return 0
    w = W.config(args.workload)
    rp, c, v = W.generate(w)
    k = w.k
    if args.profile in ("spmm32", "spmm16"):
        prec = 1 if args.profile == "spmm32" else 2
        h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k, S.sppc_default_opts(p_max=1, precision=prec))
        X = torch.from_numpy(W.random_block(w.n, 8, 1)).cuda()
        Y = torch.empty_like(X)
        for _ in range(2):
            S.sppc_spmm(h, X, Y)
        torch.cuda.synchronize()
        print(f"profile {args.profile}: {w.name}, 2 products", flush=True)
    elif args.profile == "spmm":
        h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k,
                          S.sppc_default_opts(p_max=1, precision=args.precision))
        X = torch.from_numpy(W.random_block(w.n, 8, 1)).cuda()
        Y = torch.empty_like(X)
        for _ in range(2):
            S.sppc_spmm(h, X, Y)
        torch.cuda.synchronize()
        print(f"profile spmm: {w.name}, 2 products, column tiles {S.sppc_get_layout(h)['n_chunks']}", flush=True)
    elif args.profile == "learned":
        from paper_2407_08901_gb300 import proposal as PR
        params, mu, sd, _ = PR.load(PR.DEFAULT_NET)
        h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k, solve_opts(S, len(w.level_sizes), proposal=1))
        S.sppc_set_proposal(h, params, mu, sd)
        conv, th, rs, st = S.sppc_solve(h, k, tol=TOL)
        torch.cuda.synchronize()
        print(f"profile learned: {w.name}, converged {conv}, steps {st['refine_steps']}", flush=True)
    elif args.profile == "minres":
        h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k,
                          S.sppc_default_opts(p_max=3, precision=args.precision))
        conv, th, rs, st = S.sppc_solve(h, k, tol=1e-300, p_max=3)
        torch.cuda.synchronize()
        print(f"profile minres: {w.name}, orders {st['orders']}, MINRES iterations {st['minres_iters']}", flush=True)
    else:
        opts = solve_opts(S, len(w.level_sizes), precision=args.precision, tensor_gram=args.tensor_gram)
        h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, k, opts)
        conv, th, rs, st = S.sppc_solve(h, k, tol=TOL)
        torch.cuda.synchronize()
        print(f"profile solve: {w.name}, converged {conv}, orders {st['orders']}, steps {st['refine_steps']}, "
              f"launches {S.sppc_kernel_launches()}", flush=True)
    S.sppc_destroy(h)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile != "none":
        return run_profile(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
