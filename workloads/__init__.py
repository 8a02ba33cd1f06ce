"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module holds no eigensolver arithmetic.  It defines the five workloads
(sizes, level partitions, value law, seeds) and generates

* the symmetric hierarchical Hamiltonian H (CSR, FP64 values, int32 columns,
  int64 row pointers) through the C generator in ``gen.cpp``, or directly in
  GPU memory through its bit-identical device form ``gen_device.cu`` (for the
  matrices whose host CSR would not fit or would take minutes to upload);
* seeded dense blocks for SpMM and solver inputs.

The paper's test matrices (NCSM Hamiltonians of 6Li, 7Li, 11B, 12C with the
Daejeon16 interaction, Sec. 6 Table I) are not available; these synthetic
matrices stand in for them and imitate their hierarchy (the leading submatrix
is the smaller configuration space, Sec. 1 and Sec. 2 Eq. (split2)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_sppcgen.so")
_SO_DEV = os.path.join(_HERE, "_sppcgen_cuda.so")
_lib = None
_lib_dev = None


def _nvcc() -> str | None:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    import shutil
    return shutil.which("nvcc")


def build(force: bool = False) -> str:
    """Compile the generator (portable arithmetic: no FMA contraction) and, when
    the CUDA toolkit is present, its device form (gen_device.cu, explicitly
    rounded IEEE operations, sm_103a)."""
    src = os.path.join(_HERE, "gen.cpp")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", _SO + ".tmp", src]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    src_dev = os.path.join(_HERE, "gen_device.cu")
    nvcc = _nvcc()
    if nvcc and (force or not os.path.exists(_SO_DEV) or os.path.getmtime(_SO_DEV) < os.path.getmtime(src_dev)):
        cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-fmad=false",
               "-Xcompiler", "-fPIC", "-shared", "-o", _SO_DEV + ".tmp", src_dev]
        subprocess.run(cmd, check=True)
        os.replace(_SO_DEV + ".tmp", _SO_DEV)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.sppcgen_build.restype = ctypes.c_void_p
        lib.sppcgen_build.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_uint64, ctypes.c_int32]
        lib.sppcgen_n.restype = ctypes.c_int64
        lib.sppcgen_n.argtypes = [ctypes.c_void_p]
        lib.sppcgen_nnz.restype = ctypes.c_int64
        lib.sppcgen_nnz.argtypes = [ctypes.c_void_p]
        lib.sppcgen_copy.restype = ctypes.c_int32
        lib.sppcgen_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.sppcgen_free.restype = None
        lib.sppcgen_free.argtypes = [ctypes.c_void_p]
        lib.sppcgen_log.restype = ctypes.c_double
        lib.sppcgen_log.argtypes = [ctypes.c_double]
        lib.sppcgen_cos2pi.restype = ctypes.c_double
        lib.sppcgen_cos2pi.argtypes = [ctypes.c_double]
        lib.sppcgen_sm64.restype = ctypes.c_uint64
        lib.sppcgen_sm64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        _lib = lib
    return _lib


def level_sizes_geometric(n: int, n_levels: int, ratio: float) -> list[int]:
    """Level sizes growing by ``ratio`` per level and summing exactly to n.

    Cumulative rounding: S_i = round(n (r^(i+1) - 1) / (r^L - 1)), size_i =
    S_i - S_(i-1).  For n = 2,000,000, 7 levels, ratio 2.2 this gives
    9,660 / 21,253 / 46,757 / 102,864 / 226,302 / 497,864 / 1,095,300.
    """
    pw = [1.0]
    for _ in range(n_levels):
        pw.append(pw[-1] * ratio)
    total = pw[n_levels] - 1.0
    cum = [int(round(n * (pw[i + 1] - 1.0) / total)) for i in range(n_levels)]
    cum[-1] = n
    sizes = [cum[0]] + [cum[i] - cum[i - 1] for i in range(1, n_levels)]
    assert sum(sizes) == n and min(sizes) > 0
    return sizes


@dataclass
class Workload:
    """One synthetic eigenproblem: level partition, value law, k, seed."""
    name: str
    level_sizes: list[int]
    nnz_per_row: int
    k: int
    seed: int = 0
    sigma: float = 0.5
    n1: int | None = None          # small-space size (defaults to level 0)
    orders: int | None = None      # fixed number of correction orders, if any
    p_max: int = 15
    tol: float = 1e-6
    value_dtype: str = "f64"
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(sum(self.level_sizes))

    @property
    def level_offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.level_sizes)]).astype(np.int64)

    @property
    def small_dim(self) -> int:
        return int(self.n1 if self.n1 is not None else self.level_sizes[0])

    @property
    def draws_per_row(self) -> int:
        return int(round(self.nnz_per_row / 2))


def config(name: str) -> Workload:
    """The named synthetic workloads.

    c1: n = 20,000 in 5 levels (2k/3k/4k/5k/6k), n1 = 2,000, ~50 nnz/row, k = 5,
        two correction orders.
    c2: n = 2,000,000 in 7 levels growing x2.2, n1 = level 0 = 9,660, ~200 nnz/row,
        k = 8, stop at scaled residual 1e-6 or 15 orders.
    c3: n = 20,000,000 in 9 levels x2.2, ~250 nnz/row, k = 8 (mixed precision).
    c5train: n = 50,000 in 7 levels x2.2 (training matrices for the learned proposal).
    small: n = 3,000 in 4 levels, for quick tests.
    c2lite: c2's levels at ~60 nnz/row (1.2e8 entries, 1.45 GB): larger than L2
        but small enough for multi-pass profiler captures.
    """
    if name == "c1":
        return Workload("c1", [2000, 3000, 4000, 5000, 6000], 50, 5, seed=0, orders=2)
    if name == "c2":
        return Workload("c2", level_sizes_geometric(2_000_000, 7, 2.2), 200, 8, seed=0)
    if name == "c3":
        return Workload("c3", level_sizes_geometric(20_000_000, 9, 2.2), 250, 8, seed=0, value_dtype="f32")
    if name == "c5train":
        return Workload("c5train", level_sizes_geometric(50_000, 7, 2.2), 200, 8, seed=1)
    if name == "small":
        return Workload("small", [300, 500, 900, 1300], 40, 4, seed=7)
    if name == "c2lite":
        return Workload("c2lite", level_sizes_geometric(2_000_000, 7, 2.2), 60, 8, seed=0)
    if name == "c2mini":
        # c2's law at 1/40 of the size (oracle-friendly, spans many tiles)
        return Workload("c2mini", level_sizes_geometric(50_000, 7, 2.2), 200, 8, seed=3)
    raise KeyError(name)


def c4_batch(count: int = 64, seed: int = 0) -> list[Workload]:
    """Batched workload: `count` matrices, n log-uniform in [5e3, 2e5], 3-6 levels
    growing x2.2, ~80 nnz/row, k = 4, per-matrix seeds seed..seed+count-1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for m in range(count):
        n = int(round(float(np.exp(rng.uniform(np.log(5e3), np.log(2e5))))))
        L = int(rng.integers(3, 7))
        out.append(Workload(f"c4_{m}", level_sizes_geometric(n, L, 2.2), 80, 4, seed=seed + m))
    return out


def generate(w: Workload, threads: int = 0):
    """Return (row_ptr int64[n+1], col int32[nnz], val float64[nnz]) for workload w."""
    lib = _load()
    sizes = (ctypes.c_int64 * len(w.level_sizes))(*w.level_sizes)
    h = lib.sppcgen_build(sizes, len(w.level_sizes), w.draws_per_row, float(w.sigma),
                          ctypes.c_uint64(w.seed & 0xFFFFFFFFFFFFFFFF), int(threads))
    if not h:
        raise MemoryError("generator failed (bad sizes or out of memory)")
    try:
        n = lib.sppcgen_n(h)
        nnz = lib.sppcgen_nnz(h)
        row_ptr = np.empty(n + 1, dtype=np.int64)
        col = np.empty(nnz, dtype=np.int32)
        val = np.empty(nnz, dtype=np.float64)
        lib.sppcgen_copy(h, row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data)
    finally:
        lib.sppcgen_free(h)
    return row_ptr, col, val


def _load_dev():
    global _lib_dev
    if _lib_dev is None:
        build()
        lib = ctypes.CDLL(_SO_DEV)
        lib.sppcgen_dev_build.restype = ctypes.c_void_p
        lib.sppcgen_dev_build.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p]
        lib.sppcgen_dev_n.restype = ctypes.c_int64
        lib.sppcgen_dev_n.argtypes = [ctypes.c_void_p]
        lib.sppcgen_dev_nnz.restype = ctypes.c_int64
        lib.sppcgen_dev_nnz.argtypes = [ctypes.c_void_p]
        lib.sppcgen_dev_fill.restype = ctypes.c_int32
        lib.sppcgen_dev_fill.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_void_p]
        lib.sppcgen_dev_free.restype = None
        lib.sppcgen_dev_free.argtypes = [ctypes.c_void_p]
        _lib_dev = lib
    return _lib_dev


def generate_device(w: Workload):
    """The matrix of generate(w), built on the current CUDA device without a host
    copy (bit-identical to the host generator).  Returns torch CUDA tensors
    (row_ptr int64[n+1], col int32[nnz], val float64[nnz])."""
    import torch
    lib = _load_dev()
    sizes = (ctypes.c_int64 * len(w.level_sizes))(*w.level_sizes)
    stream = torch.cuda.current_stream().cuda_stream
    h = lib.sppcgen_dev_build(sizes, len(w.level_sizes), w.draws_per_row, float(w.sigma),
                              ctypes.c_uint64(w.seed & 0xFFFFFFFFFFFFFFFF), stream)
    if not h:
        raise MemoryError("device generator failed (bad sizes, a CUDA error or out of device memory)")
    try:
        n = lib.sppcgen_dev_n(h)
        nnz = lib.sppcgen_dev_nnz(h)
        row_ptr = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        val = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
        if lib.sppcgen_dev_fill(h, row_ptr.data_ptr(), col.data_ptr(), val.data_ptr(), stream) != 0:
            raise RuntimeError("device generator: fill failed")
    finally:
        lib.sppcgen_dev_free(h)
    return row_ptr, col[:nnz], val[:nnz]


def random_block(n: int, k: int, seed: int) -> np.ndarray:
    """Seeded standard-normal block, row-major n x k, FP64 (numpy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n, k))


def portable_log(x: float) -> float:
    return _load().sppcgen_log(float(x))


def portable_cos2pi(u: float) -> float:
    return _load().sppcgen_cos2pi(float(u))


def splitmix64_at(seed: int, n: int) -> int:
    return int(_load().sppcgen_sm64(seed & 0xFFFFFFFFFFFFFFFF, n & 0xFFFFFFFFFFFFFFFF))
