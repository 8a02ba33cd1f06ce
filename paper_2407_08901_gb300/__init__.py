"""GB300 (sm_103a) SPPC eigensolver: thin Python binding of libsppc.so.

Every function here has the name of the C entry point it wraps (declared in
include/sppc.h) and only marshals arguments: all computation runs in the CUDA
kernels of the library.  Importing the package loads libsppc.so and raises
ImportError if it has not been built (``__graft_entry__.build()``); there is no
fallback.  PyTorch is used only for device buffers and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

__all__ = [
    "SppcError", "sppc_default_opts", "sppc_create", "sppc_spmm", "sppc_spmm_noalloc", "sppc_spmm_host", "sppc_start", "sppc_correct",
    "sppc_rayleigh_ritz", "sppc_refine_step", "sppc_solve", "sppc_order_info", "sppc_get_stats", "sppc_get_state", "sppc_get_layout",
    "sppc_destroy", "sppc_last_error", "sppc_kernel_launches", "sppc_small_syev", "sppc_block_gram", "sppc_block_update",
    "sppc_set_proposal", "sppc_proposal_samples", "sppc_mlp_forward", "sppc_mlp_loss_grad", "sppc_mlp_adam",
    "sppc_mlp_train_epoch", "sppc_feature_moments", "sppc_standardize", "sppc_solve_batch", "sppc_spmm_tiling",
    "sppc_sell_sigma", "sppc_spmm_batch_plan", "sppc_spmm_batch_run", "sppc_spmm_batch_destroy",
    "EXPORTED_SYMBOLS", "STATUS",
]

STATUS = {0: "SPPC_OK", 1: "SPPC_ERR_ARG", 2: "SPPC_ERR_NOT_SYMMETRIC", 3: "SPPC_ERR_LEVELS", 4: "SPPC_ERR_OOM",
          5: "SPPC_ERR_CUDA", 6: "SPPC_ERR_BREAKDOWN", 7: "SPPC_ERR_MINRES", 8: "SPPC_ERR_TIMEOUT",
          9: "SPPC_NOT_CONVERGED", 10: "SPPC_ERR_STATE", 11: "SPPC_ERR_NAN"}
SPPC_OK = 0
SPPC_NOT_CONVERGED = 9
SLICE_H = 16  # rows per SELL slice of the device layout


class SppcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("p_max", ctypes.c_int32), ("tol", ctypes.c_double), ("minres_tol", ctypes.c_double),
                ("minres_maxit", ctypes.c_int32), ("small_tol", ctypes.c_double), ("small_block", ctypes.c_int32),
                ("degeneracy_tol", ctypes.c_double), ("check_symmetry", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("timing", ctypes.c_int32), ("spmm_chunk_cols", ctypes.c_int64),
                ("hybrid", ctypes.c_int32), ("switch_order", ctypes.c_int32), ("hybrid_maxit", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("precond_clamp", ctypes.c_double), ("hybrid_blocks", ctypes.c_int32),
                ("spmm_kernel", ctypes.c_int32), ("reorth", ctypes.c_int32), ("precond_iters", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("proposal", ctypes.c_int32), ("precond_levels", ctypes.c_int32),
                ("minres_deflate", ctypes.c_int32), ("small_degree", ctypes.c_int32),
                ("switch_stall", ctypes.c_double), ("minres_ctas", ctypes.c_int32),
                ("spin_cap", ctypes.c_int32), ("value_rounding", ctypes.c_int32), ("minres_fp32", ctypes.c_int32),
                ("minres_fp32_tol", ctypes.c_double), ("tensor_gram", ctypes.c_int32),
                ("sell_sigma", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("orders", ctypes.c_int32), ("converged", ctypes.c_int32), ("spmv_h", ctypes.c_int64),
                ("spmv_h11", ctypes.c_int64), ("minres_iters", ctypes.c_int64), ("small_eig_iters", ctypes.c_int64),
                ("spmm_launches", ctypes.c_int32), ("spmm_ms", ctypes.c_double), ("minres_ms", ctypes.c_double),
                ("small_eig_ms", ctypes.c_double), ("dense_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("refine_steps", ctypes.c_int32), ("restarts", ctypes.c_int32), ("switched_at", ctypes.c_int32),
                ("reorth_passes", ctypes.c_int32), ("refine_df", ctypes.c_int32),
                ("proposals_tried", ctypes.c_int32), ("proposals_kept", ctypes.c_int32),
                ("small_filter_retries", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_VP = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "sppc_default_opts": (None, [ctypes.POINTER(Opts)]),
    "sppc_create": (_I32, [ctypes.POINTER(Csr), _VP, _I32, _I64, _I32, ctypes.POINTER(Opts), _VP,
                           ctypes.POINTER(_VP)]),
    "sppc_spmm": (_I32, [_VP, _VP, _I64, _VP, _I64, _I32, _VP]),
    "sppc_spmm_host": (_I32, [_VP, _VP, _I64, _VP, _I64, _I32, _VP]),
    "sppc_spmm_noalloc": (_I32, [_VP, _VP, _I64, _VP, _I64, _I32, _VP]),
    "sppc_start": (_I32, [_VP, _VP, _VP, _VP]),
    "sppc_correct": (_I32, [_VP, _VP]),
    "sppc_rayleigh_ritz": (_I32, [_VP, _VP, _VP, _VP]),
    "sppc_solve": (_I32, [_VP, _D, _I32, _VP, _VP, _I64, _VP, ctypes.POINTER(Stats), _VP]),
    "sppc_refine_step": (_I32, [_VP, _VP, _VP, _VP]),
    "sppc_order_info": (_I32, [_VP, _I32, _VP, _VP, _VP, _VP, _VP]),
    "sppc_get_stats": (_I32, [_VP, ctypes.POINTER(Stats)]),
    "sppc_get_state": (_I32, [_VP, _I32, _VP, _I64]),
    "sppc_get_layout": (_I32, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "sppc_destroy": (_I32, [_VP]),
    "sppc_last_error": (ctypes.c_char_p, [_VP]),
    "sppc_kernel_launches": (_I64, []),
    "sppc_small_syev": (_I32, [_VP, _I32, _I32, _I32, _VP, _VP, _I32, _I32, _VP]),
    "sppc_block_gram": (_I32, [_VP, _I32, _VP, _I64, _I32, _VP, _VP]),
    "sppc_block_update": (_I32, [_VP, _I32, _VP, _VP, _VP, _VP, _I64, _I32, _VP]),
    "sppc_set_proposal": (_I32, [_VP, _VP, _VP, _VP]),
    "sppc_proposal_samples": (_I32, [_VP, _VP, _I64, _VP, _VP, _VP, _VP, _VP]),
    "sppc_mlp_forward": (_I32, [_VP, _VP, _I64, _I32, _VP, _VP]),
    "sppc_mlp_loss_grad": (_I32, [_VP, _VP, _VP, _VP, _I64, _VP, _VP, _VP]),
    "sppc_mlp_adam": (_I32, [_VP, _VP, _VP, _VP, _I32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, _VP]),
    "sppc_mlp_train_epoch": (_I32, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I64, _I32, _VP, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, ctypes.c_float, _VP, _VP]),
    "sppc_feature_moments": (_I32, [_VP, _I64, _VP, _VP, _VP]),
    "sppc_standardize": (_I32, [_VP, _I64, _VP, _VP, _VP, _VP]),
    "sppc_solve_batch": (_I32, [_VP, _I32, _D, _I32, _I32, _VP, _VP, _VP, _VP]),
    "sppc_spmm_tiling": (_I32, [_VP, _VP, _VP]),
    "sppc_sell_sigma": (_I32, [_VP, _VP, _VP]),
    "sppc_spmm_batch_plan": (_I32, [_VP, _I32, _VP, _VP, _I32, ctypes.POINTER(_VP)]),
    "sppc_spmm_batch_run": (_I32, [_VP, _VP]),
    "sppc_spmm_batch_destroy": (_I32, [_VP]),
}
NET_PARAMS, NET_FEATURES = 4673, 6
EXPORTED_SYMBOLS = tuple(_SIGS)


def _load():
    if not os.path.exists(LIB):
        raise ImportError(f"{LIB} is missing: build it with __graft_entry__.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (contiguity is the caller's duty)."""
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(h, st: int, allow=(SPPC_OK,)):
    if st not in allow:
        msg = _lib.sppc_last_error(h)
        raise SppcError(st, msg.decode() if msg else "")
    return st


def sppc_last_error(h=None) -> str:
    m = _lib.sppc_last_error(h)
    return m.decode() if m else ""


def sppc_default_opts(**overrides) -> Opts:
    o = Opts()
    _lib.sppc_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def sppc_create(row_ptr, col, val, level_offsets, n1: int, k: int, opts: Opts | None = None, stream=None,
                on_device: bool = False):
    """Create a handle for the CSR matrix (int64 row_ptr, int32 col, float64 val).

    Host numpy arrays (on_device=False) or torch CUDA tensors (on_device=True)."""
    n = int(row_ptr.shape[0]) - 1
    csr = Csr(n, int(col.shape[0]), _ptr(row_ptr), _ptr(col), _ptr(val), 1 if on_device else 0)
    lev = np.ascontiguousarray(level_offsets, dtype=np.int64)
    h = ctypes.c_void_p()
    st = _lib.sppc_create(ctypes.byref(csr), lev.ctypes.data, len(lev) - 1, int(n1), int(k),
                          ctypes.byref(opts) if opts is not None else None, _stream(stream), ctypes.byref(h))
    _check(None, st)
    return h


def sppc_spmm(h, X, Y, stream=None) -> None:
    """Y = H X for torch CUDA float64 tensors X, Y of shape (n, ncols), ncols <= 8."""
    assert X.dtype == Y.dtype and X.is_cuda and Y.is_cuda and X.stride(1) == 1 and Y.stride(1) == 1
    _check(h, _lib.sppc_spmm(h, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0), X.shape[1], _stream(stream)))


def sppc_spmm_noalloc(h, X, Y, stream=None) -> None:
    """Y = H X like sppc_spmm, without allocating device memory in the call (the
    scratch lives in a fixed 32 MiB device array; n * kp <= 2,097,152)."""
    assert X.dtype == Y.dtype and X.is_cuda and Y.is_cuda and X.stride(1) == 1 and Y.stride(1) == 1
    _check(h, _lib.sppc_spmm_noalloc(h, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0), X.shape[1], _stream(stream)))


def sppc_spmm_host(h, X: np.ndarray, Y: np.ndarray, stream=None) -> None:
    """Y = H X for host float64 arrays (copies inside the call)."""
    assert X.flags.c_contiguous and Y.flags.c_contiguous
    _check(h, _lib.sppc_spmm_host(h, _ptr(X), X.shape[1], _ptr(Y), Y.shape[1], X.shape[1], _stream(stream)))


def sppc_start(h, k: int, stream=None):
    th, rs = np.zeros(k), np.zeros(k)
    _check(h, _lib.sppc_start(h, th.ctypes.data, rs.ctypes.data, _stream(stream)))
    return th, rs


def sppc_correct(h, stream=None) -> None:
    _check(h, _lib.sppc_correct(h, _stream(stream)))


def sppc_rayleigh_ritz(h, k: int, stream=None):
    th, rs = np.zeros(k), np.zeros(k)
    _check(h, _lib.sppc_rayleigh_ritz(h, th.ctypes.data, rs.ctypes.data, _stream(stream)))
    return th, rs


def sppc_refine_step(h, k: int, stream=None):
    th, rs = np.zeros(k), np.zeros(k)
    _check(h, _lib.sppc_refine_step(h, th.ctypes.data, rs.ctypes.data, _stream(stream)))
    return th, rs


def sppc_solve(h, k: int, tol: float = -1.0, p_max: int = -1, Z=None, stream=None):
    """Algorithm 2 end to end.  Z: optional torch CUDA float64 tensor (n, >=k).

    Returns (converged, theta, resid, stats dict)."""
    th, rs = np.zeros(k), np.zeros(k)
    stats = Stats()
    ldz = Z.stride(0) if Z is not None else 0
    st = _lib.sppc_solve(h, float(tol), int(p_max), th.ctypes.data, _ptr(Z), ldz, rs.ctypes.data,
                         ctypes.byref(stats), _stream(stream))
    _check(h, st, allow=(SPPC_OK, SPPC_NOT_CONVERGED))
    return st == SPPC_OK, th, rs, stats.as_dict()


def sppc_order_info(h, p: int, k: int) -> dict:
    E, ang, th, rs = (np.zeros(k) for _ in range(4))
    it = np.zeros(k, dtype=np.int32)
    _check(h, _lib.sppc_order_info(h, int(p), E.ctypes.data, ang.ctypes.data, th.ctypes.data, rs.ctypes.data,
                                   it.ctypes.data))
    return {"E": E, "angle": ang, "theta": th, "resid": rs, "minres_iters": it}


def sppc_get_stats(h) -> dict:
    s = Stats()
    _check(h, _lib.sppc_get_stats(h, ctypes.byref(s)))
    return s.as_dict()


def sppc_get_state(h, which: int, shape) -> np.ndarray:
    out = np.zeros(shape)
    _check(h, _lib.sppc_get_state(h, int(which), out.ctypes.data, out.size))
    return out


def sppc_get_layout(h) -> dict:
    ns, n11, nch = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(h, _lib.sppc_get_layout(h, ctypes.byref(ns), None, None, ctypes.byref(n11), None, None,
                                   ctypes.byref(nch), None))
    sp = np.zeros(ns.value + 1, dtype=np.int64)
    sr = np.zeros(SLICE_H * ns.value, dtype=np.int32)
    sp11 = np.zeros(n11.value + 1, dtype=np.int64)
    sr11 = np.zeros(SLICE_H * n11.value, dtype=np.int32)
    cs = np.zeros(nch.value + 1, dtype=np.int64)
    _check(h, _lib.sppc_get_layout(h, None, sp.ctypes.data, sr.ctypes.data, None, sp11.ctypes.data,
                                   sr11.ctypes.data, None, cs.ctypes.data))
    return {"slice_ptr": sp, "slice_rows": sr, "h11_slice_ptr": sp11, "h11_slice_rows": sr11,
            "n_chunks": nch.value, "chunk_slice": cs}


def sppc_kernel_launches() -> int:
    return int(_lib.sppc_kernel_launches())


def sppc_small_syev(S, nev: int, f64: bool = False, stream=None):
    """nev lowest eigenpairs of the symmetric m x m torch CUDA float64 tensor S
    (m <= 144, nev <= 16); returns (theta, V) as CUDA tensors (V: m x nev).
    f64: Householder steps in FP64 instead of double-float."""
    import torch
    S = S.contiguous()
    m = int(S.shape[0])
    theta = torch.empty(nev, dtype=torch.float64, device=S.device)
    V = torch.empty(m, nev, dtype=torch.float64, device=S.device)
    _check(None, _lib.sppc_small_syev(S.data_ptr(), m, m, int(nev), theta.data_ptr(), V.data_ptr(), int(nev),
                                      1 if f64 else 0, _stream(stream)))
    return theta, V


def sppc_block_gram(A, B, tensor: bool = False, df: bool = False, stream=None):
    """G = A^T B for A a torch CUDA float64 tensor (nblocks, n, 8) and B (n, 8):
    returns G (8 nblocks, 8).  tensor: on the tensor cores (|A| < 2 required);
    df: in double-float slots.  Synchronises the stream."""
    import torch
    A = A.contiguous()
    B = B.contiguous()
    nb, n = int(A.shape[0]), int(A.shape[1])
    assert A.dtype == torch.float64 and B.dtype == torch.float64 and A.is_cuda and B.is_cuda
    assert tuple(A.shape) == (nb, n, 8) and tuple(B.shape) == (n, 8)
    G = torch.empty(8 * nb, 8, dtype=torch.float64, device=A.device)
    flags = (1 if tensor else 0) | (2 if df else 0)
    _check(None, _lib.sppc_block_gram(A.data_ptr(), nb, B.data_ptr(), n, flags, G.data_ptr(), _stream(stream)))
    return G


def sppc_block_update(A, C, alpha=None, X=None, Y=None, tensor: bool = False, df: bool = False, stream=None):
    """Y = alpha X + sum_a A_a C_a for A a torch CUDA float64 tensor (nblocks, n, 8),
    C (8 nblocks, 8), alpha (8,) or None, X (n, 8) or None; Y (n, 8) is
    allocated when None (it may be X).  Returns Y.  tensor: on the tensor cores
    (|A| < 2 required); df: in double-float slots.  Synchronises the stream."""
    import torch
    A = A.contiguous()
    nb, n = int(A.shape[0]), int(A.shape[1])
    C = C.contiguous()
    assert A.dtype == torch.float64 and C.dtype == torch.float64 and tuple(C.shape) == (8 * nb, 8)
    if Y is None:
        Y = torch.empty(n, 8, dtype=torch.float64, device=A.device)
    flags = (1 if tensor else 0) | (2 if df else 0)
    _check(None, _lib.sppc_block_update(A.data_ptr(), nb, C.data_ptr(), alpha.data_ptr() if alpha is not None else None,
                                        X.data_ptr() if X is not None else None, Y.data_ptr(), n, flags,
                                        _stream(stream)))
    return Y


def _f32_dev(t, n=None):
    assert t.is_cuda and t.dtype.is_floating_point and t.is_contiguous(), "contiguous CUDA tensor expected"
    if n is not None:
        assert t.numel() >= n
    return t.data_ptr()


def sppc_set_proposal(h, params: np.ndarray, mu: np.ndarray, sd: np.ndarray) -> None:
    """Install a trained proposal network (host float32 arrays)."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    m = np.ascontiguousarray(mu, dtype=np.float32)
    d = np.ascontiguousarray(sd, dtype=np.float32)
    assert p.size == NET_PARAMS and m.size == NET_FEATURES and d.size == NET_FEATURES
    _check(h, _lib.sppc_set_proposal(h, p.ctypes.data, m.ctypes.data, d.ctypes.data))


def sppc_proposal_samples(h, psi, F, rhat, y, stream=None) -> int:
    """Training samples of the current Rayleigh-Ritz state against exact
    eigenvectors psi (CUDA float64 (n, >=k)); F (count x 6), rhat, y CUDA float32."""
    assert psi.is_cuda and psi.dtype.__str__() == "torch.float64" and psi.stride(1) == 1
    cnt = ctypes.c_int64()
    _check(h, _lib.sppc_proposal_samples(h, psi.data_ptr(), psi.stride(0), _f32_dev(F), _f32_dev(rhat), _f32_dev(y),
                                         ctypes.byref(cnt), _stream(stream)))
    return int(cnt.value)


def sppc_mlp_forward(params, X, out, bf16: bool = False, stream=None) -> None:
    n = int(X.shape[0])
    _check(None, _lib.sppc_mlp_forward(_f32_dev(params, NET_PARAMS), _f32_dev(X, 6 * n), n, 1 if bf16 else 0,
                                       _f32_dev(out, n), _stream(stream)))


def sppc_mlp_loss_grad(params, X, rhat, y, grad, loss, stream=None) -> None:
    n = int(X.shape[0])
    _check(None, _lib.sppc_mlp_loss_grad(_f32_dev(params, NET_PARAMS), _f32_dev(X, 6 * n), _f32_dev(rhat, n),
                                         _f32_dev(y, n), n, _f32_dev(grad, NET_PARAMS), _f32_dev(loss, 1),
                                         _stream(stream)))


def sppc_mlp_adam(params, mom, vel, grad, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                  eps: float = 1e-8, stream=None) -> None:
    _check(None, _lib.sppc_mlp_adam(_f32_dev(params, NET_PARAMS), _f32_dev(mom, NET_PARAMS),
                                    _f32_dev(vel, NET_PARAMS), _f32_dev(grad, NET_PARAMS), int(t), float(lr),
                                    float(beta1), float(beta2), float(eps), _stream(stream)))


def sppc_mlp_train_epoch(params, mom, vel, X, rhat, y, perm, batch: int, step: int, lr: float,
                         beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None):
    """One epoch of minibatch Adam; perm: CUDA int64 order of the samples or None.
    Returns (new step count, mean batch loss)."""
    n = int(X.shape[0])
    st = ctypes.c_int32(int(step))
    loss = ctypes.c_double()
    pp = 0
    if perm is not None:
        assert perm.is_cuda and str(perm.dtype) == "torch.int64" and perm.numel() >= n
        pp = perm.data_ptr()
    _check(None, _lib.sppc_mlp_train_epoch(_f32_dev(params, NET_PARAMS), _f32_dev(mom, NET_PARAMS),
                                           _f32_dev(vel, NET_PARAMS), _f32_dev(X, 6 * n), _f32_dev(rhat, n),
                                           _f32_dev(y, n), pp, n, int(batch), ctypes.byref(st), float(lr),
                                           float(beta1), float(beta2), float(eps), ctypes.byref(loss),
                                           _stream(stream)))
    return int(st.value), float(loss.value)


def sppc_feature_moments(F, stream=None):
    n = int(F.shape[0])
    mean, sd = np.zeros(6), np.zeros(6)
    _check(None, _lib.sppc_feature_moments(_f32_dev(F, 6 * n), n, mean.ctypes.data, sd.ctypes.data, _stream(stream)))
    return mean, sd


def sppc_standardize(F, mu, sd, X, stream=None) -> None:
    n = int(F.shape[0])
    m = np.ascontiguousarray(mu, dtype=np.float32)
    d = np.ascontiguousarray(sd, dtype=np.float32)
    _check(None, _lib.sppc_standardize(_f32_dev(F, 6 * n), n, m.ctypes.data, d.ctypes.data, _f32_dev(X, 6 * n),
                                       _stream(stream)))


def sppc_solve_batch(handles, kmax: int, tol: float = -1.0, workers: int = 8):
    """Solve independent problems concurrently (see include/sppc.h).  Returns
    (status, theta (count x kmax), resid (count x kmax), converged (count), stats list)."""
    count = len(handles)
    arr = (ctypes.c_void_p * count)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    th = np.zeros((count, kmax))
    rs = np.zeros((count, kmax))
    cv = np.zeros(count, dtype=np.int32)
    st = (Stats * count)()
    status = _lib.sppc_solve_batch(ctypes.cast(arr, ctypes.c_void_p), count, float(tol), int(workers), int(kmax),
                                   th.ctypes.data, rs.ctypes.data, cv.ctypes.data, ctypes.cast(st, ctypes.c_void_p))
    _check(None, status, allow=(SPPC_OK, SPPC_NOT_CONVERGED))
    return status, th, rs, cv.astype(bool), [s.as_dict() for s in st]


def sppc_spmm_tiling(h):
    """(column tile of H's layout, -1 untiled; autotuner's ms per product of the candidates tried)."""
    cc = ctypes.c_int64()
    ms = np.zeros(5)
    _check(h, _lib.sppc_spmm_tiling(h, ctypes.byref(cc), ms.ctypes.data))
    return int(cc.value), ms


def sppc_sell_sigma(h):
    """(sort window of H's layout; autotuner's ms per product at windows 64, 256, 1024, zeros if not tuned)."""
    sg = ctypes.c_int32()
    ms = np.zeros(3)
    _check(h, _lib.sppc_sell_sigma(h, ctypes.byref(sg), ms.ctypes.data))
    return int(sg.value), ms


def sppc_spmm_batch_plan(handles, Xs, Ys):
    """Plan Y_i = H_i X_i for all handles (CUDA float64 tensors (n_i, ncols), one
    ncols) as one persistent launch captured in a CUDA graph."""
    count = len(handles)
    ncols = int(Xs[0].shape[1])
    for X, Y in zip(Xs, Ys):
        assert X.is_cuda and Y.is_cuda and X.is_contiguous() and Y.is_contiguous()
        assert X.shape[1] == ncols and Y.shape[1] == ncols
    hs = (ctypes.c_void_p * count)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    xs = (ctypes.c_void_p * count)(*[X.data_ptr() for X in Xs])
    ys = (ctypes.c_void_p * count)(*[Y.data_ptr() for Y in Ys])
    plan = ctypes.c_void_p()
    _check(None, _lib.sppc_spmm_batch_plan(ctypes.cast(hs, ctypes.c_void_p), count, ctypes.cast(xs, ctypes.c_void_p),
                                           ctypes.cast(ys, ctypes.c_void_p), ncols, ctypes.byref(plan)))
    return plan


def sppc_spmm_batch_run(plan, stream=None) -> None:
    _check(None, _lib.sppc_spmm_batch_run(plan, _stream(stream)))


def sppc_spmm_batch_destroy(plan) -> None:
    if plan:
        _lib.sppc_spmm_batch_destroy(plan)


def sppc_destroy(h) -> None:
    if h:
        _lib.sppc_destroy(h)
