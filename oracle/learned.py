"""Learned correction proposal: plain FP64 reference (test infrastructure only).

Not part of the paper.  A small per-row network proposes, for each of the k
lowest Ritz pairs (theta_j, z_j) with residual r_j = H z_j - theta_j z_j, a
correction vector that enters the Rayleigh-Ritz subspace of the block
continuation (the paper's Sec. 5-6 switch to a second eigensolver after SPPC
stagnates).  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
legs may import this module.

Definitions (row i, pair j; n rows; level(i) the index of the level holding i):

features   f0 = H_ii, f1 = level(i), f2 = ||H_i,:||_2 (the whole row),
           f3 = rhat_ij = r_ij sqrt(n) / ||r_j||, f4 = theta_j,
           f5 = (|H| |rhat_j|)_i (one SpMV with the entrywise absolute values);
           x = (f - mu) / sd with per-feature mean and spread of the training set.
network    h1 = gelu(W1 x + b1) (64), h2 = gelu(W2 h1 + b2) (64),
           m = w3 . h2 + b3; gelu(a) = a/2 (1 + tanh(sqrt(2/pi) (a + 0.044715 a^3)))
           (the tanh form of Hendrycks and Gimpel, 2016).
proposal   den_ij = H_ii - theta_j with |den| clamped to >= clamp (the shifted
           diagonal of the Jacobi preconditioner, Davidson 1975);
           g_ij = (r_ij / den_ij) (1 + m_ij): the network predicts a relative
           correction to the diagonally preconditioned residual.
target     the exact correction of pair j is t_j = psi_j / (z_j^T psi_j) - z_j
           (psi_j the converged eigenvector; t_j is orthogonal to z_j, the
           Jacobi-Davidson normalisation, Sleijpen and van der Vorst 1996).
           Since the Jacobi-Davidson correction is approximately
           -(diag(H) - theta_j)^-1 r_j, the regression target in the scale of
           rhat is y_ij = -den_ij t_ij sqrt(n) / ||r_j||, and the loss is
           L = mean over samples of (rhat (1 + m) - y)^2.
samples    a training sample is (x, rhat, y) for row i >= n1 and pair j; a pair whose
           Ritz vector is far from its eigenvector (|z_j^T psi_j| < 1/2: the
           Ritz value approximates another eigenvalue, so t_j is meaningless and
           huge) gets rhat = y = 0, which makes its loss and gradient zero.
keep rule  after the Rayleigh-Ritz step on the extended basis the proposal is
           kept iff the largest scaled residual ||r_j|| / |theta_j| dropped;
           otherwise the step is redone with the plain preconditioned block.
parameters one flat vector: W1 (64 x 6, row-major), b1 (64), W2 (64 x 64,
           row-major, W2[o, i]), b2 (64), w3 (64), b3 (1): 4,673 values.
training   Adam (Kingma and Ba, 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

NF, NH = 6, 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + NH * NF
OFF_W2 = OFF_B1 + NH
OFF_B2 = OFF_W2 + NH * NH
OFF_W3 = OFF_B2 + NH
OFF_B3 = OFF_W3 + NH
NPARAM = OFF_B3 + 1
_C = np.sqrt(2.0 / np.pi)


def unpack(params: np.ndarray):
    p = np.asarray(params, dtype=np.float64)
    assert p.shape == (NPARAM,)
    return (p[OFF_W1:OFF_B1].reshape(NH, NF), p[OFF_B1:OFF_W2], p[OFF_W2:OFF_B2].reshape(NH, NH),
            p[OFF_B2:OFF_W3], p[OFF_W3:OFF_B3], p[OFF_B3])


def pack(W1, b1, W2, b2, w3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def init_params(seed: int) -> np.ndarray:
    """Seeded start: weights uniform in +-1/sqrt(fan_in) (PyTorch's default law),
    biases zero, output layer zero (the proposal starts as the Jacobi block)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.uniform(-1, 1, (NH, NF)) / np.sqrt(NF)
    W2 = rng.uniform(-1, 1, (NH, NH)) / np.sqrt(NH)
    return pack(W1, np.zeros(NH), W2, np.zeros(NH), np.zeros(NH), 0.0)


def gelu(a):
    return 0.5 * a * (1.0 + np.tanh(_C * (a + 0.044715 * a ** 3)))


def gelu_grad(a):
    u = _C * (a + 0.044715 * a ** 3)
    th = np.tanh(u)
    return 0.5 * (1.0 + th) + 0.5 * a * (1.0 - th * th) * _C * (1.0 + 3 * 0.044715 * a * a)


def _csr(row_ptr, col, val):
    n = row_ptr.shape[0] - 1
    return sp.csr_matrix((val, col, row_ptr), shape=(n, n))


def row_constants(row_ptr, col, val, level_offsets):
    """(H_ii, level(i), ||H_i,:||_2) for every row."""
    n = row_ptr.shape[0] - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    diag = np.zeros(n)
    on = rows == col
    diag[rows[on]] = val[on]
    level = np.zeros(n)
    for lv in range(len(level_offsets) - 1):
        level[level_offsets[lv]:level_offsets[lv + 1]] = lv
    rownorm = np.sqrt(np.bincount(rows, weights=val * val, minlength=n))
    return diag, level, rownorm


def features(row_ptr, col, val, level_offsets, R: np.ndarray, theta: np.ndarray):
    """Raw features F (n, k, 6) and rhat (n, k) of the Ritz residual block R."""
    n, k = R.shape
    diag, level, rownorm = row_constants(row_ptr, col, val, level_offsets)
    rhat = R * (np.sqrt(n) / np.linalg.norm(R, axis=0))
    agg = np.abs(_csr(row_ptr, col, val)) @ np.abs(rhat)
    F = np.empty((n, k, NF))
    F[..., 0] = diag[:, None]
    F[..., 1] = level[:, None]
    F[..., 2] = rownorm[:, None]
    F[..., 3] = rhat
    F[..., 4] = np.asarray(theta)[None, :]
    F[..., 5] = agg
    return F, rhat


def standardize(F, mu, sd):
    return (F - np.asarray(mu)) / np.asarray(sd)


def forward(params, X):
    """m for every row of X (..., 6), FP64."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    h1 = gelu(X @ W1.T + b1)
    h2 = gelu(h1 @ W2.T + b2)
    return h2 @ w3 + b3


def loss_and_grad(params, X, rhat, y):
    """L = mean((rhat (1 + m) - y)^2) over the samples (rows of X) and dL/dparams
    by reverse-mode differentiation of the three layers."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    B = X.shape[0]
    a1 = X @ W1.T + b1
    h1 = gelu(a1)
    a2 = h1 @ W2.T + b2
    h2 = gelu(a2)
    m = h2 @ w3 + b3
    e = rhat * (1.0 + m) - y
    L = np.mean(e * e)
    dm = 2.0 * e * rhat / B                      # dL/dm per sample
    gw3 = h2.T @ dm
    gb3 = dm.sum()
    d2 = (dm[:, None] * w3[None, :]) * gelu_grad(a2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * gelu_grad(a1)
    gW1 = d1.T @ X
    gb1 = d1.sum(axis=0)
    return L, pack(gW1, gb1, gW2, gb2, gw3, gb3)


def adam_step(params, mom, vel, grad, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (step number t >= 1); returns new (params, mom, vel)."""
    mom = beta1 * mom + (1.0 - beta1) * grad
    vel = beta2 * vel + (1.0 - beta2) * grad * grad
    mhat = mom / (1.0 - beta1 ** t)
    vhat = vel / (1.0 - beta2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), mom, vel


def round_bf16(x):
    """Nearest BF16 (ties to even) of the FP32 rounding of x, as FP64."""
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def infer_bf16(params, X):
    """BF16 inference: standardized inputs, weights (not biases) and the hidden
    activations rounded to BF16 before each product; sums and biases unrounded."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    x = round_bf16(X)
    h1 = round_bf16(gelu(x @ round_bf16(W1).T + b1))
    h2 = round_bf16(gelu(h1 @ round_bf16(W2).T + b2))
    return h2 @ round_bf16(w3) + b3


def shifted_diag(diag, theta, clamp: float):
    den = np.asarray(diag)[:, None] - np.asarray(theta)[None, :]
    small = np.abs(den) < clamp
    den[small] = np.where(den[small] >= 0, clamp, -clamp)
    return den


def proposal(R, diag, theta, clamp: float, m):
    """g = (R / den) (1 + m), elementwise."""
    return R / shifted_diag(diag, theta, clamp) * (1.0 + m)


def target(psi, Z, R, diag, theta, clamp: float):
    """Regression target y (n, k) from converged eigenvectors psi (n, k) and the
    Ritz vectors Z, residuals R of the current subspace."""
    n = Z.shape[0]
    c = np.sum(Z * psi, axis=0)
    t = psi / c - Z
    return -shifted_diag(diag, theta, clamp) * t * (np.sqrt(n) / np.linalg.norm(R, axis=0))


MIN_OVERLAP = 0.5


def training_pairs(psi, Z, R, diag, theta, clamp: float, rhat):
    """(rhat, y) of the training samples: the target of `target`, both zeroed
    for the pairs with |z_j^T psi_j| < MIN_OVERLAP."""
    ok = np.abs(np.sum(Z * psi, axis=0)) >= MIN_OVERLAP
    y = target(psi, Z, R, diag, theta, clamp)
    return np.where(ok, rhat, 0.0), np.where(ok, y, 0.0)


def keep(resid_before, resid_after) -> bool:
    return float(np.max(resid_after)) < float(np.max(resid_before))
