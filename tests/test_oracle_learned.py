"""Pins of the learned-proposal oracle (oracle/learned.py) against finite
differences, library routines, exact identities and closed forms."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.special import erf

from conftest import dense, make_matrix
from oracle import learned as L


def test_gelu_identities_and_erf_form():
    x = np.linspace(-8, 8, 4001)
    assert L.gelu(0.0) == 0.0
    # tanh is odd, so gelu(x) - gelu(-x) = x exactly in real arithmetic
    assert np.allclose(L.gelu(x) - L.gelu(-x), x, rtol=0, atol=1e-14)
    # the tanh form approximates x Phi(x) to within 1e-3 (Hendrycks and Gimpel)
    exact = 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))
    assert np.max(np.abs(L.gelu(x) - exact)) < 1e-3
    # derivative against central differences
    h = 1e-6
    fd = (L.gelu(x + h) - L.gelu(x - h)) / (2 * h)
    assert np.allclose(L.gelu_grad(x), fd, rtol=1e-7, atol=1e-8)


def _batch(seed, B=64):
    rng = np.random.Generator(np.random.PCG64(seed))
    p = L.init_params(seed)
    p[L.OFF_W3:L.OFF_B3] = rng.standard_normal(L.NH) * 0.3   # non-zero output layer
    p[L.OFF_B3] = 0.2
    p[L.OFF_B1:L.OFF_W2] = rng.standard_normal(L.NH) * 0.1
    p[L.OFF_B2:L.OFF_W3] = rng.standard_normal(L.NH) * 0.1
    X = rng.standard_normal((B, L.NF))
    rhat = rng.standard_normal(B)
    y = rng.standard_normal(B)
    return p, X, rhat, y


def test_gradient_matches_central_differences():
    p, X, rhat, y = _batch(3)
    _, g = L.loss_and_grad(p, X, rhat, y)
    rng = np.random.Generator(np.random.PCG64(5))
    idx = np.concatenate([rng.choice(np.arange(lo, hi), size=min(12, hi - lo), replace=False)
                          for lo, hi in ((L.OFF_W1, L.OFF_B1), (L.OFF_B1, L.OFF_W2), (L.OFF_W2, L.OFF_B2),
                                         (L.OFF_B2, L.OFF_W3), (L.OFF_W3, L.OFF_B3), (L.OFF_B3, L.NPARAM))])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (L.loss_and_grad(pp, X, rhat, y)[0] - L.loss_and_grad(pm, X, rhat, y)[0]) / (2 * h)
        assert abs(g[i] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, g[i], fd)


def test_forward_special_cases():
    p, X, _, _ = _batch(4)
    q = p.copy()
    q[L.OFF_W2:L.OFF_W3] = 0.0          # W2 = 0, b2 = 0: h2 = gelu(0) = 0, m = b3
    assert np.array_equal(L.forward(q, X), np.full(X.shape[0], q[L.OFF_B3]))
    q = p.copy()
    q[L.OFF_W1:L.OFF_B1] = 0.0          # W1 = 0: every sample gives the same m
    m = L.forward(q, X)
    assert np.allclose(m, m[0], rtol=0, atol=1e-15)
    # loss at m = 0 (zero output layer) is mean((rhat - y)^2)
    p0, X0, r0, y0 = _batch(6)
    p0[L.OFF_W3:] = 0.0
    assert np.isclose(L.loss_and_grad(p0, X0, r0, y0)[0], np.mean((r0 - y0) ** 2), rtol=1e-15)


def test_adam_first_step_and_quadratic():
    rng = np.random.Generator(np.random.PCG64(8))
    p = rng.standard_normal(10)
    g = rng.standard_normal(10)
    z = np.zeros(10)
    # first step with bias correction: mhat = g, vhat = g^2, step = lr g / (|g| + eps)
    p1, _, _ = L.adam_step(p, z, z, g, 1, 0.01)
    assert np.allclose(p1, p - 0.01 * np.sign(g), rtol=0, atol=1e-7)
    # minimises 0.5 ||p - a||^2
    a = rng.standard_normal(10)
    q, mo, ve = np.zeros(10), np.zeros(10), np.zeros(10)
    for t in range(1, 3001):
        q, mo, ve = L.adam_step(q, mo, ve, q - a, t, 0.01)
    assert np.allclose(q, a, atol=1e-3)


def test_features_against_library_routines():
    w, rp, c, v = make_matrix("small")
    n = w.n
    H = sp.csr_matrix((v, c, rp), shape=(n, n))
    rng = np.random.Generator(np.random.PCG64(9))
    R = rng.standard_normal((n, 3))
    theta = np.array([-3.0, -2.5, 1.0])
    F, rhat = L.features(rp, c, v, w.level_offsets, R, theta)
    assert np.allclose(F[:, 0, 0], H.diagonal(), rtol=0, atol=0)
    assert np.allclose(F[:, 0, 2], spla.norm(H, axis=1), rtol=1e-14)
    assert np.allclose(np.linalg.norm(rhat, axis=0), np.sqrt(n), rtol=1e-14)
    assert np.allclose(F[..., 5], (abs(H) @ np.abs(rhat)), rtol=1e-14)
    lo = w.level_offsets
    for lv in range(len(lo) - 1):
        assert F[lo[lv], 0, 1] == lv and F[lo[lv + 1] - 1, 0, 1] == lv
    assert np.array_equal(F[0, :, 4], theta)


def test_target_satisfies_the_correction_equation():
    """t = psi / (z^T psi) - z is orthogonal to z and solves the projected
    correction equation (I - z z^T)(H - lambda)(I - z z^T) t = -r exactly, lambda the
    eigenvalue of psi; y = -den t sqrt(n) / ||r|| carries it."""
    w, rp, c, v = make_matrix("small")
    A = dense(rp, c, v)
    n = A.shape[0]
    lam, V = np.linalg.eigh(A)
    k = 3
    rng = np.random.Generator(np.random.PCG64(10))
    Z = V[:, :k] + 1e-3 * rng.standard_normal((n, k))
    Z /= np.linalg.norm(Z, axis=0)
    theta = np.sum(Z * (A @ Z), axis=0)
    R = A @ Z - Z * theta
    diag = np.diag(A).copy()
    y = L.target(V[:, :k], Z, R, diag, theta, 1e-2)
    den = L.shifted_diag(diag, theta, 1e-2)
    t = -y / den * np.linalg.norm(R, axis=0) / np.sqrt(n)
    for j in range(k):
        z = Z[:, j]
        assert abs(z @ t[:, j]) < 1e-12
        P = np.eye(n) - np.outer(z, z)
        lhs = P @ (A - lam[j] * np.eye(n)) @ P @ t[:, j]
        assert np.allclose(lhs, -R[:, j], rtol=0, atol=1e-10 * np.linalg.norm(R[:, j]))
    # exact eigenvectors need no correction (the residual block only sets the scale)
    y0 = L.target(V[:, :k], V[:, :k], np.ones((n, k)), diag, lam[:k], 1e-2)
    assert np.max(np.abs(y0)) < 1e-10


def test_proposal_reduces_to_jacobi_and_clamps():
    R = np.array([[1.0, 2.0], [3.0, -4.0]])
    diag = np.array([5.0, -2.0])
    theta = np.array([-1.0, -2.0])
    g = L.proposal(R, diag, theta, 1e-2, np.zeros((2, 2)))
    assert np.array_equal(g, np.array([[1.0 / 6.0, 2.0 / 7.0], [3.0 / -1.0, -4.0 / 1e-2]]))
    assert np.array_equal(L.proposal(R, diag, theta, 1e-2, np.full((2, 2), 1.0)), 2 * g)


def test_bf16_inference_tracks_fp64_forward():
    p, X, _, _ = _batch(11, B=512)
    m = L.forward(p, X)
    mb = L.infer_bf16(p, X)
    assert np.max(np.abs(mb - m)) < 3e-2 * max(1.0, np.max(np.abs(m)))
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -3.140625])
    assert np.array_equal(L.round_bf16(x), [1.0, 1.0, 1.0 + 2.0 ** -6, -3.140625])


def test_keep_rule():
    assert L.keep([1e-3, 2e-3], [1e-3, 1.5e-3])
    assert not L.keep([1e-3, 2e-3], [1e-4, 2e-3])


def test_training_pairs_zero_unmatched_ritz_vectors():
    w, rp, c, v = make_matrix("small")
    A = dense(rp, c, v)
    n = A.shape[0]
    lam, V = np.linalg.eigh(A)
    Z = V[:, :3].copy()
    Z[:, 2] = V[:, 3]                  # pair 2's Ritz vector is another eigenvector
    theta = np.sum(Z * (A @ Z), axis=0)
    R = A @ Z - Z * theta + 1e-3       # any residual block (sets the scale)
    rhat = R * np.sqrt(n) / np.linalg.norm(R, axis=0)
    rh, y = L.training_pairs(V[:, :3], Z, R, np.diag(A).copy(), theta, 1e-2, rhat)
    assert np.array_equal(rh[:, :2], rhat[:, :2]) and np.all(rh[:, 2] == 0) and np.all(y[:, 2] == 0)
    assert np.array_equal(y[:, :2], L.target(V[:, :3], Z, R, np.diag(A).copy(), theta, 1e-2)[:, :2])


def test_clamp_keeps_the_sign_of_the_shift():
    """|H_ii - theta| below the clamp becomes the clamp with the shift's sign (a
    zero shift counts as positive); larger shifts pass unchanged."""
    diag = np.array([-2.005, -1.995, -2.0, -2.5, 3.0])
    den = L.shifted_diag(diag, np.array([-2.0]), 1e-2)[:, 0]
    assert np.array_equal(den, np.array([-1e-2, 1e-2, 1e-2, -0.5, 5.0]))


def test_bf16_inference_rounds_every_operand_and_activation():
    """Inputs, weights and both hidden activations pass through BF16 before each
    product, so perturbations far below half a BF16 step of any of them (here
    1e-12 relative) leave the result bit-identical, while the unrounded final
    bias still moves it."""
    p, X, _, _ = _batch(11, B=256)
    m0 = L.infer_bf16(p, X)
    W1, b1, W2, b2, w3, b3 = L.unpack(p)
    eps = 1e-12
    cases = {
        "x": (p, X * (1.0 + eps)),
        "W1": (L.pack(W1 * (1.0 + eps), b1, W2, b2, w3, b3), X),
        "b1": (L.pack(W1, b1 + eps, W2, b2, w3, b3), X),
        "W2": (L.pack(W1, b1, W2 * (1.0 + eps), b2, w3, b3), X),
        "b2": (L.pack(W1, b1, W2, b2 + eps, w3, b3), X),
        "w3": (L.pack(W1, b1, W2, b2, w3 * (1.0 + eps), b3), X),
    }
    for name, (pp, XX) in cases.items():
        assert np.array_equal(L.infer_bf16(pp, XX), m0), name
    assert not np.array_equal(L.infer_bf16(L.pack(W1, b1, W2, b2, w3, b3 + 1e-6), X), m0)


def test_bf16_inference_rounds_the_input_and_the_first_activation():
    """Two one-unit networks whose later stages are exact (gelu(a) = a for a >= 8
    in FP64, power-of-two weights) expose where BF16 rounding happens.
    (1) a1 = 1024 (x - 1), a2 = a1 / 8: with x rounded to BF16 (steps of 2^-7
    on [1, 2)) a1 is a multiple of 8 and the output an integer; unrounded x
    gives fractions.  (2) a1 = x in gelu's curved range, a2 = 1024 (h1 - 0.5)
    + 8: with h1 rounded to BF16 (steps of 2^-8 on [0.5, 1)) the output is a
    multiple of 4 and at least 8."""
    rng = np.random.default_rng(5)
    z = np.zeros
    W1, b1, W2, b2, w3 = z((L.NH, L.NF)), z(L.NH), z((L.NH, L.NH)), z(L.NH), z(L.NH)
    W1[0, 0], b1[0], W2[0, 0], w3[0] = 1024.0, -1024.0, 0.125, 1.0
    X = np.zeros((400, L.NF))
    X[:, 0] = rng.uniform(1.07, 1.9, 400)
    m = L.infer_bf16(L.pack(W1, b1, W2, b2, w3, 0.0), X)
    assert np.all(m >= 8) and np.array_equal(m, np.round(m))
    W1, b1, W2, b2 = z((L.NH, L.NF)), z(L.NH), z((L.NH, L.NH)), z(L.NH)
    W1[0, 0], W2[0, 0], b2[0] = 1.0, 1024.0, -504.0
    X[:, 0] = rng.uniform(0.72, 1.1, 400)
    m = L.infer_bf16(L.pack(W1, b1, W2, b2, w3, 0.0), X)
    assert np.all(m >= 8) and np.array_equal(m, 4.0 * np.round(m / 4.0))
