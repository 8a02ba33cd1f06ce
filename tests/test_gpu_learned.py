"""Learned correction proposal on the GPU against the FP64 oracle
(oracle/learned.py): network forward (FP32 and BF16 inference), the minibatch
gradient, Adam, feature moments, training samples (features and exact-correction
targets), the in-solve proposal block, and solves with the proposal switched on."""
import numpy as np
import pytest

import workloads as W
from conftest import dense, make_matrix
from oracle import learned as L
from oracle.sppc import sppc as oracle_sppc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _net(seed, scale_out=0.3):
    rng = np.random.Generator(np.random.PCG64(seed))
    p = L.init_params(seed)
    p[L.OFF_B1:L.OFF_W2] = rng.standard_normal(L.NH) * 0.1
    p[L.OFF_B2:L.OFF_W3] = rng.standard_normal(L.NH) * 0.1
    p[L.OFF_W3:L.OFF_B3] = rng.standard_normal(L.NH) * scale_out
    p[L.OFF_B3] = 0.05
    return p.astype(np.float32).astype(np.float64)


def _cuda32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_forward_fp32_and_bf16_match_the_oracle():
    import paper_2407_08901_gb300 as S
    p = _net(1)
    X = np.random.Generator(np.random.PCG64(2)).standard_normal((3001, 6)).astype(np.float32).astype(np.float64)
    out = torch.empty(3001, dtype=torch.float32, device="cuda")
    S.sppc_mlp_forward(_cuda32(p), _cuda32(X), out, bf16=False)
    torch.cuda.synchronize()
    m = L.forward(p, X)
    scale = max(1.0, float(np.max(np.abs(m))))
    assert np.max(np.abs(out.cpu().numpy() - m)) <= 2e-5 * scale
    S.sppc_mlp_forward(_cuda32(p), _cuda32(X), out, bf16=True)
    torch.cuda.synchronize()
    mb = L.infer_bf16(p, X)
    # tanh.approx (about 2^-11 relative) can flip a BF16 rounding of a hidden unit
    assert np.max(np.abs(out.cpu().numpy() - mb)) <= 2e-2 * scale


@pytest.mark.parametrize("B", [1, 127, 1000, 4096])
def test_gradient_matches_the_oracle(B):
    import paper_2407_08901_gb300 as S
    rng = np.random.Generator(np.random.PCG64(B))
    p = _net(3)
    X = rng.standard_normal((B, 6)).astype(np.float32).astype(np.float64)
    rh = rng.standard_normal(B).astype(np.float32).astype(np.float64)
    y = rng.standard_normal(B).astype(np.float32).astype(np.float64)
    g = torch.empty(L.NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    S.sppc_mlp_loss_grad(_cuda32(p), _cuda32(X), _cuda32(rh), _cuda32(y), g, loss)
    Lr, gr = L.loss_and_grad(p, X, rh, y)
    assert abs(float(loss.item()) - Lr) <= 1e-5 * Lr
    gg = g.cpu().numpy().astype(np.float64)
    for lo, hi in ((L.OFF_W1, L.OFF_B1), (L.OFF_B1, L.OFF_W2), (L.OFF_W2, L.OFF_B2), (L.OFF_B2, L.OFF_W3),
                   (L.OFF_W3, L.OFF_B3), (L.OFF_B3, L.NPARAM)):
        ref = np.linalg.norm(gr[lo:hi])
        assert np.linalg.norm(gg[lo:hi] - gr[lo:hi]) <= 1e-4 * max(ref, 1e-12), (lo, hi)


def test_adam_and_epoch_match_the_oracle():
    import paper_2407_08901_gb300 as S
    rng = np.random.Generator(np.random.PCG64(4))
    p = _net(5)
    g = rng.standard_normal(L.NPARAM)
    mo = rng.standard_normal(L.NPARAM) * 0.1
    ve = np.abs(rng.standard_normal(L.NPARAM)) * 0.1
    P, M, V, G = (_cuda32(a) for a in (p, mo, ve, g))
    S.sppc_mlp_adam(P, M, V, G, 7, 1e-3)
    torch.cuda.synchronize()
    p32, m32, v32, g32 = (a.astype(np.float32).astype(np.float64) for a in (p, mo, ve, g))
    # the kernel's constants are FP32 (1 - beta is then exact in FP32 and FP64)
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    pr, mr, vr = L.adam_step(p32, m32, v32, g32, 7, f32(1e-3), beta1=f32(0.9), beta2=f32(0.999), eps=f32(1e-8))
    assert np.allclose(P.cpu().numpy(), pr, rtol=1e-6, atol=1e-7)
    # FP32 rounding of b1 m + (1 - b1) g (terms of size ~0.1 that can cancel)
    assert np.allclose(M.cpu().numpy(), mr, rtol=1e-6, atol=1e-7)
    assert np.allclose(V.cpu().numpy(), vr, rtol=1e-6, atol=1e-8)
    # an epoch with one minibatch = one gradient + one Adam step (same kernels)
    B = 300
    X = rng.standard_normal((B, 6)).astype(np.float32)
    rh = rng.standard_normal(B).astype(np.float32)
    y = rng.standard_normal(B).astype(np.float32)
    Xd, rd, yd = _cuda32(X), _cuda32(rh), _cuda32(y)
    P1, M1, V1 = _cuda32(p), torch.zeros(L.NPARAM, device="cuda"), torch.zeros(L.NPARAM, device="cuda")
    step, _ = S.sppc_mlp_train_epoch(P1, M1, V1, Xd, rd, yd, None, B, 0, 1e-3)
    assert step == 1
    P2, M2, V2 = _cuda32(p), torch.zeros(L.NPARAM, device="cuda"), torch.zeros(L.NPARAM, device="cuda")
    G2 = torch.empty(L.NPARAM, device="cuda")
    S.sppc_mlp_loss_grad(P2, Xd, rd, yd, G2, torch.empty(1, device="cuda"))
    S.sppc_mlp_adam(P2, M2, V2, G2, 1, 1e-3)
    torch.cuda.synchronize()
    assert torch.equal(P1, P2)


def test_training_learns_a_teacher_network():
    """Students trained by the GPU kernels approach a teacher's outputs."""
    import paper_2407_08901_gb300 as S
    rng = np.random.Generator(np.random.PCG64(6))
    teacher = _net(7, scale_out=0.5)
    N = 40_000
    X = rng.standard_normal((N, 6))
    rh = rng.standard_normal(N)
    y = rh * (1.0 + L.forward(teacher, X))
    Xd, rd, yd = _cuda32(X), _cuda32(rh), _cuda32(y)
    P = _cuda32(L.init_params(8))
    M, V = torch.zeros_like(P), torch.zeros_like(P)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(0)
    step, losses = 0, []
    for _ in range(6):
        perm = torch.randperm(N, generator=gen, device="cuda")
        step, loss = S.sppc_mlp_train_epoch(P, M, V, Xd, rd, yd, perm, 256, step, 3e-3)
        losses.append(loss)
    base = float(np.mean((rh - y) ** 2))
    assert losses[-1] < 0.2 * base, (base, losses)
    assert step == 6 * ((N + 255) // 256)


def test_feature_moments_and_standardize():
    import paper_2407_08901_gb300 as S
    rng = np.random.Generator(np.random.PCG64(9))
    F = (rng.standard_normal((50_001, 6)) * [1, 2, 3, 4, 5, 6] + [50, 3, 50, 0, -6, 80]).astype(np.float32)
    Fd = _cuda32(F)
    mu, sd = S.sppc_feature_moments(Fd)
    F64 = F.astype(np.float64)
    assert np.allclose(mu, F64.mean(axis=0), rtol=1e-12, atol=1e-12)
    assert np.allclose(sd, F64.std(axis=0), rtol=1e-9)
    X = torch.empty_like(Fd)
    S.sppc_standardize(Fd, mu, sd, X)
    ref = (F64 - mu.astype(np.float32)) / sd.astype(np.float32)
    assert np.allclose(X.cpu().numpy(), ref, rtol=1e-6, atol=1e-6)


def _column_signs(a, b):
    """+-1 per column so that a * s ~ b (Ritz vectors carry arbitrary signs)."""
    return np.where(np.sum(a * b, axis=0) >= 0, 1.0, -1.0)


def test_training_samples_match_the_oracle():
    """Features and exact-correction targets from the GPU's order-3 Ritz pairs
    against the oracle's, built from its own SPPC run and dense eigenvectors."""
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix("small")
    k, n, n1 = w.k, w.n, w.small_dim
    A = dense(rp, c, v)
    lam, V = np.linalg.eigh(A)
    psi = np.ascontiguousarray(V[:, :k])
    p = 3
    r = oracle_sppc(rp, c, v, n1, k, p_max=p, tol=1e-14, keep=True)
    m = k * (p + 1)
    Ht = r.Q[:, :m].T @ r.W[:, :m]
    th, Y = np.linalg.eigh(0.5 * (Ht + Ht.T))
    th, Y = th[:k], Y[:, :k]
    Z = r.Q[:, :m] @ Y
    R = r.W[:, :m] @ Y - Z * th
    F0, rh0 = L.features(rp, c, v, w.level_offsets, R, th)
    diag = F0[:, 0, 0]
    rh0, y0 = L.training_pairs(psi, Z, R, diag, th, 1e-2, rh0)
    h = S.sppc_create(rp, c, v, w.level_offsets, n1, k, S.sppc_default_opts(p_max=6))
    try:
        S.sppc_start(h, k)
        for _ in range(p):
            S.sppc_correct(h)
            S.sppc_rayleigh_ritz(h, k)
        cnt = (n - n1) * k
        F = torch.empty(cnt, 6, device="cuda")
        rh = torch.empty(cnt, device="cuda")
        y = torch.empty(cnt, device="cuda")
        got = S.sppc_proposal_samples(h, torch.from_numpy(psi).cuda(), F, rh, y)
    finally:
        S.sppc_destroy(h)
    assert got == cnt
    F = F.cpu().numpy().reshape(n - n1, k, 6).astype(np.float64)
    rh = rh.cpu().numpy().reshape(n - n1, k)
    y = y.cpu().numpy().reshape(n - n1, k)
    sg = _column_signs(rh, rh0[n1:])
    ref = F0[n1:]
    for f in (0, 1, 2, 4):
        assert np.allclose(F[..., f], ref[..., f], rtol=1e-6, atol=1e-6), f
    assert np.allclose(F[..., 3] * sg, ref[..., 3], rtol=1e-5, atol=1e-5 * np.max(np.abs(ref[..., 3])))
    assert np.allclose(F[..., 5], ref[..., 5], rtol=1e-5, atol=1e-5 * np.max(np.abs(ref[..., 5])))
    assert np.allclose(rh * sg, rh0[n1:], rtol=1e-5, atol=1e-5 * np.max(np.abs(rh0)))
    assert np.allclose(y * sg, y0[n1:], rtol=1e-4, atol=1e-5 * np.max(np.abs(y0[n1:])))


def _trained_net(device="cuda"):
    """A network trained by the GPU kernels on samples of three small training
    matrices (plain SPPC orders 2-5 against exact dense eigenvectors)."""
    import paper_2407_08901_gb300 as S
    Fs, Rs, Ys = [], [], []
    for seed in (11, 12, 13):
        w = W.Workload(f"t{seed}", [300, 500, 900, 1300], 40, 4, seed=seed)
        rp, c, v = W.generate(w)
        lam, V = np.linalg.eigh(dense(rp, c, v))
        psi = torch.from_numpy(np.ascontiguousarray(V[:, :w.k])).cuda()
        for p in (2, 3, 5):
            h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, S.sppc_default_opts(p_max=6))
            try:
                S.sppc_start(h, w.k)
                for _ in range(p):
                    S.sppc_correct(h)
                    S.sppc_rayleigh_ritz(h, w.k)
                cnt = (w.n - w.small_dim) * w.k
                F = torch.empty(cnt, 6, device=device)
                rh = torch.empty(cnt, device=device)
                y = torch.empty(cnt, device=device)
                S.sppc_proposal_samples(h, psi, F, rh, y)
            finally:
                S.sppc_destroy(h)
            Fs.append(F)
            Rs.append(rh)
            Ys.append(y)
    from paper_2407_08901_gb300.proposal import train
    params, mu, sd, losses, base, trained = train(torch.cat(Fs), torch.cat(Rs), torch.cat(Ys), epochs=3,
                                                  batch=1024, lr=2e-3, log=lambda *_: None)
    return params, mu, sd, base, trained


def test_solve_with_proposal_matches_truth_and_reports_the_gain():
    """SPPC + continuation with the trained network's block (kept iff the
    largest scaled residual drops) converges to the dense eigenvalues; the
    counts of H-vector products are reported beside plain SPPC's and the
    Jacobi-preconditioned continuation's."""
    import paper_2407_08901_gb300 as S
    params, mu, sd, base, trained = _trained_net()
    assert trained < base           # training lowered the loss below the plain block's (m = 0)
    w = W.Workload("small8", [300, 500, 900, 1300], 40, 8, seed=7)
    rp, c, v = W.generate(w)
    lam = np.linalg.eigvalsh(dense(rp, c, v))[: w.k]
    kw = dict(p_max=8, hybrid=1, switch_order=4, precond=1, tol=1e-8, hybrid_maxit=400)
    res = {}
    for name, opts in (("plain_sppc", S.sppc_default_opts(p_max=8, tol=1e-8)),
                       ("jacobi", S.sppc_default_opts(**kw)),
                       ("learned", S.sppc_default_opts(proposal=1, **kw))):
        h = S.sppc_create(rp, c, v, w.level_offsets, w.small_dim, w.k, opts)
        try:
            if name == "learned":
                S.sppc_set_proposal(h, params, mu, sd)
            conv, th, rs, st = S.sppc_solve(h, w.k, tol=1e-8)
        finally:
            S.sppc_destroy(h)
        res[name] = (conv, th, rs, st)
    conv, th, rs, st = res["learned"]
    assert conv and np.all(rs <= 1e-8)
    assert np.allclose(th, lam, rtol=1e-10, atol=0), (th - lam) / np.abs(lam)
    assert st["proposals_tried"] == st["refine_steps"] and 0 <= st["proposals_kept"] <= st["proposals_tried"]
    print("\nH-vector products to 1e-8:", {k_: (bool(r[0]), int(r[3]["spmv_h"])) for k_, r in res.items()},
          "proposals kept", st["proposals_kept"], "of", st["proposals_tried"])
    # plain SPPC stalls above the tolerance within p_max orders; with the
    # network's blocks the same orders plus the continuation reach it
    assert not res["plain_sppc"][0] and np.max(res["plain_sppc"][2]) > 1e-8
    assert res["jacobi"][0]


def test_zero_network_gives_the_jacobi_block_and_in_solve_inference_matches():
    """With m = 0 the proposal equals the plain block; with a trained network the
    in-solve BF16 inference (Tprop / Tplain - 1) matches the oracle's BF16
    inference on the GPU's own features of the same Ritz pairs."""
    import paper_2407_08901_gb300 as S
    w, rp, c, v = make_matrix(W.Workload("small8", [300, 500, 900, 1300], 40, 8, seed=7))
    k, n, n1 = w.k, w.n, w.small_dim
    opts = S.sppc_default_opts(p_max=8, hybrid=1, switch_order=3, precond=1, proposal=1, tol=1e-12)
    rng = np.random.Generator(np.random.PCG64(3))
    for kind in ("zero", "random"):
        params = np.zeros(L.NPARAM) if kind == "zero" else _net(21, scale_out=0.2)
        mu = np.array([30.0, 2.0, 30.0, 0.0, -4.0, 60.0])
        sd = np.array([10.0, 1.0, 10.0, 1.0, 0.5, 30.0])
        h = S.sppc_create(rp, c, v, w.level_offsets, n1, k, opts)
        try:
            S.sppc_set_proposal(h, params, mu, sd)
            S.sppc_start(h, k)
            for _ in range(3):
                S.sppc_correct(h)
                S.sppc_rayleigh_ritz(h, k)
            cnt = (n - n1) * k
            F = torch.empty(cnt, 6, device="cuda")
            rh = torch.empty(cnt, device="cuda")
            y = torch.empty(cnt, device="cuda")
            psi = torch.from_numpy(rng.standard_normal((n, k))).cuda()
            S.sppc_proposal_samples(h, psi, F, rh, y)
            S.sppc_refine_step(h, k)
            Tp = S.sppc_get_state(h, 6, (n, k))
            Tq = S.sppc_get_state(h, 7, (n, k))
        finally:
            S.sppc_destroy(h)
        if kind == "zero":
            assert np.array_equal(Tp, Tq)
            continue
        Fh = F.cpu().numpy().astype(np.float64)
        mu32, sd32 = mu.astype(np.float32), sd.astype(np.float32)
        X = ((Fh.astype(np.float32) - mu32) / sd32).astype(np.float64)
        m_ref = L.infer_bf16(params, X).reshape(n - n1, k)
        sel = np.abs(Tq[n1:]) > 1e-30
        m_gpu = Tp[n1:][sel] / Tq[n1:][sel] - 1.0
        assert np.max(np.abs(m_gpu - m_ref[sel])) <= 2e-2 * max(1.0, np.max(np.abs(m_ref)))
