// Host driver, part 2: the steps of Algorithm 2 and of the continuation on a
// live handle (small eigensolve, MINRES, block Gram-Schmidt and CholeskyQR2,
// Rayleigh-Ritz, thick restart, leading-block correction, learned proposal,
// RMM-DIIS).
#include "driver.h"

namespace sppc::drv {


// ---------------------------------------------------- small-space eigensolve
// Chebyshev-filtered subspace iteration (Zhou and Saad, 2007) on H0_hat:
// filter the block with T_d of the interval [cut, upper] mapped to [-1, 1]
// (damps the unwanted upper spectrum), orthonormalise (shifted CholeskyQR then
// CholeskyQR2), Rayleigh-Ritz on the block; stop when the k lowest residuals are
// <= small_tol * ||H0_hat||.  Products with H0_hat use the same SpMM kernel.

// G (b x b, ld 16) = X^T Z for block sets X, Z of nb blocks (8 columns each).
sppc_status gram_set(sppc_ctx* h, float2** X, float2** Z, int nb, double* G16) {
  cudaStream_t s = h->stream;
  BlockList L;
  L.n = nb;
  for (int a = 0; a < nb; ++a) L.p[a] = X[a];
  for (int ob = 0; ob < nb; ++ob) {
    // out[(a*8+i)*8 + j] for column block ob
    CK(gram(L, Z[ob], 8, 0, h->n1, h->dGram, h->partials, h->partial_cap, h->f64, s));
    // scatter into G16[(a*8+i)*16 + ob*8 + j]
    for (int a = 0; a < nb; ++a)
      CK(cudaMemcpy2DAsync(G16 + (a * 8) * 16 + ob * 8, 16 * sizeof(double), h->dGram + a * 64, 8 * sizeof(double),
                           8 * sizeof(double), 8, cudaMemcpyDeviceToDevice, s));
  }
  return SPPC_OK;
}

// Y_set = X_set * M (M: 16 x 16 double-float, ld 16)
sppc_status rotate_set(sppc_ctx* h, float2** X, float2** Y, int nb, const float2* M16) {
  cudaStream_t s = h->stream;
  BlockList L;
  L.n = nb;
  for (int a = 0; a < nb; ++a) L.p[a] = X[a];
  for (int ob = 0; ob < nb; ++ob) {
    k_subblock<<<1, 128, 0, s>>>(M16, 16, nb, ob, h->dCoefBig); count_launch();
    CK(cudaGetLastError());
    CK(update(Y[ob], nullptr, nullptr, L, h->dCoefBig, 8, 0, h->n1, h->f64, s));
  }
  return SPPC_OK;
}

sppc_status ortho_set(sppc_ctx* h, float2** X, float2** Tmp, int nb, int b) {
  // shifted CholeskyQR, then CholeskyQR twice (result back in X).  A breakdown
  // leaves a finite factor (the pivot set to 1), so the three passes run and
  // their statuses (dStatus[2..4]) are read once at the end; the caller
  // discards the block on a breakdown.
  for (int pass = 0; pass < 3; ++pass) {
    CKS(gram_set(h, X, X, nb, h->dS));
    const double shift = (pass == 0) ? 1e-12 : 0.0;
    CK(chol_rinv(h->dS, 16, b, 16, shift, h->dR1, h->dRinv, h->dStatus + 2 + pass, h->f64, h->stream));
    CKS(rotate_set(h, X, Tmp, nb, h->dRinv));
    for (int a = 0; a < nb; ++a) std::swap(X[a], Tmp[a]);
  }
  int st[3] = {0, 0, 0};
  CK(cudaMemcpyAsync(st, h->dStatus + 2, sizeof(int) * 3, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int pass = 0; pass < 3; ++pass)
    if (st[pass] != 0)
      return fail(h, SPPC_ERR_BREAKDOWN, "small eigensolve: Cholesky breakdown at column %d", st[pass] - 1);
  return SPPC_OK;
}

sppc_status small_eigensolve(sppc_ctx* h) {
  PhaseRange nvtx_range("small_eigensolve");
  cudaStream_t s = h->stream;
  const int64_t n1 = h->n1;
  const int k = h->k;
  int b = h->opt.small_block;
  if (b <= 0) b = std::min(16, std::max(k + 2, 2 * k));
  b = std::max(b, k + 1);
  b = std::min<int64_t>(std::min(b, 16), n1);
  const int nb = (b + 7) / 8;
  float2* X[2] = {h->se[0], h->se[1]};
  float2* AX[2] = {h->se[2], h->se[3]};
  float2* Y0[2] = {h->se[4], h->se[5]};
  float2* Y1[2] = {h->se[6], h->se[7]};
  float2* Tmp[2] = {h->se[8], h->se[9]};
  // seeded normal start block (columns >= b are zero)
  {
    std::vector<float2> host((size_t)n1 * 8 * nb, make_float2(0.f, 0.f));
    const uint64_t seed = h->opt.seed;
    for (int64_t r = 0; r < n1; ++r)
      for (int c = 0; c < b; ++c) {
        const uint64_t idx = (uint64_t)r * 16 + c;
        const double u1 = ((mix64(seed + (2 * idx + 1) * 0x9E3779B97F4A7C15ULL) >> 11) + 1) * 0x1.0p-53;
        const double u2 = (mix64(seed + (2 * idx + 2) * 0x9E3779B97F4A7C15ULL) >> 11) * 0x1.0p-53;
        const double g = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
        put_slot(g, host[(size_t)(c / 8) * n1 * 8 + (size_t)r * 8 + (c % 8)], h->f64);
      }
    for (int a = 0; a < nb; ++a)
      CK(cudaMemcpyAsync(X[a], host.data() + (size_t)a * n1 * 8, sizeof(float2) * n1 * 8, cudaMemcpyHostToDevice, s));
  }
  CKS(ortho_set(h, X, Tmp, nb, b));
  const double upper = h->h11_hi;
  std::vector<double> th(16), res(16);
  const int degree = h->opt.small_degree;
  int outer = 0;
  for (; outer < 400; ++outer) {
    // Rayleigh-Ritz on the block
    CK(spmm11_set(h, 8, X, AX, nullptr, nb, Epi{}, s));
    h->stats.spmv_h11 += 8 * nb;
    CKS(gram_set(h, X, AX, nb, h->dS));
    CK(syev_lowest(h->dS, 16, b, b, h->dTheta, h->dV, b, h->f64, s));
    k_vmat_df<<<1, 256, 0, s>>>(h->dV, b, b, b, h->dRinv, h->f64); count_launch();
    CK(cudaGetLastError());
    CKS(rotate_set(h, X, Tmp, nb, h->dRinv));
    for (int a = 0; a < nb; ++a) std::swap(X[a], Tmp[a]);
    CKS(rotate_set(h, AX, Tmp, nb, h->dRinv));
    for (int a = 0; a < nb; ++a) std::swap(AX[a], Tmp[a]);
    // residuals of the k lowest: D = AX - X theta (block 0 holds columns 0..7);
    // theta and the residual norms come back in one synchronisation
    k_neg_theta<<<1, 32, 0, s>>>(h->dTheta, b, h->dCoef + kTheta, h->f64); count_launch();
    CK(cudaGetLastError());
    CK(combine_diag(Tmp[0], AX[0], h->dCoef + kOnes, one(X[0]), h->dCoef + kTheta, 8, 0, n1, h->f64, s));
    const float2* A1[1] = {Tmp[0]};
    const float2* B1[1] = {Tmp[0]};
    CK(coldots(A1, B1, 1, 8, 0, n1, h->dDots, h->partials, h->partial_cap, h->f64, s));
    CK(cudaMemcpyAsync(th.data(), h->dTheta, sizeof(double) * b, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(res.data(), h->dDots, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double worst = 0.0;
    for (int c = 0; c < k; ++c) worst = std::max(worst, std::sqrt(std::max(res[c], 0.0)));
    if (worst <= h->opt.small_tol * h->h11_norm) break;
    // Chebyshev filter on [cut, upper]
    const double cut = th[b - 1];
    if (!(upper > cut)) return fail(h, SPPC_ERR_BREAKDOWN, "small eigensolve: empty filter interval");
    const double e = 0.5 * (upper - cut), c = 0.5 * (upper + cut);
    auto put3 = [&](double al, double be, double ga) -> sppc_status {
      std::vector<float2> v(48);
      for (int j = 0; j < 16; ++j) {
        put_slot(al, v[j], h->f64);
        put_slot(be, v[16 + j], h->f64);
        put_slot(ga, v[32 + j], h->f64);
      }
      CK(cudaMemcpyAsync(h->dCoef + kCheb, v.data(), sizeof(float2) * 48, cudaMemcpyHostToDevice, s));
      return SPPC_OK;
    };
    // A filter of high degree can leave the block too ill-conditioned for
    // CholeskyQR (its columns collapse onto the lowest eigenvectors): then the
    // block is restored and filtered again with half the degree.
    for (int a = 0; a < nb; ++a)
      CK(cudaMemcpyAsync(h->se[10 + a], X[a], sizeof(float2) * n1 * 8, cudaMemcpyDeviceToDevice, s));
    sppc_status st_f = SPPC_OK;
    for (int deg = degree;; deg /= 2) {
      // Y1 = (A X - c X)/e
      CKS(put3(1.0 / e, -c / e, 0.0));
      Epi e1;
      e1.alpha = h->dCoef + kCheb;
      e1.beta = h->dCoef + kCheb + 16;
      CK(spmm11_set(h, 8, X, Y1, nullptr, nb, e1, s));
      CKS(put3(2.0 / e, -2.0 * c / e, -1.0));
      float2* setA[2] = {X[0], X[1]};
      float2* setB[2] = {Y1[0], Y1[1]};
      float2* setC[2] = {Y0[0], Y0[1]};
      for (int dgi = 2; dgi <= deg; ++dgi) {
        Epi e2;
        e2.alpha = h->dCoef + kCheb;
        e2.beta = h->dCoef + kCheb + 16;
        e2.gamma = h->dCoef + kCheb + 32;
        CK(spmm11_set(h, 8, setB, setC, setA, nb, e2, s));
        for (int a = 0; a < nb; ++a) {
          float2* t0 = setA[a];
          setA[a] = setB[a];
          setB[a] = setC[a];
          setC[a] = t0;
        }
      }
      h->stats.spmv_h11 += (int64_t)8 * nb * deg;
      h->stats.small_eig_iters += deg;
      // new X = setB (the last filtered block); keep the buffers distinct
      for (int a = 0; a < nb; ++a) {
        X[a] = setB[a];
        // the remaining two buffers become AX / Tmp / filter scratch
      }
      {
        // re-assign scratch buffers so that none aliases X
        std::vector<float2*> pool;
        for (int i = 0; i < 10; ++i) pool.push_back(h->se[i]);
        std::vector<float2*> freeb;
        for (float2* q : pool) {
          bool used = false;
          for (int a = 0; a < nb; ++a) used |= (q == X[a]);
          if (!used) freeb.push_back(q);
        }
        int fi = 0;
        for (int a = 0; a < nb; ++a) AX[a] = freeb[fi++];
        for (int a = 0; a < nb; ++a) Y0[a] = freeb[fi++];
        for (int a = 0; a < nb; ++a) Y1[a] = freeb[fi++];
        for (int a = 0; a < nb; ++a) Tmp[a] = freeb[fi++];
      }
      st_f = ortho_set(h, X, Tmp, nb, b);
      if (st_f == SPPC_OK) break;
      if (st_f != SPPC_ERR_BREAKDOWN || deg <= 2) return st_f;
      for (int a = 0; a < nb; ++a)
        CK(cudaMemcpyAsync(X[a], h->se[10 + a], sizeof(float2) * n1 * 8, cudaMemcpyDeviceToDevice, s));
      h->stats.small_filter_retries += 1;
    }
  }
  if (outer >= 400) return fail(h, SPPC_ERR_BREAKDOWN, "small eigensolve did not converge");
  // psi_hat = first k columns (block 0), padded to kp
  h->E0.assign(th.begin(), th.begin() + k);
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < j; ++i)
      if (std::fabs(h->E0[i] - h->E0[j]) <= h->opt.degeneracy_tol * h->h11_norm)
        return fail(h, SPPC_ERR_ARG, "degenerate small-space eigenvalues E_%d ~ E_%d are not supported", i, j);
  if (b > k && std::fabs(th[k] - h->E0[k - 1]) <= h->opt.degeneracy_tol * h->h11_norm)
    return fail(h, SPPC_ERR_ARG, "E_k of the small space is degenerate with E_(k+1)");
  for (int j = 0; j < k; ++j)
    if (std::fabs(h->E0[j]) <= 1e-8 * h->h11_norm)
      return fail(h, SPPC_ERR_ARG, "E^(0)_%d is zero: x2 = -b2/E^(0) is undefined", j);
  // keep all b eigenpairs of the block (deflation of the small solves)
  for (int a = 0; a < nb; ++a)
    CK(cudaMemcpyAsync(h->psib[a], X[a], sizeof(float2) * n1 * 8, cudaMemcpyDeviceToDevice, s));
  {
    std::vector<double> eb(16, 0.0);
    for (int j = 0; j < b; ++j) eb[j] = th[j];
    CK(cudaMemcpyAsync(h->dEb, eb.data(), sizeof(double) * 16, cudaMemcpyHostToDevice, s));
  }
  h->nb_small = nb;
  h->b_small = b;
  // copy columns 0..k-1 of X[0] (n1 x 8) into psi_hat (n1 x kp)
  CK(cudaMemcpy2DAsync(h->psi_hat, sizeof(float2) * h->kp, X[0], sizeof(float2) * 8, sizeof(float2) * h->kp, n1,
                       cudaMemcpyDeviceToDevice, s));
  if (k < h->kp) {
    // zero the padding columns
    CK(cudaMemset2DAsync(h->psi_hat + k, sizeof(float2) * h->kp, 0, sizeof(float2) * (h->kp - k), n1, s));
  }
  std::vector<double> e0p(h->kp, 0.0);
  for (int j = 0; j < k; ++j) e0p[j] = h->E0[j];
  CK(cudaMemcpyAsync(h->dE, e0p.data(), sizeof(double) * h->kp, cudaMemcpyHostToDevice, s));
  k_set_e0<<<1, 32, 0, s>>>(h->dE, k, h->kp, h->dCoef, h->f64); count_launch();
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return SPPC_OK;
}

// ----------------------------------------------------------------- MINRES
// Solves (H0_hat - E_k) x = b1 for the k columns at once on the complement of
// psi_hat_k (Eq. sm_lin_proj) with the persistent kernel of k_minres.cu (one
// cooperative launch); the right-hand side is already deflated.  x0 = 0; stop at
// ||r|| <= minres_tol ||b1||.  Afterwards x is re-projected onto the complement.
// Iterative refinement of the small solves with FP32 MINRES: the right-hand side
// b (h->b1, on the complement of psi_hat) is kept in mref; each sweep runs the
// persistent MINRES in FP32 on the current residual r (relative tolerance
// minres_fp32_tol, at most 2,000 iterations), adds its solution to x (h->mx) and
// recomputes r = b - (H0_hat - E) x in the value format, projected off psi_hat,
// until every ||r_j|| <= minres_tol ||b_j|| (at most 8 sweeps, else
// SPPC_ERR_MINRES).  iters gets each column's FP32 iterations over the sweeps.
sppc_status minres_refined(sppc_ctx* h, int maxit, std::vector<int32_t>& iters) {
  cudaStream_t s = h->stream;
  const int k = h->k, kp = h->kp;
  const int64_t n1 = h->n1;
  float2* c = h->dCoef;
  int* dstat = h->dStatus + 32;
  const size_t bytes = sizeof(float2) * (size_t)n1 * kp;
  CK(cudaMemcpyAsync(h->mref, h->b1, bytes, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->mres, h->b1, bytes, cudaMemcpyDeviceToDevice, s));
  CK(fill_zero(h->mx, (int64_t)n1 * kp, s));
  std::vector<double> bn2(kp), rn2(kp);
  {
    const float2* A[1] = {h->mref};
    const float2* B[1] = {h->mref};
    CK(coldots(A, B, 1, kp, 0, n1, h->dDots, h->partials, h->partial_cap, h->f64, s));
    CK(cudaMemcpyAsync(bn2.data(), h->dDots, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
  }
  const int inner = std::min(maxit, 2000);
  for (int sweep = 0;; ++sweep) {
    if (sweep == 8) return fail(h, SPPC_ERR_MINRES, "refined MINRES: no convergence in 8 sweeps");
    // dx: FP32 MINRES on the residual (its right-hand-side buffer is overwritten)
    CK(cudaMemcpyAsync(h->b1, h->mres, bytes, cudaMemcpyDeviceToDevice, s));
    CK(minres_persistent(h->H11c, k, kp, c + kShiftNegE, h->psi_hat, h->b1, h->mv, h->mvprev, h->my, h->mw1,
                         h->mw2, h->mdx, h->opt.minres_fp32_tol, inner, h->partials, h->partial_cap, h->dBar, dstat,
                         s, h->opt.minres_ctas, h->opt.spin_cap, true));
    int st[10] = {0};
    CK(cudaMemcpyAsync(st, dstat, sizeof(int) * 10, cudaMemcpyDeviceToHost, s));
    // x += dx; r = b - (H0_hat - E) x, projected off psi_hat
    CK(combine_diag(h->mx, h->mx, c + kOnes, one(h->mdx), c + kOnes, kp, 0, n1, h->f64, s));
    Epi e;
    e.alpha = c + kNegOnes;
    e.beta = c + kPosE0;
    e.gamma = c + kOnes;
    e.Z = h->mref;
    CK(spmm11(h, kp, h->mx, h->mres, e, s));
    {
      const float2* A[1] = {h->psi_hat};
      const float2* B[1] = {h->mres};
      CK(coldots(A, B, 1, kp, 0, n1, h->dDots, h->partials, h->partial_cap, h->f64, s));
      k_neg_dots_to_coef<<<1, 32, 0, s>>>(h->dDots, k, kp, c + kDefl, h->f64); count_launch();
      CK(cudaGetLastError());
      CK(combine_diag(h->mres, h->mres, c + kOnes, one(h->psi_hat), c + kDefl, kp, 0, n1, h->f64, s));
      const float2* R[1] = {h->mres};
      CK(coldots(R, R, 1, kp, 0, n1, h->dDots, h->partials, h->partial_cap, h->f64, s));
      CK(cudaMemcpyAsync(rn2.data(), h->dDots, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    if (st[0]) return fail(h, SPPC_ERR_TIMEOUT, "MINRES: a grid barrier timed out");
    int mxit = 0;
    for (int j = 0; j < k; ++j) {
      iters[j] += st[2 + j];
      mxit = std::max(mxit, st[2 + j]);
    }
    h->stats.minres_iters += mxit;
    h->stats.spmv_h11 += (int64_t)k * (std::abs(st[1]) + 1);
    bool done = true;
    for (int j = 0; j < k; ++j)
      done = done && std::sqrt(std::max(rn2[j], 0.0)) <= h->opt.minres_tol * std::sqrt(std::max(bn2[j], 0.0));
    if (done) break;
  }
  return SPPC_OK;
}

sppc_status minres(sppc_ctx* h, std::vector<int32_t>& iters) {
  PhaseRange nvtx_range("minres");
  cudaStream_t s = h->stream;
  const int kp = h->kp;
  const int64_t n1 = h->n1;
  float2* c = h->dCoef;
  int maxit = h->opt.minres_maxit;
  if (maxit <= 0) maxit = (int)std::min<int64_t>(200000, 20 * n1);
  int* dstat = h->dStatus + 32;
  // Deflation by the small eigensolve's other eigenvectors (kp = 8): with
  // Psi_b (b > k vectors, E_b) the solution on span(Psi_b) is exact,
  // x_defl = Psi_b D, D[v][c] = (psi_v^T b1_c) / (E_v - E_c) (v != c); MINRES then
  // solves for the rest, right-hand side b1 - (H0_hat - E) x_defl (exact whatever
  // the accuracy of Psi_b), projected off psi_hat_c.  Same solution, far fewer
  // iterations: the eigenvalues nearest the shift are gone from the operator.
  const bool defl = h->opt.minres_deflate && kp == 8 && h->b_small > h->k;
  if (defl) {
    BlockList Lb;
    Lb.n = h->nb_small;
    Lb.p[0] = h->psib[0];
    Lb.p[1] = h->psib[1];
    // (dC2, not dGram: this may run beside a Rayleigh-Ritz step, which uses dGram)
    CK(gram(Lb, h->b1, 8, 0, n1, h->dC2, h->partials, h->partial_cap, h->f64, s));
    k_defl_coefs<<<1, 128, 0, s>>>(h->dC2, h->dEb, h->b_small, h->k, h->dCoefBig, h->f64); count_launch();
    CK(cudaGetLastError());
    CK(update(h->T2, nullptr, nullptr, Lb, h->dCoefBig, 8, 0, n1, h->f64, s));       // x_defl
    Epi e;
    e.alpha = c + kNegOnes;
    e.beta = c + kPosE0;
    e.gamma = c + kOnes;
    e.Z = h->b1;
    CK(spmm11(h, 8, h->T2, h->T1, e, s));                                // b1 - (H - E) x_defl
    h->stats.spmv_h11 += h->k;
    const float2* A[1] = {h->psi_hat};
    const float2* B[1] = {h->T1};
    CK(coldots(A, B, 1, kp, 0, n1, h->dDots, h->partials, h->partial_cap, h->f64, s));
    k_neg_dots_to_coef<<<1, 32, 0, s>>>(h->dDots, h->k, kp, c + kDefl, h->f64); count_launch();
    CK(cudaGetLastError());
    CK(combine_diag(h->b1, h->T1, c + kOnes, one(h->psi_hat), c + kDefl, kp, 0, n1, h->f64, s));
  }
  iters.assign(h->k, 0);
  if (h->opt.minres_fp32) {
    CKS(minres_refined(h, maxit, iters));
  } else {
    CK(minres_persistent(h->H11c, h->k, kp, c + kShiftNegE, h->psi_hat, h->b1, h->mv, h->mvprev, h->my, h->mw1,
                         h->mw2, h->mx, h->opt.minres_tol, maxit, h->partials, h->partial_cap, h->dBar, dstat, s,
                         h->opt.minres_ctas, h->opt.spin_cap));
  }
  if (defl) CK(combine_diag(h->mx, h->mx, c + kOnes, one(h->T2), c + kOnes, kp, 0, n1, h->f64, s));  // + x_defl
  // x -= psi_hat (psi_hat^T x): keep the solution on the complement of psi_hat_k
  float2* x = h->mx;
  {
    const float2* A[1] = {h->psi_hat};
    const float2* B[1] = {x};
    CK(coldots(A, B, 1, kp, 0, n1, h->dDots, h->partials, h->partial_cap, h->f64, s));
    k_neg_dots_to_coef<<<1, 32, 0, s>>>(h->dDots, h->k, kp, c + kDefl, h->f64); count_launch();
    CK(cudaGetLastError());
    CK(combine_diag(x, x, c + kOnes, one(h->psi_hat), c + kDefl, kp, 0, n1, h->f64, s));
  }
  if (h->opt.minres_fp32) return SPPC_OK;  // statistics kept by minres_refined
  int st[10] = {0};
  CK(cudaMemcpyAsync(st, dstat, sizeof(int) * 10, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (st[0]) return fail(h, SPPC_ERR_TIMEOUT, "MINRES: a grid barrier timed out");
  int mx = 0;
  for (int j = 0; j < h->k; ++j) {
    iters[j] = st[2 + j];
    mx = std::max(mx, st[2 + j]);
  }
  h->stats.minres_iters += mx;
  h->stats.spmv_h11 += (int64_t)h->k * std::abs(st[1]);
  if (st[1] < 0) return fail(h, SPPC_ERR_MINRES, "MINRES reached %d iterations without meeting the tolerance", maxit);
  return SPPC_OK;
}

// Digit tiles of basis blocks 0 .. nq - 1 for the tensor-core kernels, cut for
// every block whose tiles are stale (h->qd_valid; every write of a basis block
// clears its bit).  Error flag in dStatus[8], read with the orthogonalisation's
// status.
cudaError_t ensure_qdigits(sppc_ctx* h, int nq, cudaStream_t s) {
  for (int a = 0; a < nq; ++a) {
    if ((h->qd_valid >> a) & 1ull) continue;
    cudaError_t e = qcut(blk(h->Q, h->n, 8, a), h->n, qdigits_block(h->Qd, h->n, a), h->f64, h->dStatus + 8, s);
    if (e != cudaSuccess) return e;
    h->qd_valid |= 1ull << a;
  }
  return cudaSuccess;
}

// Gram product [Q_0 .. Q_{nq-1}]^T B (Eq. blkGS, Eq. proj): on the tensor cores
// with opts.tensor_gram and 8-column blocks from the block count where they beat
// the CUDA cores (measured on c2: 2 blocks in FP64, where one DFMA Gram block
// costs as much as the tensor kernel's fixed part; 5 in double-float), else on
// the CUDA cores.
cudaError_t qgram(sppc_ctx* h, int nq, const float2* B, double* out, cudaStream_t s) {
  const int64_t n = h->n;
  if (h->Qd && h->kp == 8 && nq >= (h->f64 ? 2 : 5)) {
    cudaError_t e = ensure_qdigits(h, nq, s);
    if (e != cudaSuccess) return e;
    return gram_tc(h->Qd, nq, B, n, out, h->partials, h->partial_cap, h->f64, h->dStatus + 8, h->dStatus + 16, s);
  }
  return gram(blocks(h->Q, n, h->kp, 0, nq), B, h->kp, 0, n, out, h->partials, h->partial_cap, h->f64, s);
}

// Block update Y = alpha X + [Q_0 .. Q_{nq-1}] coef (Eq. blkGS, the restart's
// Q Y): on the tensor cores under the same conditions as qgram, from 2 blocks
// in FP64 and 4 in double-float (measured on 2e6 rows: 214 against 237 us at 4
// blocks, 200 against 144 us at 2), else on the CUDA cores.
cudaError_t qupdate(sppc_ctx* h, int nq, float2* Y, const float2* X, const float2* alpha, const float2* coef,
                    cudaStream_t s) {
  const int64_t n = h->n;
  if (h->Qd && h->kp == 8 && nq >= (h->f64 ? 2 : 4)) {
    cudaError_t e = ensure_qdigits(h, nq, s);
    if (e != cudaSuccess) return e;
    return update_tc(h->Qd, nq, coef, alpha, X, Y, n, h->f64, h->dStatus + 8, s);
  }
  return update(Y, X, alpha, blocks(h->Q, n, h->kp, 0, nq), coef, h->kp, 0, n, h->f64, s);
}

// Digit tiles of W blocks 0 .. nq - 1 (W = H Q, not orthonormal): column
// exponents, then the cut at 2^(61 - e) per column.
cudaError_t ensure_wdigits(sppc_ctx* h, int nq, cudaStream_t s) {
  for (int a = 0; a < nq; ++a) {
    if ((h->wd_valid >> a) & 1ull) continue;
    const float2* w = blk(h->W, h->n, 8, a);
    cudaError_t e = colexp(w, h->n, h->wexp + 8 * a, h->f64, s);
    if (e == cudaSuccess)
      e = qcut(w, h->n, qdigits_block(h->Wd, h->n, a), h->f64, h->dStatus + 8, s, h->wexp + 8 * a);
    if (e != cudaSuccess) return e;
    h->wd_valid |= 1ull << a;
  }
  return cudaSuccess;
}

// Whether a product over nq basis blocks takes the tensor cores: from 2 blocks
// in FP64; in double-float from 4 for block updates and 10 for the Ritz pass
// (two tensor-core updates against one fused CUDA-core pass over Q and W).
bool tensor_dense(const sppc_ctx* h, int nq, DenseKind kind) {
  if (!h->Qd || h->kp != 8) return false;
  return nq >= (h->f64 ? 2 : (kind == DenseKind::update ? 4 : 10));
}

// Update against W blocks 0 .. nq - 1 (the restart's W Y, the recycled H Psi of
// Eq. HPsip): tensor cores under qupdate's conditions, else CUDA cores.
cudaError_t wupdate(sppc_ctx* h, int nq, float2* Y, const float2* X, const float2* alpha, const float2* coef,
                    cudaStream_t s) {
  if (tensor_dense(h, nq, DenseKind::update)) {
    cudaError_t e = ensure_wdigits(h, nq, s);
    if (e != cudaSuccess) return e;
    return update_tc(h->Wd, nq, coef, alpha, X, Y, h->n, h->f64, h->dStatus + 8, s, h->wexp);
  }
  return update(Y, X, alpha, blocks(h->W, h->n, h->kp, 0, nq), coef, h->kp, 0, h->n, h->f64, s);
}

__global__ void k_neg_slots(const float2* in, float2* out, int count, bool f64) {
  const int i = threadIdx.x;
  if (i < count) out[i] = f64 ? make_float2(in[i].x, -in[i].y) : make_float2(-in[i].x, -in[i].y);
}

// The Ritz pass over blocks 0 .. np1 - 1 (Eq. rrn): ritz_resid's outputs (dDots =
// squared residual norms; optional Z, T, leading rows).  On the tensor cores:
// Zt = Q Y, Dt = W Y - Z theta (two tensor-core updates), then the norms, the
// preconditioned block and the copies from Zt and Dt.
cudaError_t qritz(sppc_ctx* h, int np1, double* Zout, int64_t ldz, int ncols, float2* Tout, const float2* diag,
                  float clamp, float2* Zlead, float2* Rlead, int64_t nlead, cudaStream_t s) {
  const int kp = h->kp;
  const int64_t n = h->n;
  if (!tensor_dense(h, np1, DenseKind::ritz))
    return ritz_resid(blocks(h->Q, n, kp, 0, np1), blocks(h->W, n, kp, 0, np1), h->dY, h->dCoef + kTheta, kp, n,
                      h->dDots, h->partials, h->partial_cap, Zout, ldz, ncols, Tout, diag, clamp, h->f64, s, Zlead,
                      Rlead, nlead);
  cudaError_t e = ensure_qdigits(h, np1, s);
  if (e == cudaSuccess) e = ensure_wdigits(h, np1, s);
  if (e != cudaSuccess) return e;
  k_neg_slots<<<1, 32, 0, s>>>(h->dCoef + kTheta, h->dCoef + kRitzNegTh, kp, h->f64);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = update_tc(h->Qd, np1, h->dY, nullptr, nullptr, h->Zt, n, h->f64, h->dStatus + 8, s)) != cudaSuccess) return e;
  if ((e = update_tc(h->Wd, np1, h->dY, h->dCoef + kRitzNegTh, h->Zt, h->Dt, n, h->f64, h->dStatus + 8, s, h->wexp)) !=
      cudaSuccess)
    return e;
  {
    const float2* A[1] = {h->Dt};
    const float2* B[1] = {h->Dt};
    if ((e = coldots(A, B, 1, kp, 0, n, h->dDots, h->partials, h->partial_cap, h->f64, s)) != cudaSuccess) return e;
  }
  if (Zout && (e = df_to_f64(h->Zt, kp, Zout, ldz, ncols, 0, n, h->f64, s)) != cudaSuccess) return e;
  if (nlead > 0 && Zlead) {
    if ((e = cudaMemcpyAsync(Zlead, h->Zt, sizeof(float2) * nlead * kp, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
    if ((e = cudaMemcpyAsync(Rlead, h->Dt, sizeof(float2) * nlead * kp, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
  }
  if (Tout) e = ritz_precond(h->Dt, h->dCoef + kTheta, diag, clamp, Tout, kp, n, h->f64, s);
  return e;
}

// ------------------------------------------------------- Rayleigh-Ritz core
// Rayleigh-Ritz on blocks 0..p: border the projected matrix with Q^T W_p (Eq.
// proj), its nev = min(2k, m) lowest eigenpairs (the first k are the Ritz pairs;
// 2k are kept for a thick restart), Ritz residuals (Eq. rrn).  Optionally writes
// the Ritz vectors (Z) and the preconditioned residual block (T, see ritz_resid).
sppc_status rr_core(sppc_ctx* h, int p, bool want_z, double* Z, int64_t ldz, float2* T, const float2* diag,
                    bool defer) {
  PhaseRange nvtx_range("rayleigh_ritz");
  cudaStream_t s = h->stream;
  const int k = h->k, kp = h->kp;
  const int64_t n = h->n;
  CK(qgram(h, p + 1, blk(h->W, n, kp, p), h->dGram, s));
  k_assemble_ht<<<1, 256, 0, s>>>(h->dGram, p, k, kp, h->dHt, h->mmax); count_launch();
  CK(cudaGetLastError());
  const int m = (p + 1) * k;
  const int nev = std::min(std::min(2 * k, m), 16);
  h->nev = nev;
  CK(syev_lowest(h->dHt, h->mmax, m, nev, h->dTheta, h->dV, nev, h->f64, s));
  k_expand_y<<<1, 256, 0, s>>>(h->dV, nev, p, k, kp, h->dTheta, h->dY, h->dCoef + kTheta, h->f64); count_launch();
  CK(cudaGetLastError());
  const bool lead = T != nullptr && h->opt.precond == 2;
  CK(qritz(h, p + 1, want_z ? Z : nullptr, ldz, k, T, diag, (float)h->opt.precond_clamp, lead ? h->zlead : nullptr,
           lead ? h->rlead : nullptr, lead ? h->n_lead : 0, s));
  if (defer) {
    // results land in pinned host memory; rr_finish() reads them after a sync
    CK(cudaMemcpyAsync(h->pinned, h->dTheta, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->pinned + 16, h->dDots, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
    return SPPC_OK;
  }
  std::vector<double> th(k), r2(kp);
  CK(cudaMemcpyAsync(th.data(), h->dTheta, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(r2.data(), h->dDots, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->theta = th;
  h->resid.assign(k, 0.0);
  for (int j = 0; j < k; ++j) h->resid[j] = std::sqrt(std::max(r2[j], 0.0)) / std::fabs(th[j]);
  return SPPC_OK;
}

// Completes a deferred rr_core: waits for its stream, then Ritz values and
// scaled residuals from the pinned copies.
sppc_status rr_finish(sppc_ctx* h, cudaStream_t s) {
  CK(cudaStreamSynchronize(s));
  const int k = h->k;
  h->theta.assign(h->pinned, h->pinned + k);
  h->resid.assign(k, 0.0);
  for (int j = 0; j < k; ++j)
    h->resid[j] = std::sqrt(std::max(h->pinned[16 + j], 0.0)) / std::fabs(h->pinned[j]);
  return SPPC_OK;
}

// Block Gram-Schmidt (Eq. blkGS) of src against Q blocks 0..p-1, then
// CholeskyQR2 (Eq. QR) into Q block p (Eq. Qp).  SPPC orders apply the
// projector of Eq. blkGS twice (CGS2, against round-off).  With `cond` (the block continuation) the
// second application runs only when the first removed more than half of some
// column's norm (criterion of Daniel, Gragg, Kaufman and Stewart with Kahan's
// factor: after a pass that keeps at least half the norm the result is
// orthogonal to Q to working accuracy).  Leaves the projection coefficients C
// (sum of the passes) in dC1 and R = R2 R1 in the recycle coefficients [C; R]
// (Eq. HPsip).  dd (host, 2*kp) receives ||src_j||^2 and ||Phi_j||^2.
sppc_status orth_append(sppc_ctx* h, const float2* src, int p, double* dd, bool cond) {
  PhaseRange nvtx_range("orth_append");
  cudaStream_t s = h->stream;
  const int k = h->k, kp = h->kp;
  const int64_t n = h->n;
  float2* c = h->dCoef;
  const int nc = p * kp * kp;
  CK(qgram(h, p, src, h->dC1, s));
  k_negmat<<<(nc + 255) / 256, 256, 0, s>>>(h->dC1, nc, h->dCoefBig, h->f64); count_launch();
  CK(cudaGetLastError());
  CK(qupdate(h, p, h->T1, src, c + kOnes, h->dCoefBig, s));
  {
    const float2* A[2] = {src, h->T1};
    const float2* B[2] = {src, h->T1};
    CK(coldots(A, B, 2, kp, 0, n, h->dDots, h->partials, h->partial_cap, h->f64, s));
  }
  CK(cudaMemcpyAsync(dd, h->dDots, sizeof(double) * 2 * kp, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  bool again = !cond;
  for (int j = 0; j < k; ++j) again |= !(dd[kp + j] >= 0.25 * dd[j]);  // ||Phi_j|| < ||src_j|| / 2
  h->stats.reorth_passes += again ? 1 : 0;
  if (again) {
    CK(qgram(h, p, h->T1, h->dC2, s));
    k_negmat<<<(nc + 255) / 256, 256, 0, s>>>(h->dC2, nc, h->dCoefBig, h->f64); count_launch();
    CK(cudaGetLastError());
    CK(qupdate(h, p, h->T1, h->T1, c + kOnes, h->dCoefBig, s));
    k_addmat<<<(nc + 255) / 256, 256, 0, s>>>(h->dC1, h->dC2, nc, h->dC1); count_launch();  // C = C1 + C2
    CK(cudaGetLastError());
    const float2* A[1] = {h->T1};
    const float2* B[1] = {h->T1};
    CK(coldots(A, B, 1, kp, 0, n, h->dDots, h->partials, h->partial_cap, h->f64, s));
    CK(cudaMemcpyAsync(dd + kp, h->dDots, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
  }
  float2* q = blk(h->Q, n, kp, p);
  h->qd_valid &= ~(1ull << p);  // block p is rewritten below
  CK(gram_sym(h->T1, kp, 0, n, h->dS, h->partials, h->partial_cap, h->f64, s));
  CK(chol_rinv(h->dS, kp, k, kp, 0.0, h->dR1, h->dRinv, h->dStatus, h->f64, s));
  CK(update_tri(h->T2, h->T1, h->dRinv, kp, 0, n, h->f64, s));
  CK(gram_sym(h->T2, kp, 0, n, h->dS, h->partials, h->partial_cap, h->f64, s));
  CK(chol_rinv(h->dS, kp, k, kp, 0.0, h->dR2, h->dRinv, h->dStatus + 1, h->f64, s));
  CK(update_tri(q, h->T2, h->dRinv, kp, 0, n, h->f64, s));
  k_recycle_coefs<<<1, 256, 0, s>>>(h->dC1, p, kp, h->dR2, h->dR1, h->dRecycle, h->f64); count_launch();
  CK(cudaGetLastError());
  int st[2] = {0, 0}, tmo = 0, tcf = 0;
  CK(cudaMemcpyAsync(st, h->dStatus, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
  CK(spmm_tma_read_timeout(h->H, &tmo, s));
  if (h->opt.tensor_gram) CK(cudaMemcpyAsync(&tcf, h->dStatus + 8, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (tmo) return fail(h, SPPC_ERR_TIMEOUT, "SpMM: a shared-memory pipeline wait timed out");
  if (tcf) CK(cudaMemsetAsync(h->dStatus + 8, 0, sizeof(int), s));  // reported once
  if (tcf & 2) return fail(h, SPPC_ERR_TIMEOUT, "tensor-core Gram: a pipeline wait timed out");
  if (tcf & 1) return fail(h, SPPC_ERR_NAN, "tensor-core Gram: a basis entry is not finite (or |q| >= 2)");
  if (st[0] || st[1])
    return fail(h, SPPC_ERR_BREAKDOWN, "CholeskyQR breakdown appending block %d (rank-deficient block)", p);
  return SPPC_OK;
}

// Thick restart of the continuation: Q <- Q Y_2k, W <- W Y_2k (two blocks of k
// Ritz vectors, the 2k lowest), projected matrix recomputed from the new blocks.
sppc_status restart(sppc_ctx* h, bool fresh_products) {
  PhaseRange nvtx_range("restart");
  cudaStream_t s = h->stream;
  const int k = h->k, kp = h->kp, p = h->p;
  const int64_t n = h->n;
  if (h->nev < 2 * k) return fail(h, SPPC_ERR_STATE, "restart needs 2k Ritz vectors");
  for (int b = 0; b < 2; ++b) {
    k_restart_coef<<<1, 256, 0, s>>>(h->dV, h->nev, p, k, kp, b, h->dCoefBig, h->f64); count_launch();
    CK(cudaGetLastError());
    CK(qupdate(h, p + 1, blk(h->Psi, n, kp, b), nullptr, nullptr, h->dCoefBig, s));
    CK(wupdate(h, p + 1, blk(h->Psi, n, kp, 2 + b), nullptr, nullptr, h->dCoefBig, s));
  }
  CK(cudaMemcpyAsync(h->Q, h->Psi, sizeof(float2) * 2 * n * kp, cudaMemcpyDeviceToDevice, s));
  h->qd_valid = 0;
  if (fresh_products) {
    // W = H Q recomputed (mixed precision: replaces products made in FP32)
    for (int b = 0; b < 2; ++b) CKS(big_spmm(h, blk(h->Q, n, kp, b), blk(h->W, n, kp, b), kp));
    h->stats.spmv_h += 2 * h->k;
  } else {
    CK(cudaMemcpyAsync(h->W, blk(h->Psi, n, kp, 2), sizeof(float2) * 2 * n * kp, cudaMemcpyDeviceToDevice, s));
    h->wd_valid = 0;
  }
  for (int b = 0; b < 2; ++b) {
    CK(qgram(h, b + 1, blk(h->W, n, kp, b), h->dGram, s));
    k_assemble_ht<<<1, 256, 0, s>>>(h->dGram, b, k, kp, h->dHt, h->mmax); count_launch();
    CK(cudaGetLastError());
  }
  h->p = 1;
  h->stats.restarts += 1;
  return SPPC_OK;
}

// Leading-block preconditioner of the continuation (opts.precond = 2): replace the
// leading n1 rows of T by precond_iters MINRES steps (x0 = 0, no stopping test) on
// P (H0_hat - theta_j) P t = P r_j[:n1] with P = I - z z^T, z = z_j[:n1] / ||z_j[:n1]||,
// then t <- P t.  The Ritz vectors' and residuals' leading rows come from the pass
// that produced T (zlead, rlead).  The shifted exact leading block, deflated by the
// Ritz vector, with the shifted diagonal elsewhere: this repository's reading of
// the shifted block-diagonal preconditioner the paper pairs with LOBPCG (Sec. 5).
sppc_status lead_correction(sppc_ctx* h, float2* T) {
  cudaStream_t s = h->stream;
  const int k = h->k, kp = h->kp;
  const int64_t n1 = h->n_lead;  // rows of the leading block
  float2* c = h->dCoef;
  const int iters = h->opt.precond_iters;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (h->opt.timing) {
    t0 = next_event(h);
    t1 = next_event(h);
    CK(cudaEventRecord(t0, s));
  }
  {  // z <- z / ||z|| (columnwise)
    const float2* A[1] = {h->zlead};
    const float2* B[1] = {h->zlead};
    CK(coldots(A, B, 1, kp, 0, n1, h->dDots, h->partials, h->partial_cap, h->f64, s));
    k_inv_norm_coef<<<1, 32, 0, s>>>(h->dDots, k, kp, c + kLeadScale, h->f64); count_launch();
    CK(cudaGetLastError());
    CK(combine_diag(h->zlead, nullptr, nullptr, one(h->zlead), c + kLeadScale, kp, 0, n1, h->f64, s));
  }
  {  // b = r - z (z^T r)
    const float2* A[1] = {h->zlead};
    const float2* B[1] = {h->rlead};
    CK(coldots(A, B, 1, kp, 0, n1, h->dDots, h->partials, h->partial_cap, h->f64, s));
    k_neg_dots_to_coef<<<1, 32, 0, s>>>(h->dDots, k, kp, c + kDefl, h->f64); count_launch();
    CK(cudaGetLastError());
    CK(combine_diag(h->b1, h->rlead, c + kOnes, one(h->zlead), c + kDefl, kp, 0, n1, h->f64, s));
  }
  k_neg_coef<<<1, 32, 0, s>>>(c + kTheta, k, kp, c + kLeadNegE, h->f64); count_launch();
  CK(cudaGetLastError());
  int* dstat = h->dStatus + 32;
  if (iters > 0) {
    CK(minres_persistent(h->Hlead, k, kp, c + kLeadNegE, h->zlead, h->b1, h->mv, h->mvprev, h->my, h->mw1, h->mw2,
                         h->mx, 0.0, iters, h->partials, h->partial_cap, h->dBar, dstat, s, 0, h->opt.spin_cap));
    // x <- x - z (z^T x)
    const float2* A[1] = {h->zlead};
    const float2* B[1] = {h->mx};
    CK(coldots(A, B, 1, kp, 0, n1, h->dDots, h->partials, h->partial_cap, h->f64, s));
    k_neg_dots_to_coef<<<1, 32, 0, s>>>(h->dDots, k, kp, c + kDefl, h->f64); count_launch();
    CK(cudaGetLastError());
    CK(combine_diag(h->mx, h->mx, c + kOnes, one(h->zlead), c + kDefl, kp, 0, n1, h->f64, s));
    CK(cudaMemcpyAsync(T, h->mx, sizeof(float2) * n1 * kp, cudaMemcpyDeviceToDevice, s));
  } else {
    CK(fill_zero(T, n1 * kp, s));
  }
  int st[10] = {0};
  if (iters > 0) CK(cudaMemcpyAsync(st, dstat, sizeof(int) * 10, cudaMemcpyDeviceToHost, s));
  if (h->opt.timing) CK(cudaEventRecord(t1, s));
  CK(cudaStreamSynchronize(s));
  if (st[0]) return fail(h, SPPC_ERR_TIMEOUT, "leading-block MINRES: a grid barrier timed out");
  int mx = 0;
  for (int j = 0; j < k; ++j) mx = std::max(mx, st[2 + j]);
  h->stats.minres_iters += mx;
  h->stats.spmv_h11 += (int64_t)k * std::abs(st[1]);
  if (h->opt.timing) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, t0, t1));
    h->stats.minres_ms += ms;
  }
  return SPPC_OK;
}

// Diagonal of the Ritz-residual pass's T output: the Jacobi denominators, or none
// (T = the raw residual) when the learned proposal builds the block itself.
const float2* t_diag(const sppc_ctx* h) {
  if (h->opt.proposal == 1) return nullptr;
  return h->opt.precond ? h->dDiag : nullptr;
}

// Buffers of the learned proposal (allocated on first use).
sppc_status ensure_proposal_buffers(sppc_ctx* h) {
  const int64_t n = h->n;
  cudaError_t e = cudaSuccess;
  if (!h->net) e = dalloc(h, &h->net, (size_t)(kNetParams + 2 * kNetFeatures));
  if (e == cudaSuccess && !h->rhat32) e = dalloc(h, &h->rhat32, (size_t)n * 8);
  if (e == cudaSuccess && !h->Tprop) e = dalloc(h, &h->Tprop, (size_t)n * h->kp);
  if (e == cudaSuccess && !h->Tplain) e = dalloc(h, &h->Tplain, (size_t)n * h->kp);
  if (e == cudaSuccess && !h->X32) e = dalloc(h, &h->X32, (size_t)n * 8);
  if (e == cudaSuccess && !h->val32 && !h->val16) {
    // FP32 copy of the values for the |H| product (their double-float high words)
    const int64_t total = h->h_slice_ptr.empty() ? 0 : h->h_slice_ptr.back();
    e = dalloc(h, &h->val32, (size_t)(total > 0 ? total : 1));
    if (e == cudaSuccess) e = df_hi_parts(h->H.val, h->val32, total, h->stream);
  }
  if (e != cudaSuccess)
    return fail(h, e == cudaErrorMemoryAllocation ? SPPC_ERR_OOM : SPPC_ERR_CUDA, "proposal buffers: %s",
                cudaGetErrorString(e));
  return SPPC_OK;
}

// Learned proposal from the raw Ritz residuals R (n x kp) of the last
// Rayleigh-Ritz pass and their squared norms in dDots: rhat, |H| |rhat|, the
// network, Tprop = (R / den)(1 + m) and Tplain = R / den for rows [n0, n)
// (n0 = n1 when the leading block has its own correction).
sppc_status proposal_block(sppc_ctx* h, const float2* R) {
  PhaseRange nvtx_range("proposal");
  cudaStream_t s = h->stream;
  const int k = h->k, kp = h->kp;
  const int64_t n = h->n;
  const int64_t n0 = h->opt.precond == 2 ? h->n_lead : 0;
  CK(prop_prep(R, kp, k, h->dDots, n, h->rhat32, h->X32, s));
  CK(spmm_abs_f32(h->H, h->val32, h->val16, h->diag32, h->X32, h->T2, s));
  CK(prop_mlp(h->net, R, h->dDiag, h->rowc, h->rhat32, h->T2, h->dCoef + kTheta, (float)h->opt.precond_clamp, k,
              kp, n0, n, h->Tprop, h->Tplain, s));
  return SPPC_OK;
}

// One step of the continuation after SPPC (block Davidson, Jacobi-preconditioned
// residuals; without preconditioner the block Krylov extension): from the last
// Rayleigh-Ritz pairs, T = preconditioned residuals, thick restart if the basis
// is full, orthogonalise T and append it, k SpMVs, Rayleigh-Ritz.
// With the learned proposal (opts.proposal = 1) T is the network's block; it is
// kept iff the largest scaled residual drops, else the step is redone with the
// plain preconditioned block.
sppc_status refine_step(sppc_ctx* h) {
  PhaseRange nvtx_range("refine_step");
  const int kp = h->kp;
  const int64_t n = h->n;
  const bool learn = h->opt.proposal == 1;
  const bool lead = h->opt.precond == 2;
  if (learn && !h->net_ready) return fail(h, SPPC_ERR_STATE, "opts.proposal = 1 needs sppc_set_proposal first");
  // T from the current Ritz pairs: written by the previous Rayleigh-Ritz pass when
  // it already ran in continuation mode, else one extra pass over Q and W
  if (!h->t_ready) {
    CK(qritz(h, h->p + 1, nullptr, 0, 0, h->HPsi, t_diag(h), (float)h->opt.precond_clamp, lead ? h->zlead : nullptr,
             lead ? h->rlead : nullptr, lead ? h->n_lead : 0, h->stream));
  }
  h->t_ready = false;
  float2* T = h->HPsi;
  if (learn) {
    CKS(proposal_block(h, h->HPsi));
    if (lead) {
      CKS(lead_correction(h, h->Tplain));
      CK(cudaMemcpyAsync(h->Tprop, h->Tplain, sizeof(float2) * h->n_lead * kp, cudaMemcpyDeviceToDevice,
                         h->stream));
    }
    T = h->Tprop;
  } else if (lead) {
    CKS(lead_correction(h, h->HPsi));
  }
  if (h->p + 1 >= std::min(h->pmax + 1, h->opt.hybrid_blocks)) CKS(restart(h));
  const double before = h->resid.empty() ? 0.0 : *std::max_element(h->resid.begin(), h->resid.end());
  std::vector<double> dd(2 * kp);
  CKS(orth_append(h, T, h->p + 1, dd.data(), h->opt.reorth == 0));
  if (T == h->HPsi && h->Tspare) {
    // keep the appended block readable (sppc_get_state 8): the next
    // Rayleigh-Ritz pass writes its block into the other buffer
    std::swap(h->HPsi, h->Tspare);
    T = h->Tspare;
  }
  h->t_last = T;
  h->p += 1;
  CKS(big_spmm(h, blk(h->Q, n, kp, h->p), blk(h->W, n, kp, h->p), kp));
  h->stats.spmv_h += h->k;
  CKS(rr_core(h, h->p, false, nullptr, 0, h->HPsi, t_diag(h)));
  if (learn) {
    h->stats.proposals_tried += 1;
    const double after = *std::max_element(h->resid.begin(), h->resid.end());
    if (after < before) {
      h->stats.proposals_kept += 1;
    } else {
      // drop the proposal's block, extend by the plain preconditioned block
      h->p -= 1;
      CKS(orth_append(h, h->Tplain, h->p + 1, dd.data(), h->opt.reorth == 0));
      h->t_last = h->Tplain;
      h->p += 1;
      CKS(big_spmm(h, blk(h->Q, n, kp, h->p), blk(h->W, n, kp, h->p), kp));
      h->stats.spmv_h += h->k;
      CKS(rr_core(h, h->p, false, nullptr, 0, h->HPsi, t_diag(h)));
    }
  }
  h->t_ready = true;
  OrderRec r;
  r.theta = h->theta;
  r.resid = h->resid;
  r.angle.resize(h->k);
  for (int j = 0; j < h->k; ++j) r.angle[j] = std::sqrt(std::max(dd[kp + j], 0.0) / std::max(dd[j], 1e-300));
  h->rec.push_back(r);
  h->stats.refine_steps += 1;
  if (h->opt.timing) CKS(collect_timing(h));
  return SPPC_OK;
}

// SPPC + per-pair RMM-DIIS (opts.hybrid = 2; Sec. 6): from the Ritz vectors of
// the last Rayleigh-Ritz step, each column runs its own RMM-DIIS (DIIS over the
// last `depth` = min(8, p_max + 1) residuals, Jacobi-preconditioned step of
// length 1), all columns in one 8-column product per iteration; a column stops
// (is frozen) once its scaled residual meets tol.  The SPPC basis Q / W is no
// longer needed and holds the history ring (x in Q blocks, r in W blocks).
sppc_status rmm_run(sppc_ctx* h, double tol) {
  PhaseRange nvtx_range("rmm_diis");
  cudaStream_t s = h->stream;
  const int k = h->k, kp = h->kp;
  const int64_t n = h->n;
  const int d = std::min(8, h->pmax + 1);
  float2* c = h->dCoef;
  if (!h->rmm_G) {
    cudaError_t e = dalloc(h, &h->rmm_G, (size_t)8 * 64);
    if (e == cudaSuccess) e = dalloc(h, &h->rmm_th, 16);
    if (e == cudaSuccess) e = dalloc(h, &h->rmm_lam, 16);
    if (e == cudaSuccess) e = dalloc(h, &h->rmm_g, 64);
    if (e == cudaSuccess) e = dalloc(h, &h->rmm_frozen, 16);
    if (e == cudaSuccess) e = dalloc(h, &h->rmm_status, 16);
    if (e == cudaSuccess) e = dalloc(h, &h->rmm_coef, 64);
    if (e != cudaSuccess) return fail(h, SPPC_ERR_OOM, "RMM-DIIS buffers: %s", cudaGetErrorString(e));
  }
  float2* Wt = blk(h->Psi, n, kp, 0);
  float2* Xb = blk(h->Psi, n, kp, 1);
  float2* Rb = blk(h->Psi, n, kp, 2);
  BlockList Lx, Lr;
  Lx.n = Lr.n = d;
  float2* hx[8];
  float2* hr[8];
  h->qd_valid = 0;  // the RMM-DIIS history overwrites the basis blocks and W
  h->wd_valid = 0;
  for (int a = 0; a < d; ++a) {
    hx[a] = blk(h->Q, n, kp, a);
    hr[a] = blk(h->W, n, kp, a);
    Lx.p[a] = hx[a];
    Lr.p[a] = hr[a];
  }
  auto normalise = [&](float2* X) -> sppc_status {
    const float2* A[1] = {X};
    const float2* B[1] = {X};
    CK(coldots(A, B, 1, kp, 0, n, h->dDots, h->partials, h->partial_cap, h->f64, s));
    k_inv_norm_coef<<<1, 32, 0, s>>>(h->dDots, k, kp, c + kRmmScale, h->f64); count_launch();
    CK(cudaGetLastError());
    CK(combine_diag(X, nullptr, nullptr, one(X), c + kRmmScale, kp, 0, n, h->f64, s));
    return SPPC_OK;
  };
  // x_0: the Ritz vectors Z = Q Y of the last Rayleigh-Ritz step, normalised
  CK(update(Xb, nullptr, nullptr, blocks(h->Q, n, kp, 0, h->p + 1), h->dY, kp, 0, n, h->f64, s));
  CK(cudaMemcpyAsync(hx[0], Xb, sizeof(float2) * n * kp, cudaMemcpyDeviceToDevice, s));
  CKS(normalise(hx[0]));
  CK(cudaMemsetAsync(h->rmm_G, 0, sizeof(double) * 8 * 64, s));
  CK(cudaMemsetAsync(h->rmm_status, 0, sizeof(int) * 16, s));
  std::vector<int> frozen(16, 1);
  for (int j = 0; j < k; ++j) frozen[j] = 0;
  std::vector<double> lam(16, 0.0);
  std::vector<double> th(kp), rr(kp);
  int cur = 0, nh = 0;
  for (;;) {
    float2* X = hx[cur];
    CKS(big_spmm(h, X, Wt, kp));
    h->stats.spmv_h += k;
    {
      const float2* A[2] = {X, X};
      const float2* B[2] = {X, Wt};
      CK(coldots(A, B, 2, kp, 0, n, h->dDots, h->partials, h->partial_cap, h->f64, s));
    }
    k_rmm_theta<<<1, 32, 0, s>>>(h->dDots, k, kp, c + kRmmNegTh, h->rmm_th); count_launch();
    CK(cudaGetLastError());
    CK(combine_diag(hr[cur], Wt, c + kOnes, one(X), c + kRmmNegTh, kp, 0, n, h->f64, s));   // r = w - theta x
    {
      const float2* A[1] = {hr[cur]};
      const float2* B[1] = {hr[cur]};
      CK(coldots(A, B, 1, kp, 0, n, h->dDots, h->partials, h->partial_cap, h->f64, s));
    }
    CK(cudaMemcpyAsync(th.data(), h->rmm_th, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(rr.data(), h->dDots, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->theta.assign(th.begin(), th.begin() + k);
    h->resid.assign(k, 0.0);
    bool all = true;
    for (int j = 0; j < k; ++j) {
      h->resid[j] = std::sqrt(std::max(rr[j], 0.0)) / std::fabs(th[j]);
      if (h->resid[j] <= tol) frozen[j] = 1;
      all = all && frozen[j];
    }
    OrderRec r;
    r.theta = h->theta;
    r.resid = h->resid;
    r.angle.assign(k, 0.0);
    h->rec.push_back(r);
    h->rmm_x = X;
    if (all || h->stats.refine_steps >= h->opt.hybrid_maxit) break;
    h->stats.refine_steps += 1;
    nh = std::min(nh + 1, d);
    // r_a^T r_cur for the active slots, four pairs per call
    for (int t0 = 0; t0 < nh; t0 += 4) {
      const float2* A[4];
      const float2* B[4];
      const int nq = std::min(4, nh - t0);
      for (int q = 0; q < nq; ++q) {
        A[q] = hr[(cur - (nh - 1) + t0 + q + d) % d];
        B[q] = hr[cur];
      }
      CK(coldots(A, B, nq, kp, 0, n, h->rmm_g + (size_t)t0 * kp, h->partials, h->partial_cap, h->f64, s));
    }
    for (int j = 0; j < 16; ++j) lam[j] = frozen[j] ? 0.0 : 1.0;
    CK(cudaMemcpyAsync(h->rmm_frozen, frozen.data(), sizeof(int) * 16, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->rmm_lam, lam.data(), sizeof(double) * 16, cudaMemcpyHostToDevice, s));
    k_diis<<<1, 32, 0, s>>>(h->rmm_g, d, cur, nh, h->rmm_G, h->rmm_frozen, k, kp, h->rmm_coef, h->rmm_status);
    count_launch();
    CK(cudaGetLastError());
    CK(combine_diag(Xb, nullptr, nullptr, Lx, h->rmm_coef, kp, 0, n, h->f64, s));   // x_bar
    CK(combine_diag(Rb, nullptr, nullptr, Lr, h->rmm_coef, kp, 0, n, h->f64, s));   // r_bar
    const int next = (cur + 1) % d;
    k_rmm_step<<<static_cast<unsigned>((n * kp + 255) / 256), 256, 0, s>>>(
        Xb, Rb, h->dDiag, h->rmm_th, h->rmm_lam, (float)h->opt.precond_clamp, k, kp, n, hx[next]);
    count_launch();
    CK(cudaGetLastError());
    CKS(normalise(hx[next]));
    cur = next;
    if (h->opt.timing) CKS(collect_timing(h));
  }
  return SPPC_OK;
}

bool all_converged(const sppc_ctx* h, double tol) {
  for (double r : h->resid)
    if (!(r <= tol)) return false;
  return true;
}


}  // namespace sppc::drv
