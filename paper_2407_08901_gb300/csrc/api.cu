// C ABI of the SPPC eigensolver (Algorithm 2 of the paper), part 2: the
// stepwise and whole-solve entry points, the products with H, the state
// queries, the stand-alone dense entry points and the learned proposal's.
//
// The driver owns all device memory and sequences the kernels of k_spmm.cu,
// k_dense.cu, k_gram_tc.cu, k_update_tc.cu, k_small.cu and k_minres.cu on the
// caller's stream.  Host work is limited to argument checks, building the
// layouts once in sppc_create (api_create.cu), scalar bookkeeping and one small
// device->host copy per correction order (the convergence test of Alg. 2) or
// per few MINRES iterations.
#include "driver.h"

// =================================================================== C ABI
extern "C" {

sppc_status sppc_small_syev(const double* S, int32_t m, int32_t lds, int32_t nev, double* theta, double* V,
                            int32_t ldv, int32_t flags, void* stream) {
  if (!S || !theta || !V || m < 1 || m > 144 || nev < 1 || nev > 16 || nev > m || lds < m || ldv < nev ||
      (flags & ~1))
    return fail(nullptr, SPPC_ERR_ARG,
                "sppc_small_syev: bad arguments (1 <= m <= 144, 1 <= nev <= min(16, m), flags 0 or 1)");
  const cudaError_t e =
      syev_lowest(S, lds, m, nev, theta, V, ldv, (flags & 1) != 0, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(nullptr, SPPC_ERR_CUDA, "sppc_small_syev: %s", cudaGetErrorString(e));
  return SPPC_OK;
}

sppc_status sppc_block_gram(const double* A, int32_t nblocks, const double* B, int64_t n, int32_t flags, double* G,
                            void* stream) {
  if (((!A || !B) && n > 0) || !G || nblocks < 1 || nblocks > kMaxBlocks || n < 0 || n >= ((int64_t)1 << 40) ||
      (flags & ~3))
    return fail(nullptr, SPPC_ERR_ARG, "sppc_block_gram: bad arguments (1 <= nblocks <= %d, flags in 0..3)",
                kMaxBlocks);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool tc = (flags & 1) != 0, df = (flags & 2) != 0;
  // partial sums: the CUDA-core Gram cuts at >= 2048 rows when its finer cut does not fit
  const int64_t cap = ((n + 1023) / 1024 + 1) * (int64_t)nblocks * 64;
  float2* partials = nullptr;
  float2* Adf = nullptr;
  int* err = nullptr;
  cudaError_t e = cudaMalloc(&partials, sizeof(float2) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int) * 16);  // flag, then B's column exponents
  if (e == cudaSuccess && df) e = cudaMalloc(&Adf, sizeof(float2) * ((size_t)nblocks + 1) * (size_t)(n ? n : 1) * 8);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  BlockList L;
  L.n = nblocks;
  const float2* Bs = reinterpret_cast<const float2*>(B);
  if (e == cudaSuccess && df) {
    for (int a = 0; a <= nblocks && e == cudaSuccess; ++a)
      e = f64_to_df(a < nblocks ? A + (int64_t)a * n * 8 : B, 8, 8, Adf + (int64_t)a * n * 8, 8, 0, n, false, s);
    Bs = Adf + (int64_t)nblocks * n * 8;
  }
  for (int a = 0; a < nblocks; ++a)
    L.p[a] = df ? Adf + (int64_t)a * n * 8 : reinterpret_cast<const float2*>(A + (int64_t)a * n * 8);
  unsigned char* Ad = nullptr;
  if (e == cudaSuccess && tc)
    e = cudaMalloc(&Ad, (size_t)((nblocks + 15) / 16) * (size_t)qdigits_group_bytes(n) + 16);
  for (int a = 0; a < nblocks && tc && e == cudaSuccess; ++a) e = qcut(L.p[a], n, qdigits_block(Ad, n, a), !df, err, s);
  if (e == cudaSuccess)
    e = tc ? gram_tc(Ad, nblocks, Bs, n, G, partials, cap, !df, err, err + 8, s)
           : gram(L, Bs, 8, 0, n, G, partials, cap, !df, s);
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(partials);
  cudaFree(err);
  cudaFree(Adf);
  cudaFree(Ad);
  if (e != cudaSuccess) return fail(nullptr, SPPC_ERR_CUDA, "sppc_block_gram: %s", cudaGetErrorString(e));
  if (flag & 2) return fail(nullptr, SPPC_ERR_TIMEOUT, "sppc_block_gram: a tensor-core pipeline wait timed out");
  if (flag & 1)
    return fail(nullptr, SPPC_ERR_NAN, "sppc_block_gram: an entry of A has |a| >= 2, or a value is not finite");
  return SPPC_OK;
}

sppc_status sppc_block_update(const double* A, int32_t nblocks, const double* C, const double* alpha, const double* X,
                              double* Y, int64_t n, int32_t flags, void* stream) {
  if (((!A || !Y) && n > 0) || !C || nblocks < 1 || nblocks > kMaxBlocks || n < 0 || n >= ((int64_t)1 << 40) ||
      (flags & ~3))
    return fail(nullptr, SPPC_ERR_ARG, "sppc_block_update: bad arguments (1 <= nblocks <= %d, flags in 0..3)",
                kMaxBlocks);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool tc = (flags & 1) != 0, df = (flags & 2) != 0;
  const int64_t nn = n ? n : 1;
  float2* buf = nullptr;  // double-float copies: A blocks, X, Y, then C and alpha
  int* err = nullptr;
  unsigned char* Ad = nullptr;
  double* ones = nullptr;  // alpha = 1 when X comes without alpha
  cudaError_t e = cudaMalloc(&err, sizeof(int) * 16);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int) * 16, s);
  if (e == cudaSuccess && X && !alpha) {
    const double h1[8] = {1, 1, 1, 1, 1, 1, 1, 1};
    e = cudaMalloc(&ones, sizeof(double) * 8);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ones, h1, sizeof(h1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    alpha = ones;
  }
  if (e == cudaSuccess && df) e = cudaMalloc(&buf, sizeof(float2) * (((size_t)nblocks + 2) * nn * 8 + 64 * nblocks + 8));
  const float2* Ls[kMaxBlocks];
  const float2 *Cs = reinterpret_cast<const float2*>(C), *as = reinterpret_cast<const float2*>(alpha),
               *Xs = reinterpret_cast<const float2*>(X);
  float2* Ys = reinterpret_cast<float2*>(Y);
  for (int a = 0; a < nblocks; ++a) Ls[a] = reinterpret_cast<const float2*>(A + (int64_t)a * n * 8);
  if (e == cudaSuccess && df) {
    float2* Xd = buf + (int64_t)nblocks * nn * 8;
    float2* Yd = Xd + nn * 8;
    float2* Cd = Yd + nn * 8;
    float2* ad = Cd + 64 * nblocks;
    for (int a = 0; a < nblocks && e == cudaSuccess; ++a) {
      float2* d = buf + (int64_t)a * nn * 8;
      e = f64_to_df(A + (int64_t)a * n * 8, 8, 8, d, 8, 0, n, false, s);
      Ls[a] = d;
    }
    if (e == cudaSuccess) e = f64_to_df(C, 8, 8, Cd, 8, 0, 8 * nblocks, false, s);
    if (e == cudaSuccess && alpha) e = f64_to_df(alpha, 8, 8, ad, 8, 0, 1, false, s);
    if (e == cudaSuccess && X) e = f64_to_df(X, 8, 8, Xd, 8, 0, n, false, s);
    Cs = Cd;
    as = alpha ? ad : nullptr;
    Xs = X ? Xd : nullptr;
    Ys = Yd;
  }
  if (e == cudaSuccess && tc) {
    const size_t bytes = (size_t)((nblocks + 15) / 16) * (size_t)qdigits_group_bytes(n) + 16;
    e = cudaMalloc(&Ad, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(Ad, 0, bytes, s);
    for (int a = 0; a < nblocks && e == cudaSuccess; ++a) e = qcut(Ls[a], n, qdigits_block(Ad, n, a), !df, err, s);
  }
  if (e == cudaSuccess) {
    if (tc) {
      e = update_tc(Ad, nblocks, Cs, as, Xs, Ys, n, !df, err, s);
    } else {
      BlockList L;
      L.n = nblocks;
      for (int a = 0; a < nblocks; ++a) L.p[a] = Ls[a];
      e = update(Ys, Xs, as, L, Cs, 8, 0, n, !df, s);
    }
  }
  if (e == cudaSuccess && df) e = df_to_f64(Ys, 8, Y, 8, 8, 0, n, false, s);
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(buf);
  cudaFree(err);
  cudaFree(Ad);
  cudaFree(ones);
  if (e != cudaSuccess) return fail(nullptr, SPPC_ERR_CUDA, "sppc_block_update: %s", cudaGetErrorString(e));
  if (flag & 2) return fail(nullptr, SPPC_ERR_TIMEOUT, "sppc_block_update: a tensor-core pipeline wait timed out");
  if (flag & 1)
    return fail(nullptr, SPPC_ERR_NAN, "sppc_block_update: an entry of A has |a| >= 2, or a value is not finite");
  return SPPC_OK;
}


sppc_status sppc_spmm(sppc_handle h, const double* X, int64_t ldx, double* Y, int64_t ldy, int32_t ncols,
                      void* stream) {
  if (!h) return fail(nullptr, SPPC_ERR_ARG, "NULL handle");
  if (!X || !Y || ncols < 1 || ncols > 8 || ldx < ncols || ldy < ncols)
    return fail(h, SPPC_ERR_ARG, "sppc_spmm: bad arguments (ncols in [1,8], ld >= ncols)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->stream = s;
  const int kp = (ncols + 1) / 2 * 2;
  CK(f64_to_df(X, ldx, ncols, h->T1, kp, 0, h->n, h->f64, s));
  if (h->opt.precision > 0 && (kp == 4 || kp == 8))
    CK(spmm_f32(h->H, h->val32, h->val16, h->diag32, h->T1, h->X32, h->T2, kp, s));
  else
    CK(spmm(h->H, kp, h->T1, h->T2, Epi{}, s));
  CK(df_to_f64(h->T2, kp, Y, ldy, ncols, 0, h->n, h->f64, s));
  return SPPC_OK;
}

sppc_status sppc_spmm_host(sppc_handle h, const double* X, int64_t ldx, double* Y, int64_t ldy, int32_t ncols,
                           void* stream) {
  if (!h) return fail(nullptr, SPPC_ERR_ARG, "NULL handle");
  if (!X || !Y || ncols < 1 || ncols > 8 || ldx < ncols || ldy < ncols)
    return fail(h, SPPC_ERR_ARG, "sppc_spmm_host: bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->stream = s;
  if (!h->stageX) {
    CK(dalloc(h, &h->stageX, (size_t)h->n * 8));
    CK(dalloc(h, &h->stageY, (size_t)h->n * 8));
  }
  double* dX = h->stageX;
  double* dY = h->stageY;
  if (h->H.tma_flag) CK(cudaMemsetAsync(h->H.tma_flag, 0, sizeof(int), s));
  CK(cudaMemcpy2DAsync(dX, sizeof(double) * ncols, X, sizeof(double) * ldx, sizeof(double) * ncols, h->n,
                       cudaMemcpyHostToDevice, s));
  CKS(sppc_spmm(h, dX, ncols, dY, ncols, ncols, stream));
  CK(cudaMemcpy2DAsync(Y, sizeof(double) * ldy, dY, sizeof(double) * ncols, sizeof(double) * ncols, h->n,
                       cudaMemcpyDeviceToHost, s));
  int tmo = 0;
  CK(spmm_tma_read_timeout(h->H, &tmo, s));
  CK(cudaStreamSynchronize(s));
  if (tmo) return fail(h, SPPC_ERR_TIMEOUT, "SpMM: a shared-memory pipeline wait timed out");
  return SPPC_OK;
}

sppc_status sppc_start(sppc_handle h, double* theta, double* resid, void* stream) {
  if (!h) return fail(nullptr, SPPC_ERR_ARG, "NULL handle");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->stream = s;
  h->stats = sppc_stats{};
  h->pending.clear();
  h->evnext = 0;
  h->rec.clear();
  h->p = 0;
  h->started = false;
  h->corrected = false;
  h->in_refine = false;
  h->t_ready = false;
  h->t_last = nullptr;
  if (h->H.tma_flag) CK(cudaMemsetAsync(h->H.tma_flag, 0, sizeof(int), s));
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (h->opt.timing) {
    t0 = next_event(h);
    t1 = next_event(h);
    CK(cudaEventRecord(t0, s));
  }
  CKS(small_eigensolve(h));
  if (h->opt.timing) {
    CK(cudaEventRecord(t1, s));
    CK(cudaEventSynchronize(t1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, t0, t1));
    h->stats.small_eig_ms += ms;
    h->evnext = 0;
  }
  const int kp = h->kp;
  const int64_t n = h->n;
  // Q^(0) = Psi^(0) = [psi_hat; 0] (Eq. EP_small), W_0 = H Q^(0)
  h->qd_valid = 0;
  CK(fill_zero(h->Q, n * kp, s));
  CK(cudaMemcpyAsync(h->Q, h->psi_hat, sizeof(float2) * h->n1 * kp, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->Psi, h->Q, sizeof(float2) * n * kp, cudaMemcpyDeviceToDevice, s));
  CKS(big_spmm(h, h->Q, h->W, kp));
  h->stats.spmv_h += h->k;
  CKS(rr_core(h, 0, false, nullptr, 0));
  // H Psi^(0) = W_0
  CK(cudaMemcpyAsync(h->HPsi, h->W, sizeof(float2) * n * kp, cudaMemcpyDeviceToDevice, s));
  OrderRec r;
  r.E = h->E0;
  r.theta = h->theta;
  r.resid = h->resid;
  h->rec.push_back(r);
  if (h->opt.timing) CKS(collect_timing(h));
  h->started = true;
  if (theta) std::copy(h->theta.begin(), h->theta.end(), theta);
  if (resid) std::copy(h->resid.begin(), h->resid.end(), resid);
  return SPPC_OK;
}

sppc_status sppc_correct(sppc_handle h, void* stream) {
  PhaseRange nvtx_range("sppc_correct");
  if (!h) return fail(nullptr, SPPC_ERR_ARG, "NULL handle");
  if (!h->started || h->corrected || h->in_refine)
    return fail(h, SPPC_ERR_STATE, "sppc_correct needs sppc_start / rayleigh_ritz first (and no refinement yet)");
  if (h->p + 1 > h->pmax) return fail(h, SPPC_ERR_STATE, "p_max orders already done");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->stream = s;
  const int p = h->p + 1;
  const int k = h->k, kp = h->kp;
  const int64_t n = h->n, n1 = h->n1;
  float2* c = h->dCoef;
  float2* Psip = blk(h->Psi, n, kp, p);
  float2* Psim1 = blk(h->Psi, n, kp, p - 1);
  OrderRec rec;
  // coefficients of Eq. exp_seq2 need E^(p); compute the small-space part first
  // V Psi^(p-1)_1 = (H Psi^(p-1))_1 - H0_hat Psi^(p-1)_1  (Eq. avoid_SpMV2)
  {
    Epi e;
    e.alpha = c + kNegOnes;
    e.gamma = c + kOnes;
    e.Z = h->HPsi;
    CK(spmm11(h, kp, Psim1, h->vps, e, s));
    h->stats.spmv_h11 += k;
  }
  // E^(p) = psi_hat^T (V Psi^(p-1))_1 = (Psi^(p-1))^T V Psi^(0) (Eq. exp_seq, V symmetric)
  {
    const float2* A[1] = {h->psi_hat};
    const float2* B[1] = {h->vps};
    CK(coldots(A, B, 1, kp, 0, n1, h->dE + (size_t)p * kp, h->partials, h->partial_cap, h->f64, s));
  }
  k_rhs_coefs<<<1, 32, 0, s>>>(h->dE, p, k, kp, c, h->f64); count_launch();
  CK(cudaGetLastError());
  // rows >= n1: Psi^(p)_2 = -b2 / E^(0) (Eq. sm_first)
  {
    BlockList L;
    L.n = 0;
    for (int l = 1; l <= p - 2; ++l) L.p[L.n++] = blk(h->Psi, n, kp, l);
    CK(combine_diag(Psip, h->HPsi, c + kInvE0, L, c + kRhsBig, kp, n1, n, h->f64, s));
  }
  // rows < n1: b1 = -V Psi^(p-1)_1 + E^(p) psi_hat + sum_{l=1}^{p-2} E^(p-l) Psi^(l)_1
  {
    BlockList L;
    L.n = 0;
    L.p[L.n++] = h->psi_hat;
    for (int l = 1; l <= p - 2; ++l) L.p[L.n++] = blk(h->Psi, n, kp, l);
    CK(combine_diag(h->b1, h->vps, c + kNegOnes, L, c + kRhsSmall, kp, 0, n1, h->f64, s));
  }
  // deflate psi_hat_k (Eq. sm_lin_proj)
  {
    const float2* A[1] = {h->psi_hat};
    const float2* B[1] = {h->b1};
    CK(coldots(A, B, 1, kp, 0, n1, h->dDots, h->partials, h->partial_cap, h->f64, s));
    k_neg_dots_to_coef<<<1, 32, 0, s>>>(h->dDots, k, kp, c + kDefl, h->f64); count_launch();
    CK(cudaGetLastError());
    CK(combine_diag(h->b1, h->b1, c + kOnes, one(h->psi_hat), c + kDefl, kp, 0, n1, h->f64, s));
  }
  // small solves (H0_hat - E_k^(0)) x1 = b1; at p = 1 b1 = 0 since V11 = 0 (Eq. first_PC)
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (h->opt.timing) {
    t0 = next_event(h);
    t1 = next_event(h);
    CK(cudaEventRecord(t0, s));
  }
  if (p == 1) {
    CK(fill_zero(Psip, n1 * kp, s));
    rec.iters.assign(k, 0);
  } else {
    CKS(minres(h, rec.iters));
    CK(cudaMemcpyAsync(Psip, h->mx, sizeof(float2) * n1 * kp, cudaMemcpyDeviceToDevice, s));
  }
  if (h->opt.timing) {
    CK(cudaEventRecord(t1, s));
    CK(cudaEventSynchronize(t1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, t0, t1));
    h->stats.minres_ms += ms;
  }
  // block Gram-Schmidt twice (Eq. blkGS) + CholeskyQR2 (Eq. QR), q^(p) -> Q block p
  std::vector<double> dd(2 * kp);
  CKS(orth_append(h, Psip, p, dd.data(), false));
  std::vector<double> ep(kp);
  CK(cudaMemcpyAsync(ep.data(), h->dE + (size_t)p * kp, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  rec.E.assign(ep.begin(), ep.begin() + k);
  rec.angle.resize(k);
  for (int j = 0; j < k; ++j) rec.angle[j] = std::sqrt(std::max(dd[kp + j], 0.0) / std::max(dd[j], 1e-300));
  h->rec.push_back(rec);
  h->p = p;
  h->corrected = true;
  return SPPC_OK;
}

sppc_status sppc_rayleigh_ritz(sppc_handle h, double* theta, double* resid, void* stream) {
  if (!h) return fail(nullptr, SPPC_ERR_ARG, "NULL handle");
  if (!h->corrected) return fail(h, SPPC_ERR_STATE, "sppc_rayleigh_ritz needs sppc_correct first");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->stream = s;
  const int p = h->p, kp = h->kp;
  const int64_t n = h->n;
  // W_p = H q^(p): the k SpMVs of the order
  CKS(big_spmm(h, blk(h->Q, n, kp, p), blk(h->W, n, kp, p), kp));
  h->stats.spmv_h += h->k;
  CKS(rr_core(h, p, false, nullptr, 0));
  // H Psi^(p) = W_{0..p-1} C + W_p R (Eq. HPsip)
  CK(wupdate(h, p + 1, h->HPsi, nullptr, nullptr, h->dRecycle, s));
  OrderRec& r = h->rec.back();
  r.theta = h->theta;
  r.resid = h->resid;
  h->corrected = false;
  h->stats.orders = p;
  if (h->opt.timing) CKS(collect_timing(h));
  if (theta) std::copy(h->theta.begin(), h->theta.end(), theta);
  if (resid) std::copy(h->resid.begin(), h->resid.end(), resid);
  return SPPC_OK;
}

// Mixed precision: the k Ritz vectors z_j = Q Y_j, their product with H in
// double-float (the FP32-rounded matrix, exact to double-float), Rayleigh
// quotients theta_j = z^T H z / z^T z and residuals ||H z - theta z|| / |theta|.
// Replaces the Ritz values and residuals of the last Rayleigh-Ritz step, whose
// H-products were FP32.
sppc_status verify_df(sppc_ctx* h) {
  cudaStream_t s = h->stream;
  const int k = h->k, kp = h->kp;
  const int64_t n = h->n;
  float2* c = h->dCoef;
  CK(update(h->T1, nullptr, nullptr, blocks(h->Q, n, kp, 0, h->p + 1), h->dY, kp, 0, n, h->f64, s));
  CK(spmm(h->H, kp, h->T1, h->T2, Epi{}, s));
  {
    const float2* A[2] = {h->T1, h->T1};
    const float2* B[2] = {h->T2, h->T1};
    CK(coldots(A, B, 2, kp, 0, n, h->dDots, h->partials, h->partial_cap, h->f64, s));
  }
  std::vector<double> dd(2 * kp);
  CK(cudaMemcpyAsync(dd.data(), h->dDots, sizeof(double) * 2 * kp, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<double> th(k), negth(kp, 0.0);
  for (int j = 0; j < k; ++j) {
    th[j] = dd[j] / dd[kp + j];
    negth[j] = -th[j];
  }
  CK(cudaMemcpyAsync(h->dDots + 2 * kp, negth.data(), sizeof(double) * kp, cudaMemcpyHostToDevice, s));
  CK(to_df(h->dDots + 2 * kp, c + kDefl, kp, 1.0, h->f64, s));
  CK(combine_diag(h->T2, h->T2, c + kOnes, one(h->T1), c + kDefl, kp, 0, n, h->f64, s));  // H z - theta z
  {
    const float2* A[1] = {h->T2};
    const float2* B[1] = {h->T2};
    CK(coldots(A, B, 1, kp, 0, n, h->dDots, h->partials, h->partial_cap, h->f64, s));
  }
  std::vector<double> r2(kp);
  CK(cudaMemcpyAsync(r2.data(), h->dDots, sizeof(double) * kp, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->theta = th;
  h->resid.assign(k, 0.0);
  for (int j = 0; j < k; ++j) h->resid[j] = std::sqrt(std::max(r2[j], 0.0) / std::max(dd[kp + j], 1e-300)) /
                                           std::fabs(th[j]);
  return SPPC_OK;
}

// One SPPC order's Rayleigh-Ritz step (the order is h->p, corrected), with the
// next order's correction overlapped on a second stream when `next`: the
// correction needs only H Psi^(p) (the recycled product), not the Ritz pairs,
// and its small-space MINRES leaves most of the GPU idle while the Gram,
// projected eigensolve and Ritz residuals of this order run beside it.  The
// correction uses its own reduction scratch (partials2, dDots2); everything else
// it writes (Psi and Q block p+1, the MINRES vectors, its coefficient slots) the
// Rayleigh-Ritz step does not touch.  Returns in *pre whether the next order's
// correction is done (then h->p = order + 1 and h->corrected is set).
static sppc_status overlap_order(sppc_ctx* h, bool next, bool* pre) {
  cudaStream_t s = h->stream;
  const int p = h->p, kp = h->kp;
  const int64_t n = h->n;
  *pre = false;
  if (next && !h->stream2) {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_b, cudaEventDisableTiming);
    if (e == cudaSuccess) e = dalloc(h, &h->partials2, (size_t)h->partial_cap);
    if (e == cudaSuccess) e = dalloc(h, &h->dDots2, 64);
    if (e == cudaSuccess) e = cudaMallocHost(&h->pinned, sizeof(double) * 32);
    if (e != cudaSuccess) return fail(h, SPPC_ERR_CUDA, "overlap setup: %s", cudaGetErrorString(e));
  }
  // W_p = H q^(p), then H Psi^(p) = W_{0..p-1} C + W_p R (Eq. HPsip): all the
  // next correction needs
  CKS(big_spmm(h, blk(h->Q, n, kp, p), blk(h->W, n, kp, p), kp));
  h->stats.spmv_h += h->k;
  CK(wupdate(h, p + 1, h->HPsi, nullptr, nullptr, h->dRecycle, s));
  if (next) CK(cudaEventRecord(h->ev_a, s));  // the correction waits for H Psi^(p) only
  CKS(rr_core(h, p, false, nullptr, 0, nullptr, nullptr, next));
  const size_t rec_p = h->rec.size() - 1;
  h->corrected = false;
  h->stats.orders = p;
  if (next) {
    CK(cudaStreamWaitEvent(h->stream2, h->ev_a, 0));
    float2* part0 = h->partials;
    double* dots0 = h->dDots;
    h->partials = h->partials2;
    h->dDots = h->dDots2;
    const sppc_status st = sppc_correct(h, h->stream2);
    h->partials = part0;
    h->dDots = dots0;
    h->stream = s;
    CK(cudaEventRecord(h->ev_b, h->stream2));
    CK(cudaStreamWaitEvent(s, h->ev_b, 0));
    if (st != SPPC_OK) return st;
    *pre = true;
    CKS(rr_finish(h, s));
  }
  OrderRec& r = h->rec[rec_p];
  r.theta = h->theta;
  r.resid = h->resid;
  if (h->opt.timing) CKS(collect_timing(h));
  return SPPC_OK;
}

sppc_status sppc_solve(sppc_handle h, double tol, int32_t p_max, double* theta, double* Z, int64_t ldz,
                       double* resid, sppc_stats* stats, void* stream) {
  if (!h) return fail(nullptr, SPPC_ERR_ARG, "NULL handle");
  if (tol <= 0) tol = h->opt.tol;
  if (p_max < 0) p_max = h->pmax;
  if (p_max > h->pmax) return fail(h, SPPC_ERR_ARG, "p_max exceeds the p_max given at create");
  if (Z && ldz < h->k) return fail(h, SPPC_ERR_ARG, "ldz < k");
  if (h->opt.hybrid && h->pmax < 3) return fail(h, SPPC_ERR_ARG, "the continuation needs p_max >= 3");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (h->opt.timing) {
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    cudaEventRecord(t0, s);
  }
  h->f32_products = (h->opt.precision > 0);
  CKS(sppc_start(h, nullptr, nullptr, stream));
  bool conv = all_converged(h, tol);
  const int sppc_orders = h->opt.hybrid ? std::min(p_max, h->opt.switch_order) : p_max;
  // SPPC orders; each order's Rayleigh-Ritz step overlaps the next correction
  bool pending = false;  // the next order's correction is already done
  while (!conv && h->p + (pending ? 0 : 1) <= sppc_orders) {
    if (!pending) CKS(sppc_correct(h, stream));
    const int p = h->p;
    CKS(overlap_order(h, p + 1 <= sppc_orders, &pending));
    conv = all_converged(h, tol);
    // the paper's switch rule (Sec. 6): leave SPPC once the scaled residual of
    // some eigenpair stops dropping (ratio to the previous order above switch_stall)
    bool stalled = false;
    if (h->opt.hybrid && h->opt.switch_stall > 0.0 && p >= 2 && (size_t)p < h->rec.size()) {
      const std::vector<double>& r0 = h->rec[p - 1].resid;
      for (int j = 0; j < h->k && j < (int)r0.size(); ++j)
        stalled |= h->resid[j] > h->opt.switch_stall * r0[j];
    }
    if ((conv || stalled) && pending) {
      // converged (or switching) at order p: drop the overlapped correction of order p + 1
      h->rec.pop_back();
      h->p = p;
      h->corrected = false;
      pending = false;
    }
    if (stalled || (!pending && h->p >= sppc_orders)) break;
  }
  h->stats.orders = h->p;
  if (h->opt.hybrid == 2) {
    h->stats.switched_at = h->p;
    h->in_refine = true;
    if (!conv) CKS(rmm_run(h, tol));
    conv = all_converged(h, tol);
  } else if (h->opt.hybrid) {
    h->stats.switched_at = h->p;
    h->in_refine = true;
    // mixed precision: the FP32 phase stops at max(tol, 1e-6) or when its largest
    // residual estimate has not dropped by 10% in 8 steps (the FP32 products'
    // floor is about 2^-24 ||H|| / |theta|); the double-float phase below finishes
    const double tol_phase = h->f32_products ? std::max(tol, 1e-6) : tol;
    double best = 1e300;
    int since_best = 0;
    conv = all_converged(h, tol_phase);
    while (!conv && h->stats.refine_steps < h->opt.hybrid_maxit) {
      CKS(refine_step(h));
      conv = all_converged(h, tol_phase);
      if (h->f32_products) {
        const double worst = *std::max_element(h->resid.begin(), h->resid.end());
        if (worst < 0.9 * best) {
          best = worst;
          since_best = 0;
        } else if (++since_best >= 8) {
          break;
        }
      }
    }
    conv = all_converged(h, tol);
  }
  const bool fresh = h->opt.precision > 0 && h->opt.hybrid && h->p >= 1 && h->nev >= 2 * h->k;
  h->f32_products = false;
  if (fresh) {
    // Mixed precision: the residuals of the FP32 phase are estimates and its W
    // blocks carry FP32 errors.  Restart from the 2k lowest Ritz vectors with
    // their products recomputed in double-float, and continue with double-float
    // products until the (now exact) residuals meet tol.
    CKS(restart(h, true));
    CKS(rr_core(h, h->p, false, nullptr, 0, h->HPsi, t_diag(h)));
    h->t_ready = true;
    conv = all_converged(h, tol);
    while (!conv && h->stats.refine_df < h->opt.hybrid_maxit) {
      CKS(refine_step(h));
      conv = all_converged(h, tol);
      h->stats.refine_df += 1;
    }
  }
  if (Z) {
    if (h->opt.hybrid == 2 && h->rmm_x && h->in_refine)
      CK(df_to_f64(h->rmm_x, h->kp, Z, ldz, h->k, 0, h->n, h->f64, s));   // each pair's own vector
    else
      CKS(rr_core(h, h->p, true, Z, ldz));
  }
  if (h->opt.precision > 0 && !fresh) {
    // plain SPPC in mixed precision: Rayleigh quotients and residuals of the Ritz
    // vectors from double-float products
    CKS(verify_df(h));
    conv = all_converged(h, tol);
  }
  h->stats.converged = conv ? 1 : 0;
  if (h->opt.timing) {
    cudaEventRecord(t1, s);
    cudaEventSynchronize(t1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    h->stats.total_ms = ms;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    h->stats.dense_ms = h->stats.total_ms - h->stats.spmm_ms - h->stats.minres_ms - h->stats.small_eig_ms;
  }
  if (theta) std::copy(h->theta.begin(), h->theta.end(), theta);
  if (resid) std::copy(h->resid.begin(), h->resid.end(), resid);
  if (stats) *stats = h->stats;
  return conv ? SPPC_OK : SPPC_NOT_CONVERGED;
}

sppc_status sppc_refine_step(sppc_handle h, double* theta, double* resid, void* stream) {
  if (!h) return fail(nullptr, SPPC_ERR_ARG, "NULL handle");
  if (!h->started || h->corrected) return fail(h, SPPC_ERR_STATE, "sppc_refine_step needs a finished Rayleigh-Ritz step");
  if (h->pmax < 3) return fail(h, SPPC_ERR_ARG, "the continuation needs p_max >= 3");
  h->stream = static_cast<cudaStream_t>(stream);
  if (!h->in_refine) h->stats.switched_at = h->p;
  h->in_refine = true;
  CKS(refine_step(h));
  if (theta) std::copy(h->theta.begin(), h->theta.end(), theta);
  if (resid) std::copy(h->resid.begin(), h->resid.end(), resid);
  return SPPC_OK;
}

sppc_status sppc_order_info(sppc_handle h, int32_t p, double* E, double* angle, double* theta, double* resid,
                            int32_t* minres_iters) {
  if (!h) return fail(nullptr, SPPC_ERR_ARG, "NULL handle");
  if (p < 0 || p >= (int)h->rec.size()) return fail(h, SPPC_ERR_ARG, "order %d not available", p);
  const OrderRec& r = h->rec[p];
  const int k = h->k;
  auto cp = [&](const std::vector<double>& v, double* o) {
    if (!o) return;
    for (int j = 0; j < k; ++j) o[j] = j < (int)v.size() ? v[j] : 0.0;
  };
  cp(r.E, E);
  cp(r.angle, angle);
  cp(r.theta, theta);
  cp(r.resid, resid);
  if (minres_iters)
    for (int j = 0; j < k; ++j) minres_iters[j] = j < (int)r.iters.size() ? r.iters[j] : 0;
  return SPPC_OK;
}

sppc_status sppc_get_stats(sppc_handle h, sppc_stats* stats) {
  if (!h || !stats) return fail(h, SPPC_ERR_ARG, "NULL argument");
  *stats = h->stats;
  return SPPC_OK;
}

sppc_status sppc_get_state(sppc_handle h, int32_t which, double* out, int64_t count) {
  if (!h || !out) return fail(h, SPPC_ERR_ARG, "NULL argument");
  const int k = h->k, kp = h->kp;
  const int64_t n = h->n, n1 = h->n1;
  cudaStream_t s = h->stream;
  const int nbk = h->p + 1;
  auto dl = [&](const float2* src, int64_t rows, int ncols, double* dst, int64_t ld) -> sppc_status {
    double* tmp = nullptr;
    CK(cudaMalloc(&tmp, sizeof(double) * rows * ncols));
    CK(df_to_f64(src, kp, tmp, ncols, ncols, 0, rows, h->f64, s));
    std::vector<double> hbuf((size_t)rows * ncols);
    CK(cudaMemcpyAsync(hbuf.data(), tmp, sizeof(double) * rows * ncols, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    cudaFree(tmp);
    for (int64_t r = 0; r < rows; ++r)
      for (int c2 = 0; c2 < ncols; ++c2) dst[r * ld + c2] = hbuf[(size_t)r * ncols + c2];
    return SPPC_OK;
  };
  switch (which) {
    case 0:
      if (count < n1 * k) return fail(h, SPPC_ERR_ARG, "buffer too small");
      return dl(h->psi_hat, n1, k, out, k);
    case 1:
    case 2: {
      const int64_t m = (int64_t)k * nbk;
      if (count < n * m) return fail(h, SPPC_ERR_ARG, "buffer too small");
      for (int a = 0; a < nbk; ++a) {
        std::vector<double> tmp((size_t)n * k);
        CKS(dl(blk(which == 1 ? h->Q : h->W, n, kp, a), n, k, tmp.data(), k));
        for (int64_t r = 0; r < n; ++r)
          for (int j = 0; j < k; ++j) out[r * m + a * k + j] = tmp[(size_t)r * k + j];
      }
      return SPPC_OK;
    }
    case 3: {
      const int m = k * nbk;
      if (count < (int64_t)m * m) return fail(h, SPPC_ERR_ARG, "buffer too small");
      std::vector<double> hbuf((size_t)h->mmax * h->mmax);
      CK(cudaMemcpyAsync(hbuf.data(), h->dHt, sizeof(double) * hbuf.size(), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) out[i * m + j] = hbuf[(size_t)i * h->mmax + j];
      return SPPC_OK;
    }
    case 4:
      if (count < n * k) return fail(h, SPPC_ERR_ARG, "buffer too small");
      return dl(blk(h->Psi, n, kp, h->p), n, k, out, k);
    case 5:
      if (count < k) return fail(h, SPPC_ERR_ARG, "buffer too small");
      for (int j = 0; j < k; ++j) out[j] = j < (int)h->E0.size() ? h->E0[j] : 0.0;
      return SPPC_OK;
    case 6:
    case 7:
      if (!h->Tprop) return fail(h, SPPC_ERR_STATE, "no proposal block yet");
      if (count < n * k) return fail(h, SPPC_ERR_ARG, "buffer too small");
      return dl(which == 6 ? h->Tprop : h->Tplain, n, k, out, k);
    case 8:
      if (!h->t_last) return fail(h, SPPC_ERR_STATE, "no continuation step yet");
      if (count < n * k) return fail(h, SPPC_ERR_ARG, "buffer too small");
      return dl(h->t_last, n, k, out, k);
    default:
      return fail(h, SPPC_ERR_ARG, "unknown state id %d", which);
  }
}

sppc_status sppc_get_layout(sppc_handle h, int64_t* n_slices, int64_t* slice_ptr, int32_t* slice_rows,
                            int64_t* n11_slices, int64_t* h11_slice_ptr, int32_t* h11_slice_rows, int32_t* n_chunks,
                            int64_t* chunk_slice) {
  if (!h) return fail(nullptr, SPPC_ERR_ARG, "NULL handle");
  if (n_chunks) *n_chunks = h->H.nchunks;
  if (chunk_slice) std::copy(h->h_chunk_slice.begin(), h->h_chunk_slice.end(), chunk_slice);
  if (n_slices) *n_slices = h->h_slices;
  if (n11_slices) *n11_slices = h->h11_slices;
  if (slice_ptr) std::copy(h->h_slice_ptr.begin(), h->h_slice_ptr.end(), slice_ptr);
  if (slice_rows) std::copy(h->h_slice_rows.begin(), h->h_slice_rows.end(), slice_rows);
  if (h11_slice_ptr) std::copy(h->h11_slice_ptr.begin(), h->h11_slice_ptr.end(), h11_slice_ptr);
  if (h11_slice_rows) std::copy(h->h11_slice_rows.begin(), h->h11_slice_rows.end(), h11_slice_rows);
  return SPPC_OK;
}

// ---------------------------------------------------- learned proposal (C-ABI)
static_assert(kNetParams == SPPC_NET_PARAMS && kNetFeatures == SPPC_NET_FEATURES, "network layout");
sppc_status sppc_set_proposal(sppc_handle h, const float* params, const float* mu, const float* sd) {
  if (!h || !params || !mu || !sd) return fail(h, SPPC_ERR_ARG, "NULL argument");
  for (int q = 0; q < kNetParams; ++q)
    if (!std::isfinite(params[q])) return fail(h, SPPC_ERR_ARG, "network parameter %d is not finite", q);
  for (int f = 0; f < kNetFeatures; ++f)
    if (!std::isfinite(mu[f]) || !(sd[f] > 0.f) || !std::isfinite(sd[f]))
      return fail(h, SPPC_ERR_ARG, "feature %d: mean must be finite and spread positive", f);
  CKS(ensure_proposal_buffers(h));
  std::vector<float> buf(params, params + kNetParams);
  buf.insert(buf.end(), mu, mu + kNetFeatures);
  buf.insert(buf.end(), sd, sd + kNetFeatures);
  CK(cudaMemcpyAsync(h->net, buf.data(), sizeof(float) * buf.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->net_ready = true;
  return SPPC_OK;
}

sppc_status sppc_proposal_samples(sppc_handle h, const double* psi, int64_t ldpsi, float* F, float* rhat, float* y,
                                  int64_t* count, void* stream) {
  if (!h || !psi || !F || !rhat || !y) return fail(h, SPPC_ERR_ARG, "NULL argument");
  if (!h->started || h->corrected) return fail(h, SPPC_ERR_STATE, "sppc_proposal_samples needs a finished Rayleigh-Ritz step");
  if (ldpsi < h->k) return fail(h, SPPC_ERR_ARG, "ldpsi < k");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->stream = s;
  CKS(ensure_proposal_buffers(h));
  const int k = h->k, kp = h->kp;
  const int64_t n = h->n;
  double* Zd = nullptr;
  double* scr = nullptr;
  CK(cudaMallocAsync(&Zd, sizeof(double) * n * k, s));
  cudaError_t e = cudaMallocAsync(&scr, sizeof(double) * prop_samples_scratch_doubles(), s);
  // Ritz vectors and raw residuals (into Tplain) of the current subspace
  if (e == cudaSuccess)
    e = qritz(h, h->p + 1, Zd, k, k, h->Tplain, nullptr, (float)h->opt.precond_clamp, nullptr, nullptr, 0, s);
  if (e == cudaSuccess) e = prop_prep(h->Tplain, kp, k, h->dDots, n, h->rhat32, h->X32, s);
  if (e == cudaSuccess) e = spmm_abs_f32(h->H, h->val32, h->val16, h->diag32, h->X32, h->T2, s);
  if (e == cudaSuccess)
    e = prop_samples(h->Tplain, Zd, k, psi, ldpsi, h->dDots, h->dDiag, h->rowc, h->rhat32, h->T2, h->dCoef + kTheta,
                     (float)h->opt.precond_clamp, k, kp, h->n1, n, scr, F, rhat, y, s);
  if (Zd) cudaFreeAsync(Zd, s);
  if (scr) cudaFreeAsync(scr, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(h, SPPC_ERR_CUDA, "proposal samples: %s", cudaGetErrorString(e));
  if (count) *count = (n - h->n1) * k;
  return SPPC_OK;
}

sppc_status sppc_mlp_forward(const float* params, const float* X, int64_t count, int32_t bf16, float* out,
                             void* stream) {
  if (!params || !X || !out || count < 0) return fail(nullptr, SPPC_ERR_ARG, "sppc_mlp_forward: bad arguments");
  const cudaError_t e = mlp_forward(params, X, count, bf16 != 0, out, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(nullptr, SPPC_ERR_CUDA, "sppc_mlp_forward: %s", cudaGetErrorString(e));
  return SPPC_OK;
}

sppc_status sppc_mlp_loss_grad(const float* params, const float* X, const float* rhat, const float* y, int64_t count,
                               float* grad, float* loss, void* stream) {
  if (!params || !X || !rhat || !y || !grad || count < 1)
    return fail(nullptr, SPPC_ERR_ARG, "sppc_mlp_loss_grad: bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* part = nullptr;
  cudaError_t e = cudaMallocAsync(&part, sizeof(float) * mlp_grad_part_floats(count), s);
  if (e == cudaSuccess)
    e = mlp_grad(params, X, rhat, y, nullptr, 0, count, static_cast<float>(1.0 / count), part, grad, loss, s);
  if (part) cudaFreeAsync(part, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(nullptr, SPPC_ERR_CUDA, "sppc_mlp_loss_grad: %s", cudaGetErrorString(e));
  return SPPC_OK;
}

sppc_status sppc_mlp_adam(float* params, float* mom, float* vel, const float* grad, int32_t t, float lr, float beta1,
                          float beta2, float eps, void* stream) {
  if (!params || !mom || !vel || !grad || t < 1) return fail(nullptr, SPPC_ERR_ARG, "sppc_mlp_adam: bad arguments");
  const float c1 = static_cast<float>(1.0 / (1.0 - std::pow((double)beta1, t)));
  const float c2 = static_cast<float>(1.0 / (1.0 - std::pow((double)beta2, t)));
  const cudaError_t e = mlp_adam(params, mom, vel, grad, lr, beta1, beta2, eps, c1, c2, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(nullptr, SPPC_ERR_CUDA, "sppc_mlp_adam: %s", cudaGetErrorString(e));
  return SPPC_OK;
}

sppc_status sppc_mlp_train_epoch(float* params, float* mom, float* vel, const float* X, const float* rhat,
                                 const float* y, const int64_t* perm, int64_t nsamples, int32_t batch, int32_t* step,
                                 float lr, float beta1, float beta2, float eps, double* mean_loss, void* stream) {
  if (!params || !mom || !vel || !X || !rhat || !y || !step || nsamples < 1 || batch < 1 || *step < 0)
    return fail(nullptr, SPPC_ERR_ARG, "sppc_mlp_train_epoch: bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t nb = (nsamples + batch - 1) / batch;
  float *part = nullptr, *grad = nullptr, *losses = nullptr;
  cudaError_t e = cudaMallocAsync(&part, sizeof(float) * mlp_grad_part_floats(batch), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&grad, sizeof(float) * kNetParams, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&losses, sizeof(float) * nb, s);
  for (int64_t b = 0; b < nb && e == cudaSuccess; ++b) {
    const int64_t base = b * batch;
    const int64_t cnt = std::min<int64_t>(batch, nsamples - base);
    e = mlp_grad(params, X, rhat, y, perm, base, cnt, static_cast<float>(1.0 / cnt), part, grad, losses + b, s);
    if (e != cudaSuccess) break;
    const int32_t t = ++(*step);
    const float c1 = static_cast<float>(1.0 / (1.0 - std::pow((double)beta1, t)));
    const float c2 = static_cast<float>(1.0 / (1.0 - std::pow((double)beta2, t)));
    e = mlp_adam(params, mom, vel, grad, lr, beta1, beta2, eps, c1, c2, s);
  }
  std::vector<float> hl(nb > 0 ? nb : 1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hl.data(), losses, sizeof(float) * nb, cudaMemcpyDeviceToHost, s);
  if (part) cudaFreeAsync(part, s);
  if (grad) cudaFreeAsync(grad, s);
  if (losses) cudaFreeAsync(losses, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(nullptr, SPPC_ERR_CUDA, "sppc_mlp_train_epoch: %s", cudaGetErrorString(e));
  if (mean_loss) {
    double a = 0.0;
    for (int64_t b = 0; b < nb; ++b) a += hl[b];
    *mean_loss = a / static_cast<double>(nb);
  }
  return SPPC_OK;
}

sppc_status sppc_feature_moments(const float* F, int64_t count, double* mean, double* sd, void* stream) {
  if (!F || !mean || !sd || count < 1) return fail(nullptr, SPPC_ERR_ARG, "sppc_feature_moments: bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* scr = nullptr;
  const int64_t ns = feature_moments_scratch_doubles();
  cudaError_t e = cudaMallocAsync(&scr, sizeof(double) * ns, s);
  if (e == cudaSuccess) e = feature_moments(F, count, scr, s);
  double out[2 * kNetFeatures] = {0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, scr + ns - 2 * kNetFeatures, sizeof(out), cudaMemcpyDeviceToHost, s);
  if (scr) cudaFreeAsync(scr, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(nullptr, SPPC_ERR_CUDA, "sppc_feature_moments: %s", cudaGetErrorString(e));
  for (int f = 0; f < kNetFeatures; ++f) {
    mean[f] = out[f];
    sd[f] = out[kNetFeatures + f];
  }
  return SPPC_OK;
}

sppc_status sppc_standardize(const float* F, int64_t count, const float* mu, const float* sd, float* X,
                             void* stream) {
  if (!F || !mu || !sd || !X || count < 0) return fail(nullptr, SPPC_ERR_ARG, "sppc_standardize: bad arguments");
  for (int f = 0; f < kNetFeatures; ++f)
    if (!(sd[f] > 0.f)) return fail(nullptr, SPPC_ERR_ARG, "sppc_standardize: spread %d must be positive", f);
  const cudaError_t e = standardize(F, count, mu, sd, X, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(nullptr, SPPC_ERR_CUDA, "sppc_standardize: %s", cudaGetErrorString(e));
  return SPPC_OK;
}

sppc_status sppc_spmm_tiling(sppc_handle h, int64_t* chunk_cols, double* candidate_ms) {
  if (!h) return fail(nullptr, SPPC_ERR_ARG, "NULL handle");
  if (chunk_cols) *chunk_cols = h->chunk_cols_used;
  if (candidate_ms) std::copy(h->tuned_ms, h->tuned_ms + 5, candidate_ms);
  return SPPC_OK;
}

sppc_status sppc_sell_sigma(sppc_handle h, int32_t* sigma, double* candidate_ms) {
  if (!h) return fail(nullptr, SPPC_ERR_ARG, "sppc_sell_sigma: null handle");
  if (sigma) *sigma = h->sigma_used;
  if (candidate_ms) std::copy(h->sigma_ms, h->sigma_ms + 3, candidate_ms);
  return SPPC_OK;
}

}  // extern "C"
