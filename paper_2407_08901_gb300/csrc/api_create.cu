// C ABI, part 1: options, handle creation (validation, uploads, the GPU layout
// build and its autotuners) and destruction.
#include "driver.h"

namespace sppc::drv {


// ms per 8-column product of H's layout with column tile c and sort window
// sigma: built with a temporary allocator, timed on two products after a
// warm-up (register-gather kernel, X = 0: the gather pattern, not the values,
// sets the time) and freed.
cudaError_t time_layout(int64_t n, const int64_t* d_rp, const int32_t* d_ci, const double* d_va,
                        const std::vector<int64_t>& seg, bool f64, int64_t c, int sigma, const float2* X, float2* Y,
                        cudaEvent_t a, cudaEvent_t b, cudaStream_t s, double* ms_out) {
  std::vector<void*> mine;
  const DeviceAlloc tmp = [&mine](void** p, size_t bytes) {
    const cudaError_t x = cudaMalloc(p, bytes ? bytes : 1);
    if (x == cudaSuccess) mine.push_back(*p);
    return x;
  };
  SellDeviceLayout T;
  cudaError_t e = build_sell_device(n, d_rp, d_ci, d_va, n, seg, c, f64, 0, s, tmp, T, sigma);
  if (e == cudaSuccess) {
    SellDev A;
    A.nslices = T.nslices;
    A.nrows = n;
    A.nchunks = T.nchunks;
    A.chunk_cols = T.chunk_cols;
    A.chunk_slice = T.chunk_slice.data();
    A.slice_ptr = T.slice_ptr_d;
    A.slice_rows = T.rows_d;
    A.col = T.col_d;
    A.val = T.val_d;
    A.row_first = T.first_d;
    A.row_last = T.last_d;
    A.f64 = f64;
    e = spmm(A, 8, X, Y, Epi{}, s);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = spmm(A, 8, X, Y, Epi{}, s);
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) *ms_out = ms / 2.0;
  }
  const cudaError_t se = cudaStreamSynchronize(s);
  for (void* p : mine) cudaFree(p);
  return e != cudaSuccess ? e : se;
}

// Candidates of the SELL sort window: 1024, 256 and 64 rows at column tile c.
cudaError_t tune_sigma(int64_t n, const int64_t* d_rp, const int32_t* d_ci, const double* d_va,
                       const std::vector<int64_t>& seg, bool f64, int64_t c, cudaStream_t s, int* best,
                       double* ms_out) {
  const int cand[3] = {1024, 256, 64};  // reported as 64, 256, 1024
  float2 *X = nullptr, *Y = nullptr;
  cudaError_t e = cudaMallocAsync(&X, sizeof(float2) * n * 8, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&Y, sizeof(float2) * n * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(X, 0, sizeof(float2) * n * 8, s);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  double best_ms = 1e300;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    double ms = 0.0;
    e = time_layout(n, d_rp, d_ci, d_va, seg, f64, c, cand[i], X, Y, a, b, s, &ms);
    if (e == cudaSuccess) {
      ms_out[2 - i] = ms;
      if (ms < 0.98 * best_ms) {  // a narrower window must win by 2%
        best_ms = ms;
        *best = cand[i];
      }
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (X) cudaFreeAsync(X, s);
  if (Y) cudaFreeAsync(Y, s);
  const cudaError_t se = cudaStreamSynchronize(s);
  return e != cudaSuccess ? e : se;
}

// Candidates of the SpMM column tile: untiled, then 2.6M, 1.31M, 655k and
// 328k columns (at most 255 tiles), each timed as time_layout does at the
// default sort window.
cudaError_t tune_chunk_cols(int64_t n, const int64_t* d_rp, const int32_t* d_ci, const double* d_va,
                            const std::vector<int64_t>& seg, bool f64, cudaStream_t s, int64_t* best, double* ms_out) {
  const int64_t cand[5] = {-1, 2621440, 1310720, 655360, 327680};
  float2 *X = nullptr, *Y = nullptr;
  cudaError_t e = cudaMallocAsync(&X, sizeof(float2) * n * 8, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&Y, sizeof(float2) * n * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(X, 0, sizeof(float2) * n * 8, s);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  double best_ms = 1e300;
  for (int ci = 0; ci < 5 && e == cudaSuccess; ++ci) {
    const int64_t c = cand[ci];
    if (c > 0 && (c >= n || (n + c - 1) / c > 255)) continue;
    double ms = 0.0;
    e = time_layout(n, d_rp, d_ci, d_va, seg, f64, c, 1024, X, Y, a, b, s, &ms);
    if (e == cudaSuccess) {
      ms_out[ci] = ms;
      if (ms < 0.98 * best_ms) {  // a finer tile must win by 2%
        best_ms = ms;
        *best = c;
      }
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (X) cudaFreeAsync(X, s);
  if (Y) cudaFreeAsync(Y, s);
  return e;
}

}  // namespace sppc::drv

// Accessors used by the allocation-free SpMM entry point (noalloc.cu).
namespace sppc {

const SellDev* handle_matrix(sppc_handle h, int64_t* n) {
  if (n) *n = h->n;
  return &h->H;
}
sppc_status handle_fail(sppc_handle h, sppc_status st, const char* msg) { return fail(h, st, "%s", msg); }
void handle_scratch(sppc_handle h, float2** t1, float2** t2) {
  *t1 = h->T1;
  *t2 = h->T2;
}
// Value arrays of the mixed-precision products (precision 1: val32; 2: val16 and
// diag32; both null otherwise) and the handle's precision option.
void handle_values(sppc_handle h, int* precision, const float** val32, const uint16_t** val16, const float** diag32) {
  *precision = h->opt.precision;
  *val32 = h->val32;
  *val16 = h->val16;
  *diag32 = h->diag32;
}
void handle_size(sppc_handle h, int64_t* n, int64_t* nnz, int* k) {
  if (n) *n = h->n;
  if (nnz) *nnz = h->nnz;
  if (k) *k = h->k;
}
}  // namespace sppc

extern "C" {

void sppc_default_opts(sppc_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->p_max = 15;
  o->tol = 1e-6;
  o->minres_tol = 1e-12;
  o->minres_maxit = 0;
  o->small_tol = 1e-12;
  o->small_block = 0;
  o->degeneracy_tol = 1e-10;
  o->check_symmetry = 0;
  o->seed = 0;
  o->timing = 0;
  o->spmm_chunk_cols = 0;
  o->hybrid = 0;
  o->switch_order = 15;
  o->hybrid_maxit = 1000;
  o->precond = 1;
  o->precond_clamp = 1e-2;
  o->precond_iters = 20;
  o->precision = 0;
  o->proposal = 0;
  o->precond_levels = 1;
  o->minres_deflate = 1;
  o->small_degree = 30;
  o->switch_stall = 0.0;
  o->minres_ctas = 0;
  o->spin_cap = 0;
  o->value_rounding = 0;
  o->minres_fp32 = 0;
  o->minres_fp32_tol = 1e-6;
  o->tensor_gram = 0;
  o->sell_sigma = 0;
  o->hybrid_blocks = 0;
  o->spmm_kernel = 1;
  o->reorth = 0;
}

const char* sppc_last_error(sppc_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int64_t sppc_kernel_launches(void) { return (int64_t)launch_count(); }

sppc_status sppc_destroy(sppc_handle h) {
  if (!h) return SPPC_OK;
  if (h->stream2) cudaStreamSynchronize(h->stream2);
  for (void* p : h->allocs) cudaFree(p);
  if (h->stream2) cudaStreamDestroy(h->stream2);
  if (h->ev_a) cudaEventDestroy(h->ev_a);
  if (h->ev_b) cudaEventDestroy(h->ev_b);
  if (h->pinned) cudaFreeHost(h->pinned);
  for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
  delete h;
  return SPPC_OK;
}

sppc_status sppc_create(const sppc_csr* Hc, const int64_t* level_offsets, int32_t n_levels, int64_t n1, int32_t k,
                        const sppc_opts* opts, void* stream, sppc_handle* out) {
  sppc_ctx* h = nullptr;
  if (!out) return fail(nullptr, SPPC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!Hc || !level_offsets) return fail(nullptr, SPPC_ERR_ARG, "H or level_offsets is NULL");
  if (Hc->n <= 0 || Hc->nnz < 0 || !Hc->row_ptr || (Hc->nnz > 0 && (!Hc->col || !Hc->val)))
    return fail(nullptr, SPPC_ERR_ARG, "malformed CSR descriptor");
  if (Hc->n >= ((int64_t)1 << 31) - 64) return fail(nullptr, SPPC_ERR_ARG, "n must be below 2^31");
  if (k < 1 || k > 8) return fail(nullptr, SPPC_ERR_ARG, "k must be in [1, 8], got %d", k);
  if (n_levels < 1) return fail(nullptr, SPPC_ERR_LEVELS, "n_levels must be >= 1");
  const int64_t n = Hc->n;
  if (level_offsets[0] != 0 || level_offsets[n_levels] != n)
    return fail(nullptr, SPPC_ERR_LEVELS, "level_offsets must run from 0 to n");
  bool n1_ok = false;
  for (int i = 0; i < n_levels; ++i) {
    if (level_offsets[i + 1] <= level_offsets[i]) return fail(nullptr, SPPC_ERR_LEVELS, "level_offsets not increasing");
    if (level_offsets[i + 1] == n1) n1_ok = true;
  }
  if (!n1_ok) return fail(nullptr, SPPC_ERR_LEVELS, "n1 = %lld is not a level boundary", (long long)n1);
  if (k >= n1) return fail(nullptr, SPPC_ERR_ARG, "k must be smaller than n1");
  sppc_opts opt;
  sppc_default_opts(&opt);
  if (opts) opt = *opts;
  if (opt.p_max < 0 || opt.p_max > kMaxBlocks - 2 || (int64_t)k * (opt.p_max + 1) > 144)
    return fail(nullptr, SPPC_ERR_ARG, "p_max out of range (k*(p_max+1) must be <= 144)");
  if (opt.spmm_kernel != 0 && opt.spmm_kernel != 1) return fail(nullptr, SPPC_ERR_ARG, "opts.spmm_kernel must be 0 or 1");
  if (opt.reorth != 0 && opt.reorth != 1) return fail(nullptr, SPPC_ERR_ARG, "opts.reorth must be 0 or 1");
  if (opt.precond < 0 || opt.precond > 2) return fail(nullptr, SPPC_ERR_ARG, "opts.precond must be 0, 1 or 2");
  if (opt.precision < -1 || opt.precision > 2)
    return fail(nullptr, SPPC_ERR_ARG, "opts.precision must be -1, 0, 1 or 2");
  if (opt.precision == -1 && (opt.hybrid == 2 || opt.proposal != 0))
    return fail(nullptr, SPPC_ERR_ARG, "opts.precision = -1 (native FP64) runs without RMM-DIIS and the proposal");
  if (opt.spmm_chunk_cols < -2) return fail(nullptr, SPPC_ERR_ARG, "opts.spmm_chunk_cols must be >= -2");
  if (opt.hybrid < 0 || opt.hybrid > 2) return fail(nullptr, SPPC_ERR_ARG, "opts.hybrid must be 0, 1 or 2");
  if (opt.hybrid == 2 && (opt.precision != 0 || opt.proposal != 0))
    return fail(nullptr, SPPC_ERR_ARG, "opts.hybrid = 2 (RMM-DIIS) runs with precision 0 and no proposal");
  if (opt.proposal != 0 && opt.proposal != 1) return fail(nullptr, SPPC_ERR_ARG, "opts.proposal must be 0 or 1");
  if (opt.proposal == 1 && (opt.hybrid != 1 || opt.precond < 1))
    return fail(nullptr, SPPC_ERR_ARG, "opts.proposal = 1 needs hybrid = 1 and precond 1 or 2");
  if (opt.precond_levels < 1 || opt.precond_levels > n_levels)
    return fail(nullptr, SPPC_ERR_ARG, "opts.precond_levels must be in [1, n_levels]");
  if (opt.minres_deflate != 0 && opt.minres_deflate != 1)
    return fail(nullptr, SPPC_ERR_ARG, "opts.minres_deflate must be 0 or 1");
  if (opt.small_degree < 1 || opt.small_degree > 200)
    return fail(nullptr, SPPC_ERR_ARG, "opts.small_degree must be in [1, 200]");
  if (!(opt.switch_stall >= 0.0) || opt.switch_stall > 1.0)
    return fail(nullptr, SPPC_ERR_ARG, "opts.switch_stall must be in [0, 1]");
  if (opt.minres_ctas < 0) return fail(nullptr, SPPC_ERR_ARG, "opts.minres_ctas must be >= 0");
  if (opt.spin_cap < 0) return fail(nullptr, SPPC_ERR_ARG, "opts.spin_cap must be >= 0");
  if (opt.value_rounding < 0 || opt.value_rounding > 2)
    return fail(nullptr, SPPC_ERR_ARG, "opts.value_rounding must be 0, 1 or 2");
  if (opt.minres_fp32 != 0 && opt.minres_fp32 != 1) return fail(nullptr, SPPC_ERR_ARG, "opts.minres_fp32 must be 0 or 1");
  if (opt.minres_fp32 && opt.precision == -1)
    return fail(nullptr, SPPC_ERR_ARG, "opts.minres_fp32 needs double-float slots (precision 0, 1 or 2)");
  if (opt.minres_fp32 && !(opt.minres_fp32_tol > 0.0 && opt.minres_fp32_tol < 1.0))
    return fail(nullptr, SPPC_ERR_ARG, "opts.minres_fp32_tol must be in (0, 1)");
  if (opt.tensor_gram != 0 && opt.tensor_gram != 1) return fail(nullptr, SPPC_ERR_ARG, "opts.tensor_gram must be 0 or 1");
  if (!(opt.sell_sigma == 0 || opt.sell_sigma == -2 ||
        (opt.sell_sigma >= 16 && opt.sell_sigma <= 1024 && opt.sell_sigma % 16 == 0)))
    return fail(nullptr, SPPC_ERR_ARG, "opts.sell_sigma must be 0, -2 or a multiple of 16 in [16, 1024]");
  if (opt.precision > 0 && (k + 1) / 2 * 2 != 8 && (k + 1) / 2 * 2 != 4)
    return fail(nullptr, SPPC_ERR_ARG, "opts.precision 1 or 2 needs k in {3, 4, 7, 8} (4- or 8-column FP32 products)");
  if (opt.precond_iters < 0 || opt.precond_iters > 10000)
    return fail(nullptr, SPPC_ERR_ARG, "opts.precond_iters must be in [0, 10000]");

  h = new sppc_ctx();
  if (opt.hybrid_blocks <= 0 || opt.hybrid_blocks > opt.p_max + 1) opt.hybrid_blocks = opt.p_max + 1;
  if (opt.hybrid_blocks < 3) opt.hybrid_blocks = 3;
  h->opt = opt;
  h->f64 = opt.precision == -1;
  h->stream = static_cast<cudaStream_t>(stream);
  h->n = n;
  h->nnz = Hc->nnz;
  h->n1 = n1;
  h->k = k;
  h->kp = (k + 1) / 2 * 2;
  h->pmax = opt.p_max;
  h->mmax = k * (opt.p_max + 1);
  h->lev.assign(level_offsets, level_offsets + n_levels + 1);
  h->n_lead = (opt.precond == 2) ? std::max<int64_t>(n1, level_offsets[opt.precond_levels]) : n1;
  auto bail = [&](sppc_status st) {
    g_create_error = h->err;
    sppc_destroy(h);
    return st;
  };
  // The CSR.  A host CSR is read on the host.  A device CSR stays on the device:
  // the host reads its row pointers and the leading rows (the small space and
  // the preconditioner's leading block) only, and the checks, the rounding of
  // precision 1 / 2 and the diagonal run on the GPU, so a matrix whose host copy
  // would not fit is never copied.
  const bool dev_in = Hc->on_device != 0;
  std::vector<int64_t> rp_h;
  std::vector<int32_t> ci_h;
  std::vector<double> va_h;
  const int64_t* rp = Hc->row_ptr;
  const int32_t* ci = Hc->col;
  const double* va = Hc->val;
  const int64_t rows_h = dev_in ? std::max<int64_t>(n1, h->n_lead) : n;  // rows readable on the host
  const int round_mode = opt.precision > 0 ? opt.precision : opt.value_rounding;
  if (dev_in) {
    rp_h.resize(n + 1);
    if (cudaMemcpy(rp_h.data(), rp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
      return bail(fail(h, SPPC_ERR_CUDA, "copying the device row pointers to the host failed"));
    if (rp_h[0] != 0 || rp_h[n] != Hc->nnz)
      return bail(fail(h, SPPC_ERR_ARG, "row_ptr[0] must be 0 and row_ptr[n] = nnz"));
    for (int64_t r = 0; r < n; ++r)
      if (rp_h[r + 1] < rp_h[r]) return bail(fail(h, SPPC_ERR_ARG, "row_ptr is not monotone"));
    const int64_t lead_nnz = rp_h[rows_h];
    ci_h.resize(std::max<int64_t>(lead_nnz, 1));
    va_h.resize(std::max<int64_t>(lead_nnz, 1));
    if (lead_nnz > 0 &&
        (cudaMemcpy(ci_h.data(), ci, sizeof(int32_t) * lead_nnz, cudaMemcpyDeviceToHost) != cudaSuccess ||
         cudaMemcpy(va_h.data(), va, sizeof(double) * lead_nnz, cudaMemcpyDeviceToHost) != cudaSuccess))
      return bail(fail(h, SPPC_ERR_CUDA, "copying the leading rows of the device CSR to the host failed"));
    rp = rp_h.data();
    ci = ci_h.data();
    va = va_h.data();
  }
  if (round_mode == 1) {
    // mixed precision: the matrix is H rounded to FP32, everywhere (SpMM, leading
    // block, diagonal); the solver's error is measured against that matrix
    const int64_t cnt = rp[rows_h];
    if (va_h.empty()) va_h.assign(va, va + cnt);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < cnt; ++t) va_h[t] = static_cast<double>(static_cast<float>(va_h[t]));
    va = va_h.data();
  } else if (round_mode == 2) {
    // BF16 path: off-diagonal values rounded to FP32 and then to BF16 (round to
    // nearest even), the diagonal to FP32, everywhere; the solver's error is
    // measured against that matrix
    if (va_h.empty()) va_h.assign(va, va + Hc->nnz);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < rows_h; ++r) {
      const int64_t lo = rp[r], hi = rp[r + 1];
      if (lo < 0 || hi < lo || hi > Hc->nnz) continue;  // rejected by the validation below
      for (int64_t t = lo; t < hi; ++t) {
        const float f = static_cast<float>(va_h[t]);
        va_h[t] = ci[t] == r ? static_cast<double>(f) : static_cast<double>(round_bf16(f));
      }
    }
    va = va_h.data();
  }
  // validation
  if (rp[0] != 0 || rp[n] != Hc->nnz) return bail(fail(h, SPPC_ERR_ARG, "row_ptr[0] must be 0 and row_ptr[n] = nnz"));
  if (dev_in) {
    int flags = 0;
    const cudaError_t e = csr_check_device(n, Hc->row_ptr, Hc->col, Hc->val, opt.check_symmetry != 0, &flags,
                                           h->stream);
    if (e != cudaSuccess) return bail(fail(h, SPPC_ERR_CUDA, "device CSR check: %s", cudaGetErrorString(e)));
    if (flags & 2) return bail(fail(h, SPPC_ERR_ARG, "column index out of range"));
    if (flags & 4) return bail(fail(h, SPPC_ERR_ARG, "column indices must increase strictly within a row"));
    if (flags & 8) return bail(fail(h, SPPC_ERR_NAN, "H holds a NaN or Inf"));
    if (flags & 1) return bail(fail(h, SPPC_ERR_NOT_SYMMETRIC, "H is not symmetric"));
  }
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t r = 0; r < (dev_in ? 0 : n); ++r) {
    if (rp[r + 1] < rp[r]) {
      bad |= 1;
      continue;
    }
    for (int64_t t = rp[r]; t < rp[r + 1]; ++t) {
      if (ci[t] < 0 || ci[t] >= n) bad |= 2;
      if (t > rp[r] && ci[t] <= ci[t - 1]) bad |= 4;
      if (!std::isfinite(va[t])) bad |= 8;
    }
  }
  if (bad & 1) return bail(fail(h, SPPC_ERR_ARG, "row_ptr is not monotone"));
  if (bad & 2) return bail(fail(h, SPPC_ERR_ARG, "column index out of range"));
  if (bad & 4) return bail(fail(h, SPPC_ERR_ARG, "column indices must increase strictly within a row"));
  if (bad & 8) return bail(fail(h, SPPC_ERR_NAN, "H holds a NaN or Inf"));
  if (opt.check_symmetry && !dev_in) {
    int asym = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(| : asym)
    for (int64_t r = 0; r < n; ++r) {
      for (int64_t t = rp[r]; t < rp[r + 1]; ++t) {
        const int32_t c = ci[t];
        const int32_t* b = ci + rp[c];
        const int32_t* e = ci + rp[c + 1];
        const int32_t* f = std::lower_bound(b, e, (int32_t)r);
        if (f == e || *f != r || va[rp[c] + (f - b)] != va[t]) asym = 1;
      }
    }
    if (asym) return bail(fail(h, SPPC_ERR_NOT_SYMMETRIC, "H is not symmetric"));
  }
  // Gershgorin interval of H0_hat
  {
    double lo = 1e300, hi = -1e300;
#pragma omp parallel for reduction(min : lo) reduction(max : hi)
    for (int64_t r = 0; r < n1; ++r) {
      double dg = 0.0, off = 0.0;
      for (int64_t t = rp[r]; t < rp[r + 1] && ci[t] < n1; ++t) {
        if (ci[t] == r)
          dg = va[t];
        else
          off += std::fabs(va[t]);
      }
      lo = std::min(lo, dg - off);
      hi = std::max(hi, dg + off);
    }
    h->h11_lo = lo;
    h->h11_hi = hi;
    h->h11_norm = std::max(std::fabs(lo), std::fabs(hi));
  }
  // layouts: H's SELL-16 built on the GPU from a device copy of the CSR
  {
    std::vector<int64_t> seg(h->lev.begin(), h->lev.end());
    int64_t chunk = opt.spmm_chunk_cols;
    const bool tune = chunk == -2;
    // default: 80 MB of an 8-column double-float block keeps X's gathered rows
    // in L2.  The native FP64 product is DFMA-bound as long as X itself fits in
    // L2, and then tiles only add passes (c2, X 128 MB: 6.12 ms untiled against
    // 6.43 ms in 1.31M-column tiles); beyond that the gathers miss L2 and the
    // tiles win again (c3, X 1.28 GB: 107 ms untiled against 90 ms)
    if (chunk == 0) {
      int dev = 0, l2 = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
      chunk = (h->f64 && n * 8 * (int64_t)sizeof(float2) <= (int64_t)l2) ? -1 : 1310720;
    }
    if (chunk > 0 && (n + chunk - 1) / chunk > 255) chunk = (n + 254) / 255;
    cudaStream_t s = h->stream;
    int64_t* d_rp = nullptr;
    int32_t* d_ci = nullptr;
    double* d_va = nullptr;
    cudaError_t e = cudaSuccess;
    if (dev_in) {
      // the caller's device CSR, read in place (values rounded in the layout fill)
      d_rp = const_cast<int64_t*>(Hc->row_ptr);
      d_ci = const_cast<int32_t*>(Hc->col);
      d_va = const_cast<double*>(Hc->val);
    } else {
      const int64_t nnz1 = Hc->nnz > 0 ? Hc->nnz : 1;
      e = cudaMallocAsync(&d_rp, sizeof(int64_t) * (n + 1), s);
      if (e == cudaSuccess) e = cudaMallocAsync(&d_ci, sizeof(int32_t) * nnz1, s);
      if (e == cudaSuccess) e = cudaMallocAsync(&d_va, sizeof(double) * nnz1, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_rp, rp, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess && Hc->nnz > 0)
        e = cudaMemcpyAsync(d_ci, ci, sizeof(int32_t) * Hc->nnz, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess && Hc->nnz > 0)
        e = cudaMemcpyAsync(d_va, va, sizeof(double) * Hc->nnz, cudaMemcpyHostToDevice, s);
    }
    SellDeviceLayout L;
    const DeviceAlloc alloc = [h](void** p, size_t bytes) {
      unsigned char* q = nullptr;
      const cudaError_t x = dalloc(h, &q, bytes);
      *p = q;
      return x;
    };
    if (e == cudaSuccess && tune) {
      // autotuner of the column tile: build the layout for each candidate, time
      // two 8-column products, keep the fastest (ties to the coarser tile)
      e = tune_chunk_cols(n, d_rp, d_ci, d_va, seg, h->f64, s, &chunk, h->tuned_ms);
    }
    h->chunk_cols_used = chunk;
    int sigma = opt.sell_sigma > 0 ? opt.sell_sigma : 1024;
    if (e == cudaSuccess && opt.sell_sigma == -2)
      e = tune_sigma(n, d_rp, d_ci, d_va, seg, h->f64, chunk, s, &sigma, h->sigma_ms);
    h->sigma_used = sigma;
    if (e == cudaSuccess)
      e = build_sell_device(n, d_rp, d_ci, d_va, n, seg, chunk, h->f64, dev_in ? round_mode : 0, s, alloc, L,
                            sigma);
    if (e == cudaSuccess) {
      // per-row constants of the learned proposal's features
      int64_t* d_lev = nullptr;
      e = cudaMallocAsync(&d_lev, sizeof(int64_t) * h->lev.size(), s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_lev, h->lev.data(), sizeof(int64_t) * h->lev.size(), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = dalloc(h, &h->rowc, (size_t)n);
      if (e == cudaSuccess) e = row_consts(n, d_rp, d_va, d_lev, (int)h->lev.size() - 1, h->rowc, s);
      if (d_lev) cudaFreeAsync(d_lev, s);
    }
    if (!dev_in) {
      if (d_rp) cudaFreeAsync(d_rp, s);
      if (d_ci) cudaFreeAsync(d_ci, s);
      if (d_va) cudaFreeAsync(d_va, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
      return bail(fail(h, e == cudaErrorMemoryAllocation ? SPPC_ERR_OOM : SPPC_ERR_CUDA, "SELL build on the GPU: %s",
                       cudaGetErrorString(e)));
    h->h_chunk_slice = L.chunk_slice;
    h->H.nslices = L.nslices;
    h->H.nrows = n;
    h->H.nchunks = L.nchunks;
    h->H.chunk_cols = L.chunk_cols;
    h->H.chunk_slice = h->h_chunk_slice.data();
    h->H.slice_ptr = L.slice_ptr_d;
    h->H.slice_rows = L.rows_d;
    h->H.col = L.col_d;
    h->H.val = L.val_d;
    h->H.row_first = L.first_d;
    h->H.row_last = L.last_d;
    h->H.f64 = h->f64;
    h->H.tma = (opt.spmm_kernel == 0 && !h->f64 && spmm_tma_available()) ? 1 : 0;
    if (h->H.tma) {
      // the TMA kernel's time-out flag (per handle; cleared by sppc_start and sppc_spmm_host)
      e = dalloc(h, &h->H.tma_flag, 1);
      if (e == cudaSuccess) e = cudaMemsetAsync(h->H.tma_flag, 0, sizeof(int), s);
      if (e != cudaSuccess) return bail(fail(h, SPPC_ERR_OOM, "TMA flag: %s", cudaGetErrorString(e)));
      h->H.spin_limit = static_cast<unsigned>(opt.spin_cap);
    }
    if (opt.precision == 1) {
      // FP32 copy of the values (exact: they are FP32 already)
      e = dalloc(h, &h->val32, (size_t)(L.total > 0 ? L.total : 1));
      if (e == cudaSuccess) e = dalloc(h, &h->X32, (size_t)n * 8);
      if (e == cudaSuccess) e = df_hi_parts(L.val_d, h->val32, L.total, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return bail(fail(h, SPPC_ERR_OOM, "FP32 values: %s", cudaGetErrorString(e)));
    } else if (opt.precision == 2) {
      // BF16 copy of the off-diagonal values (exact: they are BF16 already)
      e = dalloc(h, &h->val16, (size_t)(L.total > 0 ? L.total : 1));
      if (e == cudaSuccess) e = dalloc(h, &h->X32, (size_t)n * 8);
      if (e == cudaSuccess) e = make_val16(h->H, h->val16, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return bail(fail(h, SPPC_ERR_OOM, "BF16 values: %s", cudaGetErrorString(e)));
    }
    h->h_slices = L.nslices;
    h->h_slice_ptr = std::move(L.slice_ptr);
    h->h_slice_rows = std::move(L.rows);
  }
  {
    SellHost S;
    std::vector<int64_t> seg = {0, n1};
    build_sell(n1, rp, ci, va, n1, seg, 1024, 0, h->f64, S);
    sppc_status st = upload_sell(h, S, h->H11, n1, h->h11_chunk_slice);
    if (st != SPPC_OK) return bail(st);
    h->H11.f64 = h->f64;
    h->h11_slices = S.nslices;
    h->h11_slice_ptr = std::move(S.slice_ptr);
    h->h11_slice_rows = std::move(S.rows);
    h->H11.tma = h->H.tma;
    h->H11.tma_flag = h->H.tma_flag;
    h->H11.spin_limit = h->H.spin_limit;
    st = upload_csr11(h, n1, rp, ci, va, h->H11c);
    if (st != SPPC_OK) return bail(st);
    h->Hlead = h->H11c;
    if (h->n_lead > n1) {
      st = upload_csr11(h, h->n_lead, rp, ci, va, h->Hlead);
      if (st != SPPC_OK) return bail(st);
    }
  }
  // diag(H) for the preconditioned continuation
  {
    cudaError_t e = dalloc(h, &h->dDiag, (size_t)n);
    if (dev_in) {
      if (e == cudaSuccess)
        e = csr_diag_device(n, Hc->row_ptr, Hc->col, Hc->val, round_mode, h->f64, h->dDiag, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    } else {
      std::vector<float2> dg(n, make_float2(0.f, 0.f));
#pragma omp parallel for schedule(static)
      for (int64_t r = 0; r < n; ++r) {
        const int32_t* b = ci + rp[r];
        const int32_t* e2 = ci + rp[r + 1];
        const int32_t* f = std::lower_bound(b, e2, (int32_t)r);
        if (f != e2 && *f == r) put_slot(va[rp[r] + (f - b)], dg[r], h->f64);
      }
      if (e == cudaSuccess) e = cudaMemcpy(h->dDiag, dg.data(), sizeof(float2) * n, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && opt.precision == 2) {
      e = dalloc(h, &h->diag32, (size_t)n);
      if (e == cudaSuccess) e = df_hi_parts(h->dDiag, h->diag32, n, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) return bail(fail(h, SPPC_ERR_OOM, "diag upload failed: %s", cudaGetErrorString(e)));
  }
  // work buffers
  {
    const int kp = h->kp;
    const int64_t nb = (int64_t)(h->pmax + 1) * n * kp;
    cudaError_t e = cudaSuccess;
    auto A = [&](float2** p, size_t c) {
      if (e == cudaSuccess) e = dalloc(h, p, c);
    };
    auto D = [&](double** p, size_t c) {
      if (e == cudaSuccess) e = dalloc(h, p, c);
    };
    A(&h->Q, nb);
    if (h->opt.tensor_gram && kp == 8) {
      const size_t dbytes = (size_t)((h->pmax + 1 + 15) / 16) * (size_t)qdigits_group_bytes(n);
      if (e == cudaSuccess) e = dalloc(h, &h->Qd, dbytes);
      if (e == cudaSuccess) e = dalloc(h, &h->Wd, dbytes);
      if (e == cudaSuccess) e = dalloc(h, &h->wexp, (size_t)(h->pmax + 1) * 8);
      // stale tiles hold finite digits (blocks beyond a Gram's or update's count meet
      // zero coefficients)
      if (e == cudaSuccess) e = cudaMemsetAsync(h->Qd, 0, dbytes, h->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(h->Wd, 0, dbytes, h->stream);
      A(&h->Zt, (size_t)n * 8);
      A(&h->Dt, (size_t)n * 8);
    }
    A(&h->W, nb);
    A(&h->Psi, nb);
    A(&h->HPsi, (size_t)n * kp);
    A(&h->T1, (size_t)n * 8);
    A(&h->T2, (size_t)n * 8);
    A(&h->psi_hat, (size_t)n1 * kp);
    A(&h->vps, (size_t)n1 * kp);
    // MINRES vectors: the small-space solves (n1 rows) and the precond 2 solve (n_lead rows)
    for (float2** q : {&h->b1, &h->mv, &h->mvprev, &h->mp, &h->my, &h->mw1, &h->mw2, &h->mx})
      A(q, (size_t)std::max(n1, h->n_lead) * kp);
    if (h->opt.minres_fp32)
      for (float2** q : {&h->mref, &h->mres, &h->mdx}) A(q, (size_t)n1 * kp);
    for (int i = 0; i < 12; ++i) A(&h->se[i], (size_t)n1 * 8);
    A(&h->psib[0], (size_t)n1 * 8);
    A(&h->psib[1], (size_t)n1 * 8);
    D(&h->dEb, 16);
    D(&h->dE, (size_t)(kMaxBlocks + 2) * 8);
    D(&h->dHt, (size_t)h->mmax * h->mmax);
    D(&h->dGram, (size_t)kMaxBlocks * 64);
    D(&h->dC1, (size_t)kMaxBlocks * 64);
    D(&h->dC2, (size_t)kMaxBlocks * 64);
    D(&h->dR1, 256);
    D(&h->dR2, 256);
    D(&h->dTheta, 16);
    D(&h->dV, 160 * 16);
    D(&h->dDots, 64);
    D(&h->dS, 256);
    A(&h->dCoef, kCoefEnd);
    A(&h->dRinv, 256);
    A(&h->dRecycle, (size_t)kMaxBlocks * 64);
    A(&h->dY, (size_t)kMaxBlocks * 64);
    if (h->opt.precond == 2) {
      A(&h->zlead, (size_t)h->n_lead * kp);
      A(&h->rlead, (size_t)h->n_lead * kp);
    }
    if (h->opt.hybrid == 1) A(&h->Tspare, (size_t)n * kp);
    A(&h->dCoefBig, (size_t)kMaxBlocks * 64);
    if (e == cudaSuccess) e = dalloc(h, &h->dStatus, 64);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dStatus, 0, sizeof(int) * 64, h->stream);
    if (e == cudaSuccess) e = dalloc(h, &h->dBar, 4);
    h->partial_cap = ((n + 2047) / 2048 + 1) * (int64_t)kMaxBlocks * 64;
    A(&h->partials, (size_t)h->partial_cap);
    if (e != cudaSuccess)
      return bail(fail(h, e == cudaErrorMemoryAllocation ? SPPC_ERR_OOM : SPPC_ERR_CUDA, "allocation failed: %s",
                       cudaGetErrorString(e)));
    k_set_consts<<<1, 32, 0, h->stream>>>(h->dCoef, h->f64); count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dHt, 0, sizeof(double) * h->mmax * h->mmax, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return bail(fail(h, SPPC_ERR_CUDA, "init failed: %s", cudaGetErrorString(e)));
  }
  *out = h;
  return SPPC_OK;
}


}  // extern "C"
