// Host driver, part 1: the driver's tiny kernels (coefficient arrays, the
// projected matrix, restarts), the host SELL builder of the small space, the
// products with H0_hat and H and their timing.
#include "driver.h"

namespace sppc::drv {

thread_local std::string g_create_error;

// ------------------------------------------------------------ tiny kernels
__global__ void k_set_consts(float2* c, bool f64) {
  const int t = threadIdx.x;
  if (t < 16) {
    c[kOnes + t] = slot_put(1.0, f64);
    c[kNegOnes + t] = slot_put(-1.0, f64);
  }
}

__global__ void k_set_e0(const double* E0, int k, int kp, float2* c, bool f64) {
  const int j = threadIdx.x;
  if (j >= kp) return;
  c[kShiftNegE + j] = (j < k) ? slot_put(-E0[j], f64) : make_float2(0.f, 0.f);
  c[kPosE0 + j] = (j < k) ? slot_put(E0[j], f64) : make_float2(0.f, 0.f);
  c[kInvE0 + j] = (j < k) ? slot_put(1.0 / E0[j], f64) : make_float2(0.f, 0.f);
}

// Coefficients of the right-hand side of Eq. exp_seq2 at order p:
//  big rows:   Psi^(p)_2 = (1/E0) H Psi^(p-1)_2 - sum_{l=1}^{p-2} (E^(p-l)/E0) Psi^(l)_2
//  small rows: b1 = -V Psi^(p-1)_1 + E^(p) psi_hat + sum_{l=1}^{p-2} E^(p-l) Psi^(l)_1
// E is stored as dE[q*kp + j] = E^(q)_j.
__global__ void k_rhs_coefs(const double* dE, int p, int k, int kp, float2* c, bool f64) {
  const int j = threadIdx.x;
  if (j >= kp) return;
  const double e0 = dE[j];
  for (int l = 1; l <= p - 2; ++l) {
    const double el = (j < k) ? dE[(p - l) * kp + j] : 0.0;
    c[kRhsBig + (l - 1) * 8 + j] = (j < k) ? slot_put(-el / e0, f64) : make_float2(0.f, 0.f);
    c[kRhsSmall + l * 8 + j] = (j < k) ? slot_put(el, f64) : make_float2(0.f, 0.f);
  }
  c[kRhsSmall + j] = (j < k) ? slot_put(dE[p * kp + j], f64) : make_float2(0.f, 0.f);
}

__global__ void k_inv_norm_coef(const double* d, int k, int kp, float2* out, bool f64) {
  const int j = threadIdx.x;
  if (j < kp) out[j] = (j < k && d[j] > 0.0) ? slot_put(1.0 / sqrt(d[j]), f64) : make_float2(0.f, 0.f);
}

__global__ void k_neg_coef(const float2* in, int k, int kp, float2* out, bool f64) {
  const int j = threadIdx.x;
  if (j < kp) out[j] = (j < k) ? slot_put(-slot_get(in[j], f64), f64) : make_float2(0.f, 0.f);
}

// Deflation coefficients of the small solves: D[v][c] = G[v][c] / (E_v - E_c) for
// the small eigensolve's vectors v < b other than column c's own psi_hat_c
// (G = Psi_b^T b1, FP64, b x 8), zero elsewhere; x_defl = Psi_b D solves the
// system exactly on span(Psi_b) minus psi_hat_c.
__global__ void k_defl_coefs(const double* G, const double* Eb, int b, int k, float2* D, bool f64) {
  const int t = threadIdx.x;  // 16 x 8 entries, one thread each
  if (t >= 128) return;
  const int v = t >> 3, c = t & 7;
  double d = 0.0;
  if (v < b && c < k && v != c) d = G[v * 8 + c] / (Eb[v] - Eb[c]);
  D[t] = slot_put(d, f64);
}

// RMM-DIIS: theta_j = (x^T w) / (x^T x) per column (dots at d[0..kp) = x^T x,
// d[kp..2kp) = x^T w); -theta as a double-float coefficient and theta in FP64.
__global__ void k_rmm_theta(const double* d, int k, int kp, float2* negth, double* th) {
  const int j = threadIdx.x;
  if (j >= kp) return;
  const double t = (j < k && d[j] > 0.0) ? d[kp + j] / d[j] : 0.0;
  th[j] = t;
  negth[j] = df_from_double(-t);
}

// RMM-DIIS history step, one thread per column: the nh active ring slots end at
// `cur` (slot[t] = cur - nh + 1 + t mod nslot); g (nh x kp, FP64) holds
// r_slot[t]^T r_cur; G (kp x 8 x 8) is each column's Gram of the stored
// residuals, updated in row/column `cur`.  Solves [G 1; 1^T 0][c; mu] = [0; 1] (G's diagonal raised by 1e-14 of
// its largest entry) by Gaussian elimination with partial pivoting and writes
// the coefficients per slot (coef[slot * 8 + j], double-float; zero for
// inactive slots).  Frozen columns get c = e_cur.  status[j] = 1 on a singular
// system (then also c = e_cur).
__global__ void k_diis(const double* g, int nslot, int cur, int nh, double* G, const int* frozen, int k, int kp,
                       float2* coef, int* status) {
  const int j = threadIdx.x;
  if (j >= kp) return;
  double* Gj = G + (size_t)j * 64;
  int slot[8];
  for (int t = 0; t < nh; ++t) slot[t] = (cur - (nh - 1) + t + nslot) % nslot;
  for (int t = 0; t < nh; ++t) {
    Gj[cur * 8 + slot[t]] = g[t * kp + j];
    Gj[slot[t] * 8 + cur] = g[t * kp + j];
  }
  double c[8];
  for (int a = 0; a < 8; ++a) c[a] = 0.0;
  bool ok = j < k && !frozen[j];
  if (ok) {
    double M[9][10];
    const int m = nh;
    double mx = 0.0;
    for (int t = 0; t < m; ++t) mx = fmax(mx, Gj[slot[t] * 8 + slot[t]]);
    for (int a = 0; a < m; ++a) {
      for (int b = 0; b < m; ++b) M[a][b] = Gj[slot[a] * 8 + slot[b]];
      M[a][a] += 1e-14 * fmax(mx, 1e-300);
      M[a][m] = 1.0;
      M[a][m + 1] = 0.0;
    }
    for (int b = 0; b < m; ++b) M[m][b] = 1.0;
    M[m][m] = 0.0;
    M[m][m + 1] = 1.0;
    const int N = m + 1;
    for (int col = 0; col < N && ok; ++col) {
      int piv = col;
      for (int r = col + 1; r < N; ++r)
        if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
      if (!(fabs(M[piv][col]) > 0.0)) {
        ok = false;
        break;
      }
      if (piv != col)
        for (int q = 0; q <= N; ++q) {
          const double t = M[col][q];
          M[col][q] = M[piv][q];
          M[piv][q] = t;
        }
      for (int r = col + 1; r < N; ++r) {
        const double f = M[r][col] / M[col][col];
        for (int q = col; q <= N; ++q) M[r][q] -= f * M[col][q];
      }
    }
    if (ok) {
      double x[9];
      for (int r = N - 1; r >= 0; --r) {
        double t = M[r][N];
        for (int q = r + 1; q < N; ++q) t -= M[r][q] * x[q];
        x[r] = t / M[r][r];
      }
      for (int t = 0; t < m; ++t) c[slot[t]] = x[t];
    } else if (j < k && !frozen[j]) {
      status[j] = 1;
    }
  }
  if (!ok) c[cur] = 1.0;
  for (int a = 0; a < 8; ++a) coef[a * 8 + j] = (j < k) ? df_from_double(c[a]) : make_float2(0.f, 0.f);
}

// RMM-DIIS trial vector: Y = Xb - lam_j Rb / (D - theta_j), every |D_i - theta_j|
// clamped to >= clamp (Jacobi preconditioner); lam_j = 0 keeps Xb.
__global__ void k_rmm_step(const float2* __restrict__ Xb, const float2* __restrict__ Rb,
                           const float2* __restrict__ diag, const double* __restrict__ th,
                           const double* __restrict__ lam, float clamp, int k, int kp, int64_t n, float2* Y) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n * kp) return;
  const int64_t i = t / kp;
  const int j = static_cast<int>(t % kp);
  if (j >= k || lam[j] == 0.0) {
    Y[t] = j < k ? Xb[t] : make_float2(0.f, 0.f);
    return;
  }
  float2 den = df_sub(diag[i], df_from_double(th[j]));
  if (fabsf(den.x) < clamp) den = make_float2(den.x < 0.f ? -clamp : clamp, 0.f);
  const float2 step = df_mul(df_from_double(lam[j]), df_div(Rb[t], den));
  Y[t] = df_sub(Xb[t], step);
}

__global__ void k_neg_dots_to_coef(const double* d, int k, int kp, float2* out, bool f64) {
  const int j = threadIdx.x;
  if (j < kp) out[j] = (j < k) ? slot_put(-d[j], f64) : make_float2(0.f, 0.f);
}

// Coefficient matrix for X - A C given C (FP64, (na*kp) x kp): writes -C as double-float.
__global__ void k_negmat(const double* C, int count, float2* out, bool f64) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = slot_put(-C[i], f64);
}

__global__ void k_addmat(const double* A, const double* B, int count, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = A[i] + B[i];
}

// R = R2 * R1 (kp x kp upper triangular FP64), stored as double-float rows
// [dst + p*kp*kp ...] of the recycle coefficient matrix; Cacc (p*kp x kp) goes first.
__global__ void k_recycle_coefs(const double* Cacc, int p, int kp, const double* R2, const double* R1, float2* dst, bool f64) {
  const int t = threadIdx.x;
  for (int i = t; i < p * kp * kp; i += blockDim.x) dst[i] = slot_put(Cacc[i], f64);
  for (int e = t; e < kp * kp; e += blockDim.x) {
    const int i = e / kp, j = e % kp;
    double s = 0.0;
    for (int l = 0; l < kp; ++l) s += R2[i * kp + l] * R1[l * kp + j];
    dst[p * kp * kp + e] = slot_put(s, f64);
  }
}

// Border of the projected matrix (Eq. proj): B = Q_{0..p}^T W_p in padded layout
// ((p+1)*kp x kp).  Writes the compact m x m matrix (ld mmax), symmetrising the new
// diagonal block and mirroring the border.
__global__ void k_assemble_ht(const double* B, int p, int k, int kp, double* Ht, int ld) {
  const int t = threadIdx.x;
  const int rows = (p + 1) * k;
  for (int e = t; e < rows * k; e += blockDim.x) {
    const int r = e / k, j = e % k;
    const int a = r / k, i = r % k;
    const double v = B[(a * kp + i) * kp + j];
    const int R = a * k + i, Cc = p * k + j;
    if (a < p) {
      Ht[R * ld + Cc] = v;
      Ht[Cc * ld + R] = v;
    } else {
      const double w = B[(a * kp + j) * kp + i];
      Ht[R * ld + Cc] = 0.5 * (v + w);
    }
  }
}

// Ritz coefficients Y (compact m x k, ld k) -> padded double-float ((p+1)*kp x kp);
// theta -> double-float per column.
__global__ void k_expand_y(const double* V, int ldv, int p, int k, int kp, const double* th, float2* Y,
                           float2* thdf, bool f64) {
  const int t = threadIdx.x;
  const int rows = (p + 1) * kp;
  for (int e = t; e < rows * kp; e += blockDim.x) {
    const int r = e / kp, j = e % kp;
    const int a = r / kp, i = r % kp;
    Y[e] = (i < k && j < k) ? slot_put(V[(a * k + i) * ldv + j], f64) : make_float2(0.f, 0.f);
  }
  if (t < kp) thdf[t] = (t < k) ? slot_put(th[t], f64) : make_float2(0.f, 0.f);
}

// Thick restart: coefficients of output block b (Ritz vectors b*k .. b*k+k-1) in
// the padded layout of the block update: out[(a*kp+i)*kp + j] = V[(a*k+i)*ldv + b*k + j].
__global__ void k_restart_coef(const double* V, int ldv, int p, int k, int kp, int b, float2* out, bool f64) {
  const int t = threadIdx.x;
  const int rows = (p + 1) * kp;
  for (int e = t; e < rows * kp; e += blockDim.x) {
    const int r = e / kp, j = e % kp;
    const int a = r / kp, i = r % kp;
    out[e] = (i < k && j < k) ? slot_put(V[(a * k + i) * ldv + b * k + j], f64) : make_float2(0.f, 0.f);
  }
}

// Coefficient sub-block for block updates of multi-block sets: out[(a*8+i)*8+j] =
// src[(a*8+i)*lds + ob*8 + j] for a < na.
__global__ void k_subblock(const float2* src, int lds, int na, int ob, float2* out) {
  const int t = threadIdx.x;
  for (int e = t; e < na * 64; e += blockDim.x) {
    const int r = e / 8, j = e % 8;
    out[e] = src[r * lds + ob * 8 + j];
  }
}

// V (m x nev FP64, ld nev) -> double-float rotation coefficients (m x m padded to 16x16 ld 16)
// -theta_c (c < b, else 0) of the small eigensolve's residual columns
__global__ void k_neg_theta(const double* th, int b, float2* out, bool f64) {
  const int c = threadIdx.x;
  if (c < 8) out[c] = slot_put(c < b ? -th[c] : 0.0, f64);
}

__global__ void k_vmat_df(const double* V, int m, int nev, int ldv, float2* out, bool f64) {
  const int t = threadIdx.x;
  for (int e = t; e < 256; e += blockDim.x) {
    const int i = e / 16, j = e % 16;
    out[e] = (i < m && j < nev) ? slot_put(V[i * ldv + j], f64) : make_float2(0.f, 0.f);
  }
}

// ------------------------------------------------------------ SELL builder

void split_df(double x, float2& out) {
  const float h = static_cast<float>(x);
  out.x = h;
  out.y = static_cast<float>(x - static_cast<double>(h));
}

// x into a value slot of the given format (double-float pair, or the bits of x)
void put_slot(double x, float2& out, bool f64) {
  if (f64)
    std::memcpy(&out, &x, sizeof(double));
  else
    split_df(x, out);
}

// FP32 -> nearest BF16 (ties to even), returned as FP32; finite inputs only
// (an input whose rounding overflows becomes Inf and is rejected by validation)
float round_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// Rows [0, nrows), columns [0, ncols) cut into chunks of chunk_cols columns
// (chunk_cols <= 0: one chunk).  For every chunk, inside every segment (level)
// `seg`, the rows with entries in the chunk are sorted by decreasing entry count
// within windows of `sigma` rows (stable) and cut into slices of kSliceH rows.  Rows
// without any entry are listed in chunk 0 so that their output is written.
void build_sell(int64_t nrows, const int64_t* rp, const int32_t* ci, const double* va, int64_t ncols,
                const std::vector<int64_t>& seg, int64_t sigma, int64_t chunk_cols, bool f64, SellHost& S) {
  const int64_t C = (chunk_cols > 0 && chunk_cols < ncols) ? chunk_cols : ncols;
  const int nch = (int)((ncols + C - 1) / C);
  S.nchunks = nch;
  S.chunk_cols = C;
  const int W = nch + 1;
  std::vector<int64_t> off((size_t)nrows * W);
  S.first.assign(nrows, 0);
  S.last.assign(nrows, 0);
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nrows; ++r) {
    const int32_t* b = ci + rp[r];
    const int32_t* e = ci + rp[r + 1];
    int fq = -1, lq = 0;
    for (int q = 0; q <= nch; ++q) {
      const int64_t lim = std::min<int64_t>((int64_t)q * C, ncols);
      off[(size_t)r * W + q] = std::lower_bound(b, e, (int32_t)std::min<int64_t>(lim, INT32_MAX)) - b;
      if (q > 0 && off[(size_t)r * W + q] > off[(size_t)r * W + q - 1]) {
        if (fq < 0) fq = q - 1;
        lq = q - 1;
      }
    }
    S.first[r] = (uint8_t)(fq < 0 ? 0 : fq);
    S.last[r] = (uint8_t)lq;
  }
  auto len_of = [&](int64_t r, int q) { return off[(size_t)r * W + q + 1] - off[(size_t)r * W + q]; };
  std::vector<int32_t> slice_chunk;
  S.chunk_slice.assign(nch + 1, 0);
  S.slice_ptr.assign(1, 0);
  S.rows.clear();
  for (int q = 0; q < nch; ++q) {
    S.chunk_slice[q] = (int64_t)slice_chunk.size();
    for (size_t sgi = 0; sgi + 1 < seg.size(); ++sgi) {
      std::vector<int32_t> part;
      for (int64_t r = seg[sgi]; r < seg[sgi + 1]; ++r) {
        const bool empty_row = off[(size_t)r * W + nch] == 0;
        if (len_of(r, q) > 0 || (q == 0 && empty_row)) part.push_back((int32_t)r);
      }
      const int64_t np = (int64_t)part.size();
#pragma omp parallel for schedule(dynamic, 4)
      for (int64_t w0 = 0; w0 < np; w0 += sigma) {
        std::stable_sort(part.begin() + w0, part.begin() + std::min(w0 + sigma, np),
                         [&](int32_t x, int32_t y) { return len_of(x, q) > len_of(y, q); });
      }
      for (int64_t s0 = 0; s0 < np; s0 += kSliceH) {
        int64_t w = 0;
        for (int l = 0; l < kSliceH; ++l) {
          const int32_t r = (s0 + l < np) ? part[s0 + l] : -1;
          S.rows.push_back(r);
          if (r >= 0) w = std::max<int64_t>(w, len_of(r, q));
        }
        S.slice_ptr.push_back(S.slice_ptr.back() + kSliceH * w);
        slice_chunk.push_back(q);
      }
    }
  }
  S.chunk_slice[nch] = (int64_t)slice_chunk.size();
  const int64_t ns = (int64_t)slice_chunk.size();
  S.nslices = ns;
  S.col.assign(S.slice_ptr[ns], 0);
  S.val.assign(S.slice_ptr[ns], make_float2(0.f, 0.f));
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t s = 0; s < ns; ++s) {
    const int q = slice_chunk[s];
    const int64_t base = S.slice_ptr[s];
    const int64_t w = (S.slice_ptr[s + 1] - base) / kSliceH;
    const int32_t pad_col = (int32_t)std::min<int64_t>((int64_t)q * C, ncols - 1);
    for (int l = 0; l < kSliceH; ++l) {
      const int32_t r = S.rows[s * kSliceH + l];
      const int64_t lr = (r >= 0) ? len_of(r, q) : 0;
      const int64_t o0 = (r >= 0) ? rp[r] + off[(size_t)r * W + q] : 0;
      for (int64_t t = 0; t < w; ++t) {
        const int64_t o = base + kSliceH * t + l;
        if (t < lr) {
          S.col[o] = ci[o0 + t];
          put_slot(va[o0 + t], S.val[o], f64);
        } else {
          S.col[o] = pad_col;
        }
      }
    }
  }
}

sppc_status upload_sell(sppc_ctx* h, SellHost& S, SellDev& D, int64_t nrows, std::vector<int64_t>& chunk_store) {
  int64_t* sp;
  int32_t *rows, *col;
  float2* val;
  uint8_t *fr, *la;
  CK(dalloc(h, &sp, S.slice_ptr.size()));
  CK(dalloc(h, &rows, S.rows.size()));
  CK(dalloc(h, &col, S.col.size()));
  CK(dalloc(h, &val, S.val.size()));
  CK(dalloc(h, &fr, S.first.size()));
  CK(dalloc(h, &la, S.last.size()));
  CK(cudaMemcpyAsync(sp, S.slice_ptr.data(), sizeof(int64_t) * S.slice_ptr.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(rows, S.rows.data(), sizeof(int32_t) * S.rows.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(col, S.col.data(), sizeof(int32_t) * S.col.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(val, S.val.data(), sizeof(float2) * S.val.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(fr, S.first.data(), S.first.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(la, S.last.data(), S.last.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  chunk_store = S.chunk_slice;
  D.nslices = S.nslices;
  D.nrows = nrows;
  D.nchunks = S.nchunks;
  D.chunk_cols = S.chunk_cols;
  D.chunk_slice = chunk_store.data();
  D.slice_ptr = sp;
  D.slice_rows = rows;
  D.col = col;
  D.val = val;
  D.row_first = fr;
  D.row_last = la;
  return SPPC_OK;
}

// Products with H0_hat: a few thousand rows leave each SELL lane pair a long
// chain of dependent gathers, so up to kCsrRowsMax rows the CSR kernel (8 lanes
// per row) runs them; the SELL layout above that.
constexpr int64_t kCsrRowsMax = 65536;
cudaError_t spmm11(const sppc_ctx* h, int kp, const float2* X, float2* Y, const Epi& e, cudaStream_t s) {
  if (h->H11c.rowptr && h->H11c.nrows <= kCsrRowsMax) return spmm_csr(h->H11c, kp, X, Y, e, s);
  return spmm(h->H11, kp, X, Y, e, s);
}

cudaError_t spmm11_set(const sppc_ctx* h, int kp, const float2* const* X, float2* const* Y, const float2* const* Z,
                       int nb, Epi e, cudaStream_t s) {
  if (nb == 2 && h->H11c.rowptr && h->H11c.nrows <= kCsrRowsMax) return spmm_csr2(h->H11c, kp, X, Y, Z, e, s);
  for (int a = 0; a < nb; ++a) {
    if (Z) e.Z = Z[a];
    const cudaError_t r = spmm11(h, kp, X[a], Y[a], e, s);
    if (r != cudaSuccess) return r;
  }
  return cudaSuccess;
}

// H0_hat (rows and columns < n1 of H) as CSR with double-float values.
// Leading block H[:n1, :n1] as a double-float CSR on the device (columns sorted
// within each row, so a row's block entries are its first ones).
sppc_status upload_csr11(sppc_ctx* h, int64_t n1, const int64_t* rp, const int32_t* ci, const double* va,
                         CsrDev& out) {
  std::vector<int64_t> p(n1 + 1, 0);
  for (int64_t r = 0; r < n1; ++r) {
    int64_t c = 0;
    for (int64_t t = rp[r]; t < rp[r + 1] && ci[t] < n1; ++t) ++c;
    p[r + 1] = p[r] + c;
  }
  std::vector<int32_t> col(std::max<int64_t>(p[n1], 1));
  std::vector<float2> val(std::max<int64_t>(p[n1], 1));
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < n1; ++r)
    for (int64_t t = 0; t < p[r + 1] - p[r]; ++t) {
      col[p[r] + t] = ci[rp[r] + t];
      put_slot(va[rp[r] + t], val[p[r] + t], h->f64);
    }
  int64_t* drp;
  int32_t* dcol;
  float2* dval;
  CK(dalloc(h, &drp, p.size()));
  CK(dalloc(h, &dcol, col.size()));
  CK(dalloc(h, &dval, val.size()));
  CK(cudaMemcpyAsync(drp, p.data(), sizeof(int64_t) * p.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(dcol, col.data(), sizeof(int32_t) * col.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(dval, val.data(), sizeof(float2) * val.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  out.nrows = n1;
  out.rowptr = drp;
  out.col = dcol;
  out.val = dval;
  out.f64 = h->f64;
  return SPPC_OK;
}

// ---------------------------------------------------------- timing helpers
cudaEvent_t next_event(sppc_ctx* h) {
  if (h->evnext >= (int)h->evpool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->evpool.push_back(e);
  }
  return h->evpool[h->evnext++];
}

sppc_status collect_timing(sppc_ctx* h) {
  for (auto& pr : h->pending) {
    float ms = 0.f;
    CK(cudaEventSynchronize(pr.second));
    CK(cudaEventElapsedTime(&ms, pr.first, pr.second));
    h->stats.spmm_ms += ms;
  }
  h->pending.clear();
  h->evnext = 0;
  return SPPC_OK;
}

// The big SpMM W_p = H q^(p) (k SpMVs of the order), timed when opts.timing.
sppc_status big_spmm(sppc_ctx* h, const float2* X, float2* Y, int kp) {
  if (h->Wd && Y >= h->W && Y < h->W + (int64_t)(h->pmax + 1) * h->n * kp)
    h->wd_valid &= ~(1ull << ((Y - h->W) / (h->n * kp)));  // this W block is rewritten
  cudaEvent_t a = nullptr, b = nullptr;
  if (h->opt.timing) {
    a = next_event(h);
    b = next_event(h);
    CK(cudaEventRecord(a, h->stream));
  }
  if (h->f32_products && (kp == 4 || kp == 8))
    CK(spmm_f32(h->H, h->val32, h->val16, h->diag32, X, h->X32, Y, kp, h->stream));
  else
    CK(spmm(h->H, kp, X, Y, Epi{}, h->stream));
  if (h->opt.timing) {
    CK(cudaEventRecord(b, h->stream));
    h->pending.push_back({a, b});
  }
  h->stats.spmm_launches += 1;
  return SPPC_OK;
}


}  // namespace sppc::drv
