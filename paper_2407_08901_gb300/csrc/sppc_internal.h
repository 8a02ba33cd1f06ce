// Internal interfaces between the host driver (api.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sppc {

constexpr int kMaxBlocks = 40;  // basis blocks a launch can address (p_max + 2)

// Level-blocked SELL-32 matrix on the device.  Slice s holds 32 rows (lanes);
// its entries are stored column-major: entry t of lane l sits at
// slice_ptr[s] + 32*t + l.  slice_rows[32*s + l] is the original row index of
// lane l (-1 for a padding lane).  Padding entries have value 0.
struct SellDev {
  int64_t nslices = 0;
  int64_t nrows = 0;
  const int64_t* slice_ptr = nullptr;
  const int32_t* slice_rows = nullptr;
  const int32_t* col = nullptr;
  const float2* val = nullptr;  // double-float values
};

// SpMM epilogue: Y[r][c] = alpha[c] * (A X)[r][c] + beta[c] * X[r][c] + gamma[c] * Z[r][c].
// Coefficient arrays are double-float per column on the device; a null alpha
// means 1, a null beta/gamma means the term is absent.
struct Epi {
  const float2* alpha = nullptr;
  const float2* beta = nullptr;
  const float2* gamma = nullptr;
  const float2* Z = nullptr;
};

// A list of row-major n x kp double-float blocks (same row indexing).
struct BlockList {
  const float2* p[kMaxBlocks];
  int n = 0;
};

// ---- k_spmm.cu
cudaError_t spmm(const SellDev& A, int kp, const float2* X, float2* Y, const Epi& epi, cudaStream_t s);
int spmm_default_grid();

// ---- k_dense.cu
// Gram: out[(a*kp+i)*kp + j] = sum_{r in [r0,r1)} A_a[r][i] * B[r][j]  (FP64 out)
cudaError_t gram(const BlockList& A, const float2* B, int kp, int64_t r0, int64_t r1, double* out,
                 float2* partials, int64_t partial_cap, cudaStream_t s);
// Update: Y[r][j] = alpha[j] X[r][j] + sum_a sum_i A_a[r][i] coef[(a*kp+i)*kp + j]
// (coef double-float on device; X may be null; Y may alias X).
cudaError_t update(float2* Y, const float2* X, const float2* alpha, const BlockList& A, const float2* coef,
                   int kp, int64_t r0, int64_t r1, cudaStream_t s);
// Diagonal combine: Y[r][j] = alpha[j] X[r][j] + sum_b coef[b*8 + j] A_b[r][j]
// (coefficients of block b at stride 8 whatever kp is)
cudaError_t combine_diag(float2* Y, const float2* X, const float2* alpha, const BlockList& A,
                         const float2* coef, int kp, int64_t r0, int64_t r1, cudaStream_t s);
// Column dots: out[q*kp + j] = sum_r A_q[r][j] * B_q[r][j], q < nq <= 4 (FP64 out)
cudaError_t coldots(const float2* const* A, const float2* const* B, int nq, int kp, int64_t r0, int64_t r1,
                    double* out, float2* partials, int64_t partial_cap, cudaStream_t s);
// Ritz residual: for every row, z = sum_a Q_a[r] Y_a, hz = sum_a W_a[r] Y_a (Y: (na*kp) x kp
// double-float), accumulate (hz - theta*z)^2 per column -> out[j] (FP64); optionally
// write z (FP64, leading dim ldz, first ncols columns) to Zout.
cudaError_t ritz_resid(const BlockList& Q, const BlockList& Wb, const float2* Y, const float2* theta, int kp,
                       int64_t n, double* out, float2* partials, int64_t partial_cap, double* Zout, int64_t ldz,
                       int ncols, cudaStream_t s);
cudaError_t f64_to_df(const double* X, int64_t ldx, int ncols, float2* Y, int kp, int64_t r0, int64_t r1,
                      cudaStream_t s);
cudaError_t df_to_f64(const float2* X, int kp, double* Y, int64_t ldy, int ncols, int64_t r0, int64_t r1,
                      cudaStream_t s);
cudaError_t fill_zero(float2* Y, int64_t count, cudaStream_t s);

// ---- k_small.cu (single-CTA FP64 kernels on small matrices)
// Cholesky of the leading kk x kk part of G (ld = ldg) plus `shift` on the diagonal;
// writes R (upper, kk x kk, ld kp, FP64), Rinv as double-float coefficient matrix
// (kp x kp, identity on padding), and status[0] = 0 ok / j+1 breakdown at pivot j.
cudaError_t chol_rinv(const double* G, int ldg, int kk, int kp, double shift_rel, double* R, float2* Rinv_df,
                      int* status, cudaStream_t s);
// Symmetric eigensolve: S (m x m, ld lds), nev lowest eigenpairs -> theta[nev],
// V (m x nev, ld ldv) FP64; ascending.  m <= 160.
cudaError_t syev_lowest(const double* S, int lds, int m, int nev, double* theta, double* V, int ldv,
                        cudaStream_t s);
// Generic small-array FP64 kernels used by the driver.
cudaError_t to_df(const double* x, float2* y, int count, double scale, cudaStream_t s);
cudaError_t negate_to_df(const double* x, float2* y, int count, cudaStream_t s);

}  // namespace sppc
