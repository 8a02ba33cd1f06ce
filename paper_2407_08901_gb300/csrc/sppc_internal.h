// Internal interfaces between the host driver (api.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <vector>

namespace sppc {

// Kernel launches issued by the library since load (every launch site counts).
void count_launch();
long long launch_count();

constexpr int kMaxBlocks = 40;  // basis blocks a launch can address (p_max + 2)
constexpr int kSliceH = 16;     // rows per SELL slice (one warp, two lanes per row)

// Level-blocked SELL-16 matrix on the device, tiled by column chunks.  The
// columns are cut into `nchunks` ranges of `chunk_cols` columns; chunk q owns
// slices [chunk_slice[q], chunk_slice[q+1]).  Slice s holds kSliceH rows and
// the row's entries whose columns fall in the slice's chunk, stored
// column-major: entry t of slice row l sits at slice_ptr[s] + kSliceH*t + l.
// slice_rows[kSliceH*s + l] is the original row index (-1 = padding row).
// Padding entries have value 0.  row_first/row_last give, per row, the first and
// last chunk holding one of its entries (0 for an empty row, which chunk 0 lists).
struct SellDev {
  int64_t nslices = 0;
  int64_t nrows = 0;
  int nchunks = 1;
  int64_t chunk_cols = 0;
  const int64_t* chunk_slice = nullptr;  // host array, nchunks + 1
  const int64_t* slice_ptr = nullptr;
  const int32_t* slice_rows = nullptr;
  const int32_t* col = nullptr;
  const float2* val = nullptr;  // double-float values
  const uint8_t* row_first = nullptr;
  const uint8_t* row_last = nullptr;
  bool f64 = false;  // value format of val and of the vectors it multiplies: IEEE double (true) or double-float
  int tma = 0;  // 1: 8-column products use the TMA-gather kernel (k_spmm_tma.cu; double-float only)
  int* tma_flag = nullptr;  // device word the TMA kernel sets when an mbarrier wait gives up
  unsigned spin_limit = 0;  // TMA kernel: polls before a wait gives up (0 = about a second of clock)
};

// CSR matrix on the device with double-float values (rowptr has nrows + 1
// entries; column indices strictly increasing within a row).
struct CsrDev {
  int64_t nrows = 0;
  const int64_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const float2* val = nullptr;
  bool f64 = false;  // value format (see SellDev)
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

// ---- sell_build.cu: the SELL-16 layout of H built on the GPU from its CSR on the
// device (rp, ci, va), bit-identical to the host builder; values stored as slots
// of the given format (f64: IEEE double bits, else double-float pairs).  Persistent arrays come
// from `alloc` (bytes); temporaries are stream-ordered allocations freed before
// return.  Synchronises the stream.
using DeviceAlloc = std::function<cudaError_t(void**, size_t)>;
struct SellDeviceLayout {
  int64_t nslices = 0, chunk_cols = 0, total = 0;
  int nchunks = 1;
  std::vector<int64_t> chunk_slice, slice_ptr;  // host copies
  std::vector<int32_t> rows;                    // host copy
  int64_t* slice_ptr_d = nullptr;
  int32_t* rows_d = nullptr;
  int32_t* col_d = nullptr;
  float2* val_d = nullptr;
  uint8_t* first_d = nullptr;
  uint8_t* last_d = nullptr;
};
// round_mode: the values as opts.precision stores them (0 as given, 1 FP32,
// 2 FP32 diagonal and BF16 off-diagonal entries).
cudaError_t build_sell_device(int64_t nrows, const int64_t* rp, const int32_t* ci, const double* va, int64_t ncols,
                              const std::vector<int64_t>& seg, int64_t chunk_cols, bool f64, int round_mode,
                              cudaStream_t s, const DeviceAlloc& alloc, SellDeviceLayout& out, int sigma = 1024);
// Checks of a CSR that stays on the device: *flags_host gets 2 (column out of
// range), 4 (columns not strictly increasing), 8 (NaN/Inf) and, with symmetry,
// 1 (H != H^T bit for bit).  Synchronises the stream.
cudaError_t csr_check_device(int64_t n, const int64_t* rp, const int32_t* ci, const double* va, bool symmetry,
                             int* flags_host, cudaStream_t s);
// diag[r] = H_rr of a device CSR (0 when not stored), rounded per round_mode, as a slot
cudaError_t csr_diag_device(int64_t n, const int64_t* rp, const int32_t* ci, const double* va, int round_mode,
                            bool f64, float2* diag, cudaStream_t s);

// ---- k_spmm.cu
cudaError_t spmm(const SellDev& A, int kp, const float2* X, float2* Y, const Epi& epi, cudaStream_t s);
int spmm_default_grid();
// The same product (and epilogue) for a CSR matrix of few rows: 8 lanes per row
// (latency of the gather chains, not bandwidth, sets the time there).
cudaError_t spmm_csr(const CsrDev& A, int kp, const float2* X, float2* Y, const Epi& epi, cudaStream_t s);
// spmm_csr on two blocks in one launch (Y[b] = epilogue(A X[b]), with Z[b] as the
// epilogue's Z when Z is given): the same results as two spmm_csr calls.
cudaError_t spmm_csr2(const CsrDev& A, int kp, const float2* const X[2], float2* const Y[2], const float2* const Z[2],
                      const Epi& epi, cudaStream_t s);

// ---- k_spmm_f32.cu (mixed precision, kp = 4 or 8 columns): X (double-float)
// rounded to FP32 into X32 (n x kp floats), Y = H X with FP32 values val32 (same
// SELL layout as A) and FP32 accumulation, written as double-float with zero low
// words.  With val16 != nullptr the values are BF16 (diagonal entries 0) and
// diag32 holds the FP32 diagonal; val32 is then unused.
cudaError_t spmm_f32(const SellDev& A, const float* val32, const uint16_t* val16, const float* diag32,
                     const float2* X, float* X32, float2* Y, int kp, cudaStream_t s);
// Y = |H| X32 (entrywise absolute values; X32 FP32 n x 8, Y n x 8, prepared by the caller)
cudaError_t spmm_abs_f32(const SellDev& A, const float* val32, const uint16_t* val16, const float* diag32,
                         const float* X32, float2* Y, cudaStream_t s);
// val16[e] = BF16 bits of A.val[e].x (BF16-exact values), 0 for diagonal entries
cudaError_t make_val16(const SellDev& A, uint16_t* val16, cudaStream_t s);
// out[i] = in[i].x (the FP32 high words of double-float values)
cudaError_t df_hi_parts(const float2* in, float* out, int64_t count, cudaStream_t s);

// ---- k_spmm_batch.cu: Y_m = H_m X_m for many matrices in one persistent launch
// (device work queue over the matrices' slices; untiled layouts)
struct BatchItem {
  SellDev A;
  const float2* X;  // n_m x kp double-float
  float2* Y;        // n_m x kp double-float
};
// items, prefix (nitems + 1 global slice offsets) and queue (one counter) on the device
cudaError_t spmm_batch(const BatchItem* items, int nitems, const int64_t* prefix, int64_t total, int kp,
                       unsigned long long* queue, cudaStream_t s);

// ---- k_learned.cu: learned correction proposal (network 6 -> 64 -> 64 -> 1)
constexpr int kNetFeatures = 6, kNetHidden = 64;
constexpr int kNetParams = kNetHidden * kNetFeatures + kNetHidden + kNetHidden * kNetHidden + kNetHidden +
                           kNetHidden + 1;  // 4,673
// out[s] = network output for standardised sample X[s] (count x 6); bf16: BF16 inference
cudaError_t mlp_forward(const float* params, const float* X, int64_t count, bool bf16, float* out, cudaStream_t s);
// Minibatch gradient of L = inv_b * sum_s (rhat_s (1 + m_s) - y_s)^2 over samples
// perm[base + s] (or base + s), s < count; part holds mlp_grad_part_floats(count)
// floats; grad[kNetParams]; *loss_slot (device, nullable) = L.
cudaError_t mlp_grad(const float* params, const float* X, const float* rhat, const float* y, const int64_t* perm,
                     int64_t base, int64_t count, float inv_b, float* part, float* grad, float* loss_slot,
                     cudaStream_t s);
int64_t mlp_grad_part_floats(int64_t batch);
// Adam update; c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
cudaError_t mlp_adam(float* params, float* mom, float* vel, const float* grad, float lr, float b1, float b2,
                     float eps, float c1, float c2, cudaStream_t s);
// out[i] = (level(i), ||H_i,:||_2) from a device CSR and device level offsets
cudaError_t row_consts(int64_t n, const int64_t* rp, const double* va, const int64_t* lev, int nlev, float2* out,
                       cudaStream_t s);
// rhat (n x 8) and |rhat| (n x 8) from the residual block R (n x kp) and ||r_j||^2
cudaError_t prop_prep(const float2* R, int kp, int k, const double* rn2, int64_t n, float* rhat, float* absr,
                      cudaStream_t s);
// proposal rows [n0, n): Tprop = (R / den)(1 + m), Tplain = R / den (n x kp)
cudaError_t prop_mlp(const float* net, const float2* R, const float2* diag, const float2* rowc, const float* rhat,
                     const float2* agg, const float2* theta, float clamp, int k, int kp, int64_t n0, int64_t n,
                     float2* Tprop, float2* Tplain, cudaStream_t s);
// training samples (rows [n0, n), pairs j < k): raw features F, rhat, target y
cudaError_t prop_samples(const float2* R, const double* Z, int64_t ldz, const double* psi, int64_t ldpsi,
                         const double* rn2, const float2* diag, const float2* rowc, const float* rhat,
                         const float2* agg, const float2* theta, float clamp, int k, int kp, int64_t n0, int64_t n,
                         double* scratch, float* F, float* rh_out, float* y, cudaStream_t s);
int64_t prop_samples_scratch_doubles();
// mean and spread (population) of each feature over `count` samples: written to
// scratch[feature_moments_scratch_doubles() - 12 ...] as mean[6], sd[6]
cudaError_t feature_moments(const float* F, int64_t count, double* scratch, cudaStream_t s);
int64_t feature_moments_scratch_doubles();
// X = (F - mu) / sd per feature (mu, sd host arrays of 6)
cudaError_t standardize(const float* F, int64_t count, const float* mu, const float* sd, float* X, cudaStream_t s);

// ---- k_spmm_tma.cu (kp = 8; X 16-byte aligned)
bool spmm_tma_available();
cudaError_t spmm_tma8(const SellDev& A, const float2* X, float2* Y, const Epi& epi, cudaStream_t s);
// Copies A's time-out flag (nonzero after an mbarrier wait of the TMA kernel gave
// up) to host memory, valid after the stream synchronises (0 without a flag).
cudaError_t spmm_tma_read_timeout(const SellDev& A, int* flag, cudaStream_t s);

// ---- k_dense.cu
// Gram: out[(a*kp+i)*kp + j] = sum_{r in [r0,r1)} A_a[r][i] * B[r][j]  (FP64 out)
cudaError_t gram(const BlockList& A, const float2* B, int kp, int64_t r0, int64_t r1, double* out,
                 float2* partials, int64_t partial_cap, bool f64, cudaStream_t s);
// Fixed-order sum of per-CTA partial results (nchunks x nout slots) into FP64 out.
// A^T A for one block (symmetric: 36 of the 64 products when kp = 8); out: kp x kp.
cudaError_t gram_sym(const float2* A, int kp, int64_t r0, int64_t r1, double* out, float2* partials,
                     int64_t partial_cap, bool f64, cudaStream_t s);
// Y = A coef for one block and an upper triangular coef (zero entries below the
// diagonal are skipped).
cudaError_t update_tri(float2* Y, const float2* A, const float2* coef, int kp, int64_t r0, int64_t r1, bool f64,
                       cudaStream_t s);
cudaError_t gram_finish(const float2* partials, int64_t nchunks, int nout, double* out, bool f64, cudaStream_t s);

// ---- k_gram_tc.cu: gram() for kp = 8 on the tensor cores against basis blocks
// (entries |q| < 2) pre-cut into FP16 digit tiles (a 62-bit fixed-point split,
// exact digit products, FP64-grade result).  The tiles of blocks 16 g .. 16 g + 15
// form group g (qdigits_group_bytes(n) bytes); qcut writes block a's tiles at
// qdigits_block(Qd, n, a); gram_tc reads blocks 0 .. nblocks - 1 and B (n x 8
// slots), rows [0, n).  *err (device, sticky): bit 0 when a value is out of range
// or not finite, bit 1 when a wait timed out.  fexp: device scratch, 8 ints.
// partials needs ceil(n / per) * 64 * min(nblocks, 16) slots (gram_tc_geometry).
int64_t qdigits_group_bytes(int64_t n);
unsigned char* qdigits_block(unsigned char* Qd, int64_t n, int a);
// colexp_dev (device, 8 ints, optional): column exponents e_i (|v| < 2^e_i) for
// blocks that are not orthonormal (H Q); the tiles are then cut at 2^(61 - e_i).
cudaError_t qcut(const float2* Q, int64_t n, unsigned char* out, bool f64, int* err, cudaStream_t s,
                 const int* colexp_dev = nullptr);
// fexp[j] (device, 8 ints) = max over rows of e with |B[r][j]| < 2^e (a very
// negative value for an all-zero column).
cudaError_t colexp(const float2* B, int64_t n, int* fexp, bool f64, cudaStream_t s);
cudaError_t gram_tc(const unsigned char* Qd, int nblocks, const float2* B, int64_t n, double* out, float2* partials,
                    int64_t partial_cap, bool f64, int* err, int* fexp, cudaStream_t s);
void gram_tc_geometry(int64_t rows, int sms, int64_t* per, int64_t* ctas);

// ---- k_update_tc.cu: update() for kp = 8 on the tensor cores against basis
// blocks 0 .. nblocks - 1 of Qd (the tiles gram_tc reads): Y = alpha X + sum_a
// Q_a coef_a, coef[(8 a + i) * 8 + j], the X term present when X and alpha are
// both given (as in update()), Y may alias X.  *err as for gram_tc (bit 0: a
// coefficient not finite).
// rowexp (device, 8 nblocks ints, optional): the blocks' column exponents when
// their tiles were cut with colexp_dev (blocks of H Q).
cudaError_t update_tc(const unsigned char* Qd, int nblocks, const float2* coef, const float2* alpha, const float2* X,
                      float2* Y, int64_t n, bool f64, int* err, cudaStream_t s, const int* rowexp = nullptr);
// Preconditioned residual block T[r][j] = D[r][j] / clamp(diag[r] - theta_j)
// (|denominator| >= clamp), or T = D without diag; theta: kp slots.
cudaError_t ritz_precond(const float2* D, const float2* theta, const float2* diag, float clamp, float2* T, int kp,
                         int64_t n, bool f64, cudaStream_t s);

// Update: Y[r][j] = alpha[j] X[r][j] + sum_a sum_i A_a[r][i] coef[(a*kp+i)*kp + j]
// (coef double-float on device; X may be null; Y may alias X but no block of A).
cudaError_t update(float2* Y, const float2* X, const float2* alpha, const BlockList& A, const float2* coef,
                   int kp, int64_t r0, int64_t r1, bool f64, cudaStream_t s);
// Diagonal combine: Y[r][j] = alpha[j] X[r][j] + sum_b coef[b*8 + j] A_b[r][j]
// (coefficients of block b at stride 8 whatever kp is)
cudaError_t combine_diag(float2* Y, const float2* X, const float2* alpha, const BlockList& A,
                         const float2* coef, int kp, int64_t r0, int64_t r1, bool f64, cudaStream_t s);
// Column dots: out[q*kp + j] = sum_r A_q[r][j] * B_q[r][j], q < nq <= 4 (FP64 out)
cudaError_t coldots(const float2* const* A, const float2* const* B, int nq, int kp, int64_t r0, int64_t r1,
                    double* out, float2* partials, int64_t partial_cap, bool f64, cudaStream_t s);
// Ritz residual: for every row, z = sum_a Q_a[r] Y_a, hz = sum_a W_a[r] Y_a (Y: (na*kp) x kp
// double-float), accumulate (hz - theta*z)^2 per column -> out[j] (FP64); optionally
// write z (FP64, leading dim ldz, first ncols columns) to Zout; optionally write
// the residual hz - theta z (double-float, n x kp) to Tout, divided elementwise by
// diag[r] - theta_j (magnitude clamped to >= clamp) when diag is given;
// optionally write z and the undivided residual of rows < nlead (double-float,
// nlead x kp) to Zlead and Rlead.
cudaError_t ritz_resid(const BlockList& Q, const BlockList& Wb, const float2* Y, const float2* theta, int kp,
                       int64_t n, double* out, float2* partials, int64_t partial_cap, double* Zout, int64_t ldz,
                       int ncols, float2* Tout, const float2* diag, float clamp, bool f64, cudaStream_t s,
                       float2* Zlead = nullptr, float2* Rlead = nullptr, int64_t nlead = 0);
// FP64 (leading dimension ldx, ncols columns) <-> value slots (kp columns, padding
// columns written as 0); f64 selects the slot format (val.cuh)
cudaError_t f64_to_df(const double* X, int64_t ldx, int ncols, float2* Y, int kp, int64_t r0, int64_t r1, bool f64,
                      cudaStream_t s);
cudaError_t df_to_f64(const float2* X, int kp, double* Y, int64_t ldy, int ncols, int64_t r0, int64_t r1, bool f64,
                      cudaStream_t s);
cudaError_t fill_zero(float2* Y, int64_t count, cudaStream_t s);

// ---- k_minres.cu
// Persistent MINRES on (A - E_k) x = b for k columns on the complement of psi
// (see k_minres.cu).  P holds b on entry; X receives the solution.
cudaError_t minres_persistent(const CsrDev& A, int k, int kp, const float2* negE, const float2* psi, float2* P,
                              float2* V, float2* VP, float2* Y, float2* W1, float2* W2, float2* X, double tol,
                              int maxit, float2* partials, int64_t partial_cap, unsigned* bar, int* status,
                              cudaStream_t s, int max_ctas = 0, int spin_cap = 0, bool fp32 = false);

// ---- k_small.cu (single-CTA FP64 kernels on small matrices)
// Cholesky of the leading kk x kk part of G (ld = ldg) plus `shift` on the diagonal;
// writes R (upper, kk x kk, ld kp, FP64), Rinv as double-float coefficient matrix
// (kp x kp, identity on padding), and status[0] = 0 ok / j+1 breakdown at pivot j.
cudaError_t chol_rinv(const double* G, int ldg, int kk, int kp, double shift_rel, double* R, float2* Rinv_df,
                      int* status, bool f64, cudaStream_t s);
// Symmetric eigensolve: S (m x m, ld lds), nev lowest eigenpairs -> theta[nev],
// V (m x nev, ld ldv) FP64; ascending.  m <= 160.
cudaError_t syev_lowest(const double* S, int lds, int m, int nev, double* theta, double* V, int ldv, bool f64,
                        cudaStream_t s);
// Generic small-array FP64 kernels used by the driver.
// y[i] = scale * x[i] as value slots (f64: the slot format)
cudaError_t to_df(const double* x, float2* y, int count, double scale, bool f64, cudaStream_t s);

}  // namespace sppc
