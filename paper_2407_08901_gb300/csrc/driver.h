// Host driver internals shared by the translation units of the C ABI: the
// handle (sppc_ctx) and its device coefficient slots, the error helpers, and the
// driver's steps of Algorithm 2 (drv_host.cu: tiny kernels, the host SELL
// builder, the big SpMM; drv_solver.cu: small eigensolve, MINRES, Gram-Schmidt,
// Rayleigh-Ritz, continuation and RMM-DIIS; api_create.cu: create, layout
// tuning; api.cu: the remaining C entry points).
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <nvtx3/nvToolsExt.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "df.cuh"
#include "val.cuh"
#include "sppc.h"
#include "sppc_internal.h"

namespace sppc::drv {

// Named NVTX ranges around the solver phases (no cost unless a tool such as
// ncu or nsys is attached; profilers can filter kernels by phase).
struct PhaseRange {
  explicit PhaseRange(const char* name) { nvtxRangePushA(name); }
  ~PhaseRange() { nvtxRangePop(); }
  PhaseRange(const PhaseRange&) = delete;
  PhaseRange& operator=(const PhaseRange&) = delete;
};

extern thread_local std::string g_create_error;

struct OrderRec {
  std::vector<double> E, angle, theta, resid;
  std::vector<int32_t> iters;
};

// Device scratch for small coefficient arrays (double-float) and FP64 scalars.
enum CoefSlot : int {
  kOnes = 0,         // 16
  kNegOnes = 16,     // 16
  kShiftNegE = 32,   // -E0 per column (MINRES operator shift)
  kInvE0 = 48,       // 1/E0
  kRhsBig = 64,      // (kMaxBlocks) x 8: -E^(p-l)/E0
  kRhsSmall = 384,   // (kMaxBlocks) x 8
  kDefl = 704,       // 8
  kMinA = 720,       // 24: {-s, -beta, -alpha} for {psi_hat, v_prev, v}
  kMinWAlpha = 744,  // 8: 1/rho1
  kMinW = 752,       // 16: {-rho3/rho1, -rho2/rho1}
  kMinX = 768,       // 8: c*eta
  kMinV = 776,       // 8: 1/beta'
  kCheb = 784,       // 3 x 16: alpha, beta, gamma of the Chebyshev filter
  kTheta = 832,      // 16
  kLeadScale = 848,  // 8: 1 / ||z_j[:n1]||
  kLeadNegE = 856,   // 8: -theta_j (shift of the leading-block solve)
  kPosE0 = 864,      // 8: +E0 per column (right-hand side after deflation)
  kRmmNegTh = 872,   // 8: -theta_j of the RMM-DIIS iterate
  kRmmScale = 880,   // 8: 1 / ||x_j|| (RMM-DIIS normalisation)
  kRitzNegTh = 888,  // 8: -theta_j (tensor-core Ritz residuals)
  kCoefEnd = 896
};


}  // namespace sppc::drv

using namespace sppc;
using namespace sppc::drv;

struct sppc_ctx {
  int64_t n = 0, nnz = 0, n1 = 0;
  bool f64 = false;  // value slots hold IEEE doubles (opts.precision = -1), else double-float pairs
  int k = 0, kp = 0, pmax = 0, mmax = 0;
  std::vector<int64_t> lev;
  sppc_opts opt{};
  std::string err;
  cudaStream_t stream = nullptr;

  // matrix (device)
  SellDev H, H11;
  CsrDev H11c;  // H0_hat as CSR for the persistent MINRES
  CsrDev Hlead; // leading block of the precond 2 solve (H11c unless precond_levels > 1)
  int64_t n_lead = 0;
  std::vector<void*> allocs;
  int64_t h_slices = 0, h11_slices = 0;
  std::vector<int64_t> h_chunk_slice, h11_chunk_slice;  // host copies (SellDev points here)
  std::vector<int64_t> h_slice_ptr, h11_slice_ptr;  // host copies for sppc_get_layout
  std::vector<int32_t> h_slice_rows, h11_slice_rows;
  double h11_lo = 0, h11_hi = 0, h11_norm = 1;

  // blocks (double-float, row-major n x kp)
  float2 *Q = nullptr, *W = nullptr, *Psi = nullptr, *HPsi = nullptr, *T1 = nullptr, *T2 = nullptr;
  // small-space vectors (n1 x kp)
  float2 *psi_hat = nullptr, *vps = nullptr, *b1 = nullptr;
  float2 *zlead = nullptr, *rlead = nullptr;  // leading rows of the Ritz vectors / residuals (precond 2)
  float2 *mv = nullptr, *mvprev = nullptr, *mp = nullptr, *my = nullptr, *mw1 = nullptr, *mw2 = nullptr,
         *mx = nullptr;
  float2 *mref = nullptr, *mres = nullptr, *mdx = nullptr;  // refined FP32 MINRES: b, residual, correction
  // small eigensolve (n1 x 8 blocks, up to 2 per set; 3 filter sets + X + AX + tmp)
  float2* se[12] = {nullptr};
  // the small eigensolve's b lowest eigenpairs (two blocks of n1 x 8; values
  // ascending), kept to deflate the small solves' right-hand sides
  float2* psib[2] = {nullptr, nullptr};
  double* dEb = nullptr;
  int nb_small = 0, b_small = 0;
  // FP64 scalars / small matrices
  double *dE = nullptr, *dHt = nullptr, *dGram = nullptr, *dC1 = nullptr, *dC2 = nullptr, *dR1 = nullptr,
         *dR2 = nullptr, *dTheta = nullptr, *dV = nullptr, *dDots = nullptr, *dS = nullptr;
  float2 *dCoef = nullptr, *dRinv = nullptr, *dRecycle = nullptr, *dY = nullptr, *dCoefBig = nullptr;
  int* dStatus = nullptr;
  unsigned char* Qd = nullptr;  // opts.tensor_gram: FP16 digit tiles of the basis blocks (k_gram_tc.cu)
  uint64_t qd_valid = 0;        // bit a: Qd holds the digits of basis block a as it stands
  unsigned char* Wd = nullptr;  // the same for the blocks of W = H Q, cut per column at 2^(61 - wexp)
  int* wexp = nullptr;          // W blocks' column exponents, 8 per block (device)
  uint64_t wd_valid = 0;
  float2* Zt = nullptr;         // tensor-core Ritz pass: Ritz vectors Q Y and residuals W Y - Z theta
  float2* Dt = nullptr;
  unsigned* dBar = nullptr;
  float2* partials = nullptr;
  int64_t partial_cap = 0;
  double *stageX = nullptr, *stageY = nullptr;  // sppc_spmm_host staging (n x 8 each)
  float2* dDiag = nullptr;                        // diag(H), double-float (Jacobi preconditioner)
  float* val32 = nullptr;                         // FP32 copy of H's SELL values (mixed precision)
  float* X32 = nullptr;                           // FP32 copy of the SpMM input block (mixed precision)
  uint16_t* val16 = nullptr;                      // BF16 off-diagonal values (precision 2)
  float* diag32 = nullptr;                        // FP32 diagonal (precision 2)
  bool f32_products = false;                      // big SpMMs in FP32 (mixed precision, until verified)
  // learned correction proposal
  float2* rowc = nullptr;                         // (level(i), ||H_i,:||_2) per row
  float* net = nullptr;                           // network parameters + mu + sd (device)
  bool net_ready = false;
  float* rhat32 = nullptr;                        // scaled residual entries, n x 8
  float2 *Tprop = nullptr, *Tplain = nullptr;     // proposal and plain preconditioned blocks, n x kp
  float2* Tspare = nullptr;                       // continuation: second n x kp buffer for the appended block
  const float2* t_last = nullptr;                 // the block the last continuation step appended
  int nev = 0;                                    // Ritz pairs kept by the last Rayleigh-Ritz
  // overlap of an SPPC order's Rayleigh-Ritz step with the next order's
  // correction: a second stream and its own reduction scratch
  cudaStream_t stream2 = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  float2* partials2 = nullptr;
  double* dDots2 = nullptr;
  double* pinned = nullptr;                       // host (pinned): theta[16], r2[16] of a deferred step
  // RMM-DIIS (opts.hybrid = 2): per-column DIIS Gram matrices, theta, step
  // lengths, flags and coefficients; rmm_x = the current iterate block
  double *rmm_G = nullptr, *rmm_th = nullptr, *rmm_lam = nullptr, *rmm_g = nullptr;
  int *rmm_frozen = nullptr, *rmm_status = nullptr;
  float2* rmm_coef = nullptr;
  float2* rmm_x = nullptr;
  int64_t chunk_cols_used = 0;                    // SpMM column tile of H's layout (-1: untiled)
  double tuned_ms[8] = {0};                       // autotuner: ms per product of each candidate
  int sigma_used = 1024;                          // sort window of H's layout
  double sigma_ms[4] = {0};                       // sigma autotuner: ms per product of 64, 256, 1024

  // state
  bool started = false, corrected = false, in_refine = false, t_ready = false;
  int p = 0;
  std::vector<double> E0, theta, resid;
  std::vector<OrderRec> rec;
  sppc_stats stats{};
  std::vector<cudaEvent_t> evpool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;  // big-SpMM timing pairs
  int evnext = 0;
};

namespace sppc::drv {

inline sppc_status fail(sppc_ctx* h, sppc_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h)
    h->err = buf;
  else
    g_create_error = buf;
  return st;
}

#define CK(call)                                                                                      \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess)                                                                            \
      return fail(h, e_ == cudaErrorMemoryAllocation ? SPPC_ERR_OOM : SPPC_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                                 \
  } while (0)

#define CKS(expr)                      \
  do {                                 \
    sppc_status s_ = (expr);           \
    if (s_ != SPPC_OK) return s_;      \
  } while (0)

template <class T>
cudaError_t dalloc(sppc_ctx* h, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * (count ? count : 1));
  if (e != cudaSuccess) return e;
  h->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

inline float2* blk(float2* base, int64_t n, int kp, int a) { return base + static_cast<int64_t>(a) * n * kp; }

inline BlockList blocks(float2* base, int64_t n, int kp, int a0, int a1) {
  BlockList L;
  L.n = a1 - a0;
  for (int a = a0; a < a1; ++a) L.p[a - a0] = blk(base, n, kp, a);
  return L;
}

inline BlockList one(const float2* p) {
  BlockList L;
  L.n = 1;
  L.p[0] = p;
  return L;
}

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

struct SellHost {
  int64_t nslices = 0;
  int nchunks = 1;
  int64_t chunk_cols = 0;
  std::vector<int64_t> chunk_slice, slice_ptr;
  std::vector<int32_t> rows, col;
  std::vector<float2> val;
  std::vector<uint8_t> first, last;
};

enum class DenseKind { update, ritz };

// ---- tiny kernels, host SELL builder, timing, big SpMM (drv_host.cu)
__global__ void k_set_consts(float2* c, bool f64);
__global__ void k_set_e0(const double* E0, int k, int kp, float2* c, bool f64);
__global__ void k_rhs_coefs(const double* dE, int p, int k, int kp, float2* c, bool f64);
__global__ void k_inv_norm_coef(const double* d, int k, int kp, float2* out, bool f64);
__global__ void k_neg_coef(const float2* in, int k, int kp, float2* out, bool f64);
__global__ void k_defl_coefs(const double* G, const double* Eb, int b, int k, float2* D, bool f64);
__global__ void k_rmm_theta(const double* d, int k, int kp, float2* negth, double* th);
__global__ void k_diis(const double* g, int nslot, int cur, int nh, double* G, const int* frozen, int k, int kp,
                       float2* coef, int* status);
__global__ void k_rmm_step(const float2* __restrict__ Xb, const float2* __restrict__ Rb,
                           const float2* __restrict__ diag, const double* __restrict__ th,
                           const double* __restrict__ lam, float clamp, int k, int kp, int64_t n, float2* Y);
__global__ void k_neg_dots_to_coef(const double* d, int k, int kp, float2* out, bool f64);
__global__ void k_negmat(const double* C, int count, float2* out, bool f64);
__global__ void k_addmat(const double* A, const double* B, int count, double* out);
__global__ void k_recycle_coefs(const double* Cacc, int p, int kp, const double* R2, const double* R1, float2* dst, bool f64);
__global__ void k_assemble_ht(const double* B, int p, int k, int kp, double* Ht, int ld);
__global__ void k_expand_y(const double* V, int ldv, int p, int k, int kp, const double* th, float2* Y,
                           float2* thdf, bool f64);
__global__ void k_restart_coef(const double* V, int ldv, int p, int k, int kp, int b, float2* out, bool f64);
__global__ void k_subblock(const float2* src, int lds, int na, int ob, float2* out);
__global__ void k_neg_theta(const double* th, int b, float2* out, bool f64);
__global__ void k_vmat_df(const double* V, int m, int nev, int ldv, float2* out, bool f64);
void split_df(double x, float2& out);
void put_slot(double x, float2& out, bool f64);
float round_bf16(float f);
void build_sell(int64_t nrows, const int64_t* rp, const int32_t* ci, const double* va, int64_t ncols,
                const std::vector<int64_t>& seg, int64_t sigma, int64_t chunk_cols, bool f64, SellHost& S);
sppc_status upload_sell(sppc_ctx* h, SellHost& S, SellDev& D, int64_t nrows, std::vector<int64_t>& chunk_store);
cudaError_t spmm11(const sppc_ctx* h, int kp, const float2* X, float2* Y, const Epi& e, cudaStream_t s);
// spmm11 on nb blocks (Y[a] = epilogue(H0_hat X[a]), Z[a] as the epilogue's Z when
// Z is given); two CSR blocks go in one launch.
cudaError_t spmm11_set(const sppc_ctx* h, int kp, const float2* const* X, float2* const* Y, const float2* const* Z,
                       int nb, Epi e, cudaStream_t s);
sppc_status upload_csr11(sppc_ctx* h, int64_t n1, const int64_t* rp, const int32_t* ci, const double* va,
                         CsrDev& out);
cudaEvent_t next_event(sppc_ctx* h);
sppc_status collect_timing(sppc_ctx* h);
sppc_status big_spmm(sppc_ctx* h, const float2* X, float2* Y, int kp);

// ---- solver steps (drv_solver.cu)
sppc_status gram_set(sppc_ctx* h, float2** X, float2** Z, int nb, double* G16);
sppc_status rotate_set(sppc_ctx* h, float2** X, float2** Y, int nb, const float2* M16);
sppc_status ortho_set(sppc_ctx* h, float2** X, float2** Tmp, int nb, int b);
sppc_status small_eigensolve(sppc_ctx* h);
sppc_status minres_refined(sppc_ctx* h, int maxit, std::vector<int32_t>& iters);
sppc_status minres(sppc_ctx* h, std::vector<int32_t>& iters);
cudaError_t ensure_qdigits(sppc_ctx* h, int nq, cudaStream_t s);
cudaError_t qgram(sppc_ctx* h, int nq, const float2* B, double* out, cudaStream_t s);
cudaError_t qupdate(sppc_ctx* h, int nq, float2* Y, const float2* X, const float2* alpha, const float2* coef,
                    cudaStream_t s);
cudaError_t ensure_wdigits(sppc_ctx* h, int nq, cudaStream_t s);
bool tensor_dense(const sppc_ctx* h, int nq, DenseKind kind);
cudaError_t wupdate(sppc_ctx* h, int nq, float2* Y, const float2* X, const float2* alpha, const float2* coef,
                    cudaStream_t s);
__global__ void k_neg_slots(const float2* in, float2* out, int count, bool f64);
cudaError_t qritz(sppc_ctx* h, int np1, double* Zout, int64_t ldz, int ncols, float2* Tout, const float2* diag,
                  float clamp, float2* Zlead, float2* Rlead, int64_t nlead, cudaStream_t s);
sppc_status rr_core(sppc_ctx* h, int p, bool want_z, double* Z, int64_t ldz, float2* T = nullptr,
                    const float2* diag = nullptr, bool defer = false);
sppc_status rr_finish(sppc_ctx* h, cudaStream_t s);
sppc_status orth_append(sppc_ctx* h, const float2* src, int p, double* dd, bool cond);
sppc_status restart(sppc_ctx* h, bool fresh_products = false);
sppc_status lead_correction(sppc_ctx* h, float2* T);
const float2* t_diag(const sppc_ctx* h);
sppc_status ensure_proposal_buffers(sppc_ctx* h);
sppc_status proposal_block(sppc_ctx* h, const float2* R);
sppc_status refine_step(sppc_ctx* h);
sppc_status rmm_run(sppc_ctx* h, double tol);
bool all_converged(const sppc_ctx* h, double tol);

// ---- layout tuning (api_create.cu)
cudaError_t time_layout(int64_t n, const int64_t* d_rp, const int32_t* d_ci, const double* d_va,
                        const std::vector<int64_t>& seg, bool f64, int64_t c, int sigma, const float2* X, float2* Y,
                        cudaEvent_t a, cudaEvent_t b, cudaStream_t s, double* ms_out);
cudaError_t tune_sigma(int64_t n, const int64_t* d_rp, const int32_t* d_ci, const double* d_va,
                       const std::vector<int64_t>& seg, bool f64, int64_t c, cudaStream_t s, int* best,
                       double* ms_out);
cudaError_t tune_chunk_cols(int64_t n, const int64_t* d_rp, const int32_t* d_ci, const double* d_va,
                            const std::vector<int64_t>& seg, bool f64, cudaStream_t s, int64_t* best, double* ms_out);

}  // namespace sppc::drv
