// C ABI and host driver of the SPPC eigensolver (Algorithm 2 of the paper).
//
// The driver owns all device memory and sequences the kernels of k_spmm.cu,
// k_dense.cu and k_small.cu on the caller's stream.  Host work is limited to
// argument checks, building the SELL-32 layout once in sppc_create, scalar
// bookkeeping and one small device->host copy per correction order (the
// convergence test of Alg. 2) or per few MINRES iterations.
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

using namespace sppc;

namespace {

// Named NVTX ranges around the solver phases (no cost unless a tool such as
// ncu or nsys is attached; profilers can filter kernels by phase).
struct PhaseRange {
  explicit PhaseRange(const char* name) { nvtxRangePushA(name); }
  ~PhaseRange() { nvtxRangePop(); }
  PhaseRange(const PhaseRange&) = delete;
  PhaseRange& operator=(const PhaseRange&) = delete;
};

thread_local std::string g_create_error;

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

}  // namespace

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

// ------------------------------------------------------------------ helpers
namespace {

sppc_status fail(sppc_ctx* h, sppc_status st, const char* fmt, ...) {
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

BlockList blocks(float2* base, int64_t n, int kp, int a0, int a1) {
  BlockList L;
  L.n = a1 - a0;
  for (int a = a0; a < a1; ++a) L.p[a - a0] = blk(base, n, kp, a);
  return L;
}

BlockList one(const float2* p) {
  BlockList L;
  L.n = 1;
  L.p[0] = p;
  return L;
}

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

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
__global__ void k_vmat_df(const double* V, int m, int nev, int ldv, float2* out, bool f64) {
  const int t = threadIdx.x;
  for (int e = t; e < 256; e += blockDim.x) {
    const int i = e / 16, j = e % 16;
    out[e] = (i < m && j < nev) ? slot_put(V[i * ldv + j], f64) : make_float2(0.f, 0.f);
  }
}

// ------------------------------------------------------------ SELL builder
struct SellHost {
  int64_t nslices = 0;
  int nchunks = 1;
  int64_t chunk_cols = 0;
  std::vector<int64_t> chunk_slice, slice_ptr;
  std::vector<int32_t> rows, col;
  std::vector<float2> val;
  std::vector<uint8_t> first, last;
};

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
static cudaError_t spmm11(const sppc_ctx* h, int kp, const float2* X, float2* Y, const Epi& e, cudaStream_t s) {
  if (h->H11c.rowptr && h->H11c.nrows <= kCsrRowsMax) return spmm_csr(h->H11c, kp, X, Y, e, s);
  return spmm(h->H11, kp, X, Y, e, s);
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

}  // namespace

// The multi-block helpers below need the full context type.
namespace {

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
  // shifted CholeskyQR, then CholeskyQR twice (result back in X)
  for (int pass = 0; pass < 3; ++pass) {
    CKS(gram_set(h, X, X, nb, h->dS));
    const double shift = (pass == 0) ? 1e-12 : 0.0;
    CK(chol_rinv(h->dS, 16, b, 16, shift, h->dR1, h->dRinv, h->dStatus, h->f64, h->stream));
    int st = 0;
    CK(cudaMemcpyAsync(&st, h->dStatus, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (st != 0) return fail(h, SPPC_ERR_BREAKDOWN, "small eigensolve: Cholesky breakdown at column %d", st - 1);
    CKS(rotate_set(h, X, Tmp, nb, h->dRinv));
    for (int a = 0; a < nb; ++a) std::swap(X[a], Tmp[a]);
  }
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
    for (int a = 0; a < nb; ++a) CK(spmm11(h, 8, X[a], AX[a], Epi{}, s));
    h->stats.spmv_h11 += 8 * nb;
    CKS(gram_set(h, X, AX, nb, h->dS));
    CK(syev_lowest(h->dS, 16, b, b, h->dTheta, h->dV, b, h->f64, s));
    k_vmat_df<<<1, 256, 0, s>>>(h->dV, b, b, b, h->dRinv, h->f64); count_launch();
    CK(cudaGetLastError());
    CKS(rotate_set(h, X, Tmp, nb, h->dRinv));
    for (int a = 0; a < nb; ++a) std::swap(X[a], Tmp[a]);
    CKS(rotate_set(h, AX, Tmp, nb, h->dRinv));
    for (int a = 0; a < nb; ++a) std::swap(AX[a], Tmp[a]);
    CK(cudaMemcpyAsync(th.data(), h->dTheta, sizeof(double) * b, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // residuals of the k lowest: D = AX - X theta (block 0 holds columns 0..7)
    std::vector<float2> thdf(8);
    for (int c = 0; c < 8; ++c) put_slot((c < b) ? -th[c] : 0.0, thdf[c], h->f64);
    CK(cudaMemcpyAsync(h->dCoef + kTheta, thdf.data(), sizeof(float2) * 8, cudaMemcpyHostToDevice, s));
    CK(combine_diag(Tmp[0], AX[0], h->dCoef + kOnes, one(X[0]), h->dCoef + kTheta, 8, 0, n1, h->f64, s));
    const float2* A1[1] = {Tmp[0]};
    const float2* B1[1] = {Tmp[0]};
    CK(coldots(A1, B1, 1, 8, 0, n1, h->dDots, h->partials, h->partial_cap, h->f64, s));
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
      for (int a = 0; a < nb; ++a) CK(spmm11(h, 8, X[a], Y1[a], e1, s));
      CKS(put3(2.0 / e, -2.0 * c / e, -1.0));
      float2* setA[2] = {X[0], X[1]};
      float2* setB[2] = {Y1[0], Y1[1]};
      float2* setC[2] = {Y0[0], Y0[1]};
      for (int dgi = 2; dgi <= deg; ++dgi) {
        Epi e2;
        e2.alpha = h->dCoef + kCheb;
        e2.beta = h->dCoef + kCheb + 16;
        e2.gamma = h->dCoef + kCheb + 32;
        for (int a = 0; a < nb; ++a) {
          e2.Z = setA[a];
          CK(spmm11(h, 8, setB[a], setC[a], e2, s));
        }
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
enum class DenseKind { update, ritz };
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
sppc_status rr_core(sppc_ctx* h, int p, bool want_z, double* Z, int64_t ldz, float2* T = nullptr,
                    const float2* diag = nullptr, bool defer = false) {
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
sppc_status restart(sppc_ctx* h, bool fresh_products = false) {
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

}  // namespace

namespace {

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

}  // namespace

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

// =================================================================== C ABI
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
