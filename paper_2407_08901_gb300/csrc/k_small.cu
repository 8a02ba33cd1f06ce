// Small dense kernels, one CTA each: the k x k Cholesky factor and its inverse
// for CholeskyQR (Eq. QR, FP64), and the symmetric eigensolve of the projected
// matrix Q^T H Q (Eqs. tilde_H, proj; at most k(p_max+1) <= 144 rows).
//
// FP64 runs at ~1/70 of FP32 on this GPU, so the eigensolve does its O(m^3)
// parts (Householder tridiagonalisation, back-transformation) in the slot
// format (double-float on the default path, FP64 on the native FP64 path) and
// brackets the eigenvalues in FP32 first; FP64 is kept for the O(m) per vector
// tridiagonal work (inverse iteration, Rayleigh quotients) and for crowded
// eigenvalues.
#include <math.h>

#include "sppc_internal.h"
#include "val.cuh"

namespace sppc {

namespace {

constexpr int kMaxM = 144;
constexpr int kMaxNev = 16;

__global__ void k_chol_rinv(const double* __restrict__ G, int ldg, int kk, int kp, double shift_rel,
                            double* __restrict__ R, float2* __restrict__ Rinv_df, int* status, bool f64) {
  __shared__ double A[16][17];
  __shared__ double Ri[16][17];
  __shared__ int bad;
  const int t = threadIdx.x;
  if (t == 0) bad = 0;
  for (int e = t; e < 16 * 16; e += blockDim.x) {
    const int i = e / 16, j = e % 16;
    A[i][j] = (i < kk && j < kk) ? 0.5 * (G[i * ldg + j] + G[j * ldg + i]) : 0.0;
    Ri[i][j] = 0.0;
  }
  __syncthreads();
  if (shift_rel > 0.0) {
    if (t == 0) {
      double mx = 0.0;
      for (int i = 0; i < kk; ++i) mx = fmax(mx, fabs(A[i][i]));
      for (int i = 0; i < kk; ++i) A[i][i] += shift_rel * mx;
    }
    __syncthreads();
  }
  // right-looking Cholesky A = R^T R, R upper; thread i owns column i
  for (int j = 0; j < kk; ++j) {
    if (t == 0) {
      const double d = A[j][j];
      if (!(d > 0.0)) {
        if (!bad) bad = j + 1;
        A[j][j] = 1.0;
      } else {
        A[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    if (t > j && t < kk) A[j][t] /= A[j][j];
    __syncthreads();
    if (t > j && t < kk) {
      for (int i = j + 1; i <= t; ++i) A[i][t] -= A[j][i] * A[j][t];
    }
    __syncthreads();
  }
  // inverse of the upper triangular R: thread j solves R x = e_j
  if (t < kk) {
    for (int i = t; i >= 0; --i) {
      double s = (i == t) ? 1.0 : 0.0;
      for (int l = i + 1; l <= t; ++l) s -= A[i][l] * Ri[l][t];
      Ri[i][t] = s / A[i][i];
    }
  }
  __syncthreads();
  for (int e = t; e < kp * kp; e += blockDim.x) {
    const int i = e / kp, j = e % kp;
    const bool in = (i < kk && j < kk);
    R[i * kp + j] = (in && j >= i) ? A[i][j] : 0.0;
    Rinv_df[e] = in ? slot_put(Ri[i][j], f64) : make_float2(0.f, 0.f);
  }
  if (t == 0) status[0] = bad;
}

// Sturm count: number of eigenvalues of the tridiagonal (d, e^2) below x.
template <typename T>
__device__ int sturm_count(const T* d, const T* e2, int m, T x, T pivmin) {
  int cnt = 0;
  T q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = 1; i < m; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// Multisection for eigenvalue index w with one warp: 32 Sturm counts per round
// shrink [lo, hi] by a factor of 33.  Stops when hi - lo <= rel * max(|lo|,|hi|) + abs.
template <typename T>
__device__ void multisect(const T* d, const T* e2, int m, int w, T pivmin, T rel, T abs_tol, int max_rounds,
                          double& lo_io, double& hi_io) {
  const int lane = threadIdx.x & 31;
  T lo = static_cast<T>(lo_io), hi = static_cast<T>(hi_io);
  for (int it = 0; it < max_rounds; ++it) {
    if (hi - lo <= rel * fmax(fabs(lo), fabs(hi)) + abs_tol) break;
    const T x = lo + (hi - lo) * static_cast<T>(lane + 1) / static_cast<T>(33);
    const int c = sturm_count<T>(d, e2, m, x, pivmin);
    const unsigned ball = __ballot_sync(0xffffffffu, c > w);
    T nlo = lo, nhi = hi;
    if (ball) {
      const int f = __ffs(ball) - 1;
      nhi = lo + (hi - lo) * static_cast<T>(f + 1) / static_cast<T>(33);
      if (f > 0) nlo = lo + (hi - lo) * static_cast<T>(f) / static_cast<T>(33);
    } else {
      nlo = lo + (hi - lo) * static_cast<T>(32) / static_cast<T>(33);
    }
    lo = __shfl_sync(0xffffffffu, nlo, 0);
    hi = __shfl_sync(0xffffffffu, nhi, 0);
  }
  lo_io = static_cast<double>(lo);
  hi_io = static_cast<double>(hi);
}

// Narrow [lo, hi] for index w by 4-section in FP64: three Sturm counts per round
// (lanes 0-2 of the warp; FP64 throughput, not latency, is the scarce resource).
// Stops when hi - lo <= rel * max(|lo|,|hi|) + abs_tol.
__device__ void quadsect64(const double* d, const double* e2, int m, int w, double pivmin, double rel,
                           double abs_tol, int max_rounds, double& lo_io, double& hi_io) {
  const int lane = threadIdx.x & 31;
  double lo = lo_io, hi = hi_io;
  for (int it = 0; it < max_rounds; ++it) {
    if (hi - lo <= rel * fmax(fabs(lo), fabs(hi)) + abs_tol) break;
    const double h = hi - lo;
    const int c = (lane < 3) ? sturm_count<double>(d, e2, m, lo + h * 0.25 * (double)(lane + 1), pivmin) : m + 1;
    const unsigned ball = __ballot_sync(0xffffffffu, c > w) & 0x7u;
    const int f = ball ? __ffs(ball) - 1 : 3;  // first quarter point above index w
    const double nlo = (f > 0) ? lo + h * 0.25 * (double)f : lo;
    const double nhi = (f < 3) ? lo + h * 0.25 * (double)(f + 1) : hi;
    lo = nlo;
    hi = nhi;
  }
  lo_io = lo;
  hi_io = hi;
}

// sqrt of a double-float: fp32 root s, exact square s*s (TwoProd), one
// correction step (a - s^2) / (2 s).
__device__ __forceinline__ float2 df_sqrt(float2 a) {
  if (!(a.x > 0.f)) return make_float2(0.f, 0.f);
  const float s = __fsqrt_rn(a.x);
  const float p = __fmul_rn(s, s);
  const float2 sp = make_float2(p, __fmaf_rn(s, s, -p));
  const float2 r = df_sub(a, sp);
  return fast_two_sum(s, __fdiv_rn(r.x, __fmul_rn(2.f, s)));
}

template <bool F64>
__device__ __forceinline__ float2 slot_sqrt(float2 a) {
  if constexpr (F64) {
    const double x = slot_d(a);
    return d_slot(x > 0.0 ? __dsqrt_rn(x) : 0.0);
  } else {
    return df_sqrt(a);
  }
}

// Block-wide sum in the slot format (all threads get the result).
template <bool F64>
__device__ float2 block_sum(float2 v, float2* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum<F64>(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 t = red[0];
    for (int w2 = 1; w2 < nw; ++w2) t = Ar<F64>::add(t, red[w2]);
    red[32] = t;
  }
  __syncthreads();
  const float2 r = red[32];
  __syncthreads();
  return r;
}

// Solve (T - sigma I) y = y in place for the tridiagonal (d, e), FP64, with
// partial pivoting; returns false on an exactly zero pivot set to eps.
template <typename T>
__device__ void tri_shift_solve(const T* d, const T* e, int m, T sigma, T eps_piv, T* y, T* du, T* u1, T* u2, T* lm,
                                unsigned char* piv) {
  T a0 = d[0] - sigma, b0 = (m > 1) ? e[0] : T(0);
  for (int i = 0; i + 1 < m; ++i) {
    const T c = e[i];
    const T a1 = d[i + 1] - sigma;
    const T b1 = (i + 2 < m) ? e[i + 1] : T(0);
    if (fabs(c) > fabs(a0)) {
      piv[i] = 1;
      du[i] = c;
      u1[i] = a1;
      u2[i] = b1;
      const T l = a0 / c;
      lm[i] = l;
      a0 = b0 - l * a1;
      b0 = -l * b1;
    } else {
      piv[i] = 0;
      if (a0 == T(0)) a0 = eps_piv;
      du[i] = a0;
      u1[i] = b0;
      u2[i] = T(0);
      const T l = c / a0;
      lm[i] = l;
      a0 = a1 - l * b0;
      b0 = b1;
    }
  }
  du[m - 1] = (a0 == T(0)) ? eps_piv : a0;
  for (int i = 0; i + 1 < m; ++i) {
    if (piv[i]) {
      const T tmp = y[i];
      y[i] = y[i + 1];
      y[i + 1] = tmp - lm[i] * y[i];
    } else {
      y[i + 1] -= lm[i] * y[i];
    }
  }
  for (int i = m - 1; i >= 0; --i) {
    T sv = y[i];
    if (i + 1 < m) sv -= u1[i] * y[i + 1];
    if (i + 2 < m) sv -= u2[i] * y[i + 2];
    T di = du[i];
    if (fabs(di) < eps_piv) di = (di < 0 ? -eps_piv : eps_piv);
    y[i] = sv / di;
  }
}

template <typename T>
__device__ T rayleigh_tri(const T* d, const T* e, int m, const T* y) {
  T num = 0, den = 0;
  for (int i = 0; i < m; ++i) {
    T ty = d[i] * y[i];
    if (i > 0) ty += e[i - 1] * y[i - 1];
    if (i + 1 < m) ty += e[i] * y[i + 1];
    num += y[i] * ty;
    den += y[i] * y[i];
  }
  return num / den;
}

// Symmetric eigensolve of the projected matrix, nev lowest pairs.
//  1. Householder tridiagonalisation (Golub and Van Loan, Alg. 8.3.1) in the
//     slot format (double-float, or FP64 for the native FP64 path), matrix in
//     shared memory with leading dimension m+1.
//  2. Eigenvalue brackets by Sturm-count multisection in FP32 to ~1e-5; indices
//     whose brackets crowd a neighbour are narrowed further in FP64.
//  3. Eigenvectors of the tridiagonal matrix by inverse iteration, one thread
//     per vector: three FP32 steps, then FP64 steps (the FP64 pipe is ~1/64 of
//     FP32 here, so FP64 is kept to the last steps).  Isolated eigenvalues: FP32
//     Rayleigh-quotient shifts, one FP64 step at the FP64 Rayleigh quotient.
//     Crowded groups: shifts at the bracket midpoints (FP64 brackets ~1e-13
//     wide), two FP64 steps, then modified Gram-Schmidt in the group.  The
//     eigenvalue is the final Rayleigh quotient.
//  4. Back-transformation through the stored reflectors in the slot format.
template <bool F64>
__global__ void __launch_bounds__(512) k_syev_lowest(const double* __restrict__ S, int lds, int m, int nev,
                                                     double* __restrict__ theta, double* __restrict__ V, int ldv) {
  using AR = Ar<F64>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ld = m + 1;
  float2* A = reinterpret_cast<float2*>(smraw);  // m x ld, reflectors below the diagonal
  float2* vec = A + m * ld;                        // m
  float2* pw = vec + m;                            // m
  float2* tau = pw + m;                            // m
  float2* red = tau + m;                           // 33
  float2* Yd = red + 40;                           // nev x m (double-float eigenvectors)
  double* d = reinterpret_cast<double*>(Yd + kMaxNev * m);  // m
  double* e = d + m;                                         // m
  double* e2 = e + m;                                        // m
  double* Y = e2 + m;                                        // nev x m (FP64 eigenvectors of T)
  double* lo = Y + kMaxNev * m;                              // nev
  double* hi = lo + kMaxNev;                                 // nev
  double* ev = hi + kMaxNev;                                 // nev
  float* d32 = reinterpret_cast<float*>(ev + kMaxNev);       // m
  float* e232 = d32 + m;                                     // m
  int* crowd = reinterpret_cast<int*>(e232 + m);             // nev
  const int t = threadIdx.x, nt = blockDim.x;
  const int lane = t & 31, warp = t >> 5, nwarp = nt >> 5;
  for (int x = t; x < m * m; x += nt) {
    const int i = x / m, j = x % m;
    A[i * ld + j] = AR::from_d(0.5 * (S[i * lds + j] + S[j * lds + i]));
  }
  __syncthreads();
  // ---- 1. Householder tridiagonalisation (slot format)
  for (int j = 0; j + 2 < m; ++j) {
    const int len = m - j - 1;
    typename AR::Acc sa;
    AR::zero(sa);
    for (int i = t; i < len; i += nt) {
      const float2 xv = A[(j + 1 + i) * ld + j];
      AR::mac(sa, xv, xv);
    }
    const float2 s2 = block_sum<F64>(AR::get(sa), red);
    if (t == 0) {
      const float2 x0 = A[(j + 1) * ld + j];
      const float2 nrm = slot_sqrt<F64>(s2);
      if (AR::lead(nrm) == 0.0) {
        tau[j] = make_float2(0.f, 0.f);
        e[j] = 0.0;
        red[34] = make_float2(0.f, 0.f);
      } else {
        const float2 alpha = (AR::lead(x0) >= 0.0) ? AR::neg(nrm) : nrm;
        const float2 v0 = AR::sub(x0, alpha);
        const float2 vtv = AR::add(AR::sub(s2, AR::mul(x0, x0)), AR::mul(v0, v0));
        tau[j] = AR::div(AR::from_d(2.0), vtv);
        e[j] = AR::to_d(alpha);
        red[34] = v0;
      }
    }
    __syncthreads();
    const float2 tj = tau[j];
    for (int i = t; i < len; i += nt) vec[i] = (i == 0) ? red[34] : A[(j + 1 + i) * ld + j];
    __syncthreads();
    if (AR::lead(tj) != 0.0) {
      // p = tau A v: four threads per row (entries sub, sub+4, ...), combined by shuffles
      for (int i0 = 0; i0 < len; i0 += nt / 4) {
        const int i = i0 + (t >> 2), sub = t & 3;
        typename AR::Acc pa;
        AR::zero(pa);
        if (i < len) {
          const float2* row = A + (j + 1 + i) * ld + (j + 1);
          int c = 0;
          for (int l = sub; l < len; l += 4) {
            AR::mac(pa, row[l], vec[l]);
            if (((++c) & 15) == 0) AR::norm(pa);
          }
        }
        float2 pr = AR::get(pa);
        pr = AR::add(pr, shfl_xor_df(pr, 1));
        pr = AR::add(pr, shfl_xor_df(pr, 2));
        if (i < len && sub == 0) pw[i] = AR::mul(tj, pr);
      }
      __syncthreads();
      typename AR::Acc ka;
      AR::zero(ka);
      for (int i = t; i < len; i += nt) AR::mac(ka, pw[i], vec[i]);
      const float2 pv = block_sum<F64>(AR::get(ka), red);
      const float2 K = AR::mul(AR::mul(AR::from_d(0.5), tj), pv);
      for (int i = t; i < len; i += nt) pw[i] = AR::sub(pw[i], AR::mul(K, vec[i]));  // w
      __syncthreads();
      // A -= v w^T + w v^T: a warp per row, lanes along the row
      for (int i = warp; i < len; i += nwarp) {
        const float2 vi = vec[i], wi = pw[i];
        float2* arow = A + (j + 1 + i) * ld + (j + 1);
        for (int l = lane; l < len; l += 32)
          arow[l] = AR::sub(arow[l], AR::add(AR::mul(vi, pw[l]), AR::mul(wi, vec[l])));
      }
    }
    __syncthreads();
    for (int i = t; i < len; i += nt) A[(j + 1 + i) * ld + j] = vec[i];
    if (t == 0) d[j] = AR::to_d(A[j * ld + j]);
    __syncthreads();
  }
  if (t == 0) {
    if (m >= 2) {
      d[m - 2] = AR::to_d(A[(m - 2) * ld + (m - 2)]);
      d[m - 1] = AR::to_d(A[(m - 1) * ld + (m - 1)]);
      e[m - 2] = AR::to_d(A[(m - 1) * ld + (m - 2)]);
      tau[m - 2] = make_float2(0.f, 0.f);
    } else {
      d[0] = AR::to_d(A[0]);
    }
    if (m >= 1) tau[m - 1] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int i = t; i < m; i += nt) {
    e2[i] = (i + 1 < m) ? e[i] * e[i] : 0.0;
    d32[i] = static_cast<float>(d[i]);
    e232[i] = static_cast<float>(e2[i]);
  }
  __shared__ double gl, gu, tnorm;
  if (t == 0) {
    double l0 = 1e300, h0 = -1e300, mx = 0.0;
    for (int i = 0; i < m; ++i) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
      l0 = fmin(l0, d[i] - r);
      h0 = fmax(h0, d[i] + r);
      mx = fmax(mx, fabs(d[i]) + r);
    }
    tnorm = fmax(mx, 1e-300);
    const double pad = 1e-6 * tnorm + 1e-300;
    gl = l0 - pad;
    gu = h0 + pad;
  }
  __syncthreads();
  // ---- 2. brackets: FP32 multisection, then FP64 for crowded indices
  for (int w = warp; w < nev; w += nwarp) {
    double l0 = gl, h0 = gu;
    multisect<float>(d32, e232, m, w, 1e-30f, 2e-6f, static_cast<float>(1e-7 * tnorm), 12, l0, h0);
    if (lane == 0) {
      lo[w] = l0;
      hi[w] = h0;
    }
  }
  __syncthreads();
  if (t < nev) {
    // crowded: the bracket is not clearly separated from a neighbouring index's
    const double sep = 1e-4 * tnorm;
    int c = 0;
    if (t > 0 && lo[t] - hi[t - 1] < sep) c = 1;
    if (t + 1 < nev && lo[t + 1] - hi[t] < sep) c = 1;
    if (hi[t] - lo[t] > 1e-4 * tnorm) c = 1;
    crowd[t] = c;
  }
  __syncthreads();
  for (int w = warp; w < nev; w += nwarp) {
    if (!crowd[w]) continue;
    // start from the FP32 bracket widened well past the FP32 Sturm error
    // (about m * 2^-24 * ||T||); if the FP64 counts disagree, from the whole interval
    double l0 = lo[w] - 4e-5 * tnorm, h0 = hi[w] + 4e-5 * tnorm;
    int c = 0;
    if (lane == 0) c = sturm_count<double>(d, e2, m, l0, 1e-280);
    if (lane == 1) c = sturm_count<double>(d, e2, m, h0, 1e-280);
    const int cl = __shfl_sync(0xffffffffu, c, 0), ch = __shfl_sync(0xffffffffu, c, 1);
    if (!(cl <= w && ch > w)) {
      l0 = gl;
      h0 = gu;
    }
    quadsect64(d, e2, m, w, 1e-280, 1e-13, 1e-15 * tnorm, 80, l0, h0);
    if (lane == 0) {
      lo[w] = l0;
      hi[w] = h0;
    }
  }
  __syncthreads();
  // ---- 3. inverse iteration on T, thread c for vector c
  if (t < nev) {
    double* y = Y + t * m;
    double du[kMaxM], u1[kMaxM], u2[kMaxM], lm[kMaxM];
    unsigned char piv[kMaxM];
    const double eps_piv = 2.2e-16 * tnorm;
    // three FP32 steps (isolated: Rayleigh-quotient shifts; crowded: the bracket
    // midpoint), then FP64 steps: one at the FP64 Rayleigh quotient (isolated) or
    // two at the FP64 bracket midpoint, ~1e-13 wide (crowded; orthogonalised in
    // the group below).  The FP64 pipe is ~1/64 of FP32 here.
    float yf[kMaxM], duf[kMaxM], u1f[kMaxM], u2f[kMaxM], lmf[kMaxM], ef[kMaxM];
    for (int i = 0; i < m; ++i) {
      yf[i] = 1.f + 0.1f * (float)((i * 7 + t * 3) % 11);
      ef[i] = (i + 1 < m) ? static_cast<float>(e[i]) : 0.f;
    }
    const float epsf = static_cast<float>(1.2e-7 * tnorm);
    float sf = static_cast<float>(0.5 * (lo[t] + hi[t]));
    for (int it = 0; it < 3; ++it) {
      tri_shift_solve<float>(d32, ef, m, sf, epsf, yf, duf, u1f, u2f, lmf, piv);
      float nrm = 0.f;
      for (int i = 0; i < m; ++i) nrm = fmaxf(nrm, fabsf(yf[i]));
      const float inv = 1.f / nrm;
      for (int i = 0; i < m; ++i) yf[i] *= inv;
      if (!crowd[t] && it >= 1) {
        const float rq = rayleigh_tri<float>(d32, ef, m, yf);
        if (rq >= lo[t] - 1e-6 * tnorm && rq <= hi[t] + 1e-6 * tnorm) sf = rq;
      }
    }
    for (int i = 0; i < m; ++i) y[i] = static_cast<double>(yf[i]);
    double sigma = 0.5 * (lo[t] + hi[t]);
    if (!crowd[t]) {
      const double rq = rayleigh_tri<double>(d, e, m, y);
      if (rq >= lo[t] - 1e-6 * tnorm && rq <= hi[t] + 1e-6 * tnorm) sigma = rq;
    }
    const int steps64 = crowd[t] ? 2 : 1;
    for (int it = 0; it < steps64; ++it) {
      tri_shift_solve<double>(d, e, m, sigma, eps_piv, y, du, u1, u2, lm, piv);
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) nrm = fmax(nrm, fabs(y[i]));
      const double inv = 1.0 / nrm;
      for (int i = 0; i < m; ++i) y[i] *= inv;
    }
  }
  __syncthreads();
  // crowded groups: modified Gram-Schmidt in index order (thread 0, rare)
  if (t == 0) {
    for (int c = 0; c < nev; ++c) {
      double* yc = Y + c * m;
      if (crowd[c]) {
        for (int b = 0; b < c; ++b) {
          if (!crowd[b]) continue;
          const double* yb = Y + b * m;
          double dot = 0.0, nb = 0.0;
          for (int i = 0; i < m; ++i) {
            dot += yb[i] * yc[i];
            nb += yb[i] * yb[i];
          }
          for (int i = 0; i < m; ++i) yc[i] -= (dot / nb) * yb[i];
        }
      }
    }
  }
  __syncthreads();
  if (t < nev) {
    double* y = Y + t * m;
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += y[i] * y[i];
    nrm = 1.0 / sqrt(nrm);
    for (int i = 0; i < m; ++i) y[i] *= nrm;
    ev[t] = rayleigh_tri<double>(d, e, m, y);
    for (int i = 0; i < m; ++i) Yd[t * m + i] = AR::from_d(y[i]);
  }
  __syncthreads();
  // ---- 4. back-transform y <- H_0 H_1 ... H_{m-3} y (slot format), warp per vector
  for (int j = m - 3; j >= 0; --j) {
    const float2 tj = tau[j];
    if (AR::lead(tj) == 0.0) continue;
    const int len = m - j - 1;
    for (int c = warp; c < nev; c += nwarp) {
      typename AR::Acc pa;
      AR::zero(pa);
      for (int i = lane; i < len; i += 32) AR::mac(pa, A[(j + 1 + i) * ld + j], Yd[c * m + j + 1 + i]);
      const float2 sdot = AR::mul(tj, warp_sum<F64>(AR::get(pa)));
      for (int i = lane; i < len; i += 32)
        Yd[c * m + j + 1 + i] = AR::sub(Yd[c * m + j + 1 + i], AR::mul(sdot, A[(j + 1 + i) * ld + j]));
    }
    __syncthreads();
  }
  for (int x = t; x < m * nev; x += nt) {
    const int i = x / nev, c = x % nev;
    V[i * ldv + c] = AR::to_d(Yd[c * m + i]);
  }
  if (t < nev) theta[t] = ev[t];
}

__global__ void k_to_df(const double* __restrict__ x, float2* __restrict__ y, int count, double scale, bool f64) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) y[i] = slot_put(scale * x[i], f64);
}

}  // namespace

cudaError_t chol_rinv(const double* G, int ldg, int kk, int kp, double shift_rel, double* R, float2* Rinv_df,
                      int* status, bool f64, cudaStream_t s) {
  if (kk < 1 || kk > 16 || kp > 16) return cudaErrorInvalidValue;
  k_chol_rinv<<<1, 32, 0, s>>>(G, ldg, kk, kp, shift_rel, R, Rinv_df, status, f64); count_launch();
  return cudaGetLastError();
}

static size_t syev_smem(int m) {
  const size_t f2 = (size_t)m * (m + 1) + 3 * (size_t)m + 40 + (size_t)kMaxNev * m;   // float2 entries
  const size_t db = 3 * (size_t)m + (size_t)kMaxNev * m + 3 * kMaxNev;               // doubles
  const size_t fl = 2 * (size_t)m;                                                   // floats
  return f2 * sizeof(float2) + db * sizeof(double) + fl * sizeof(float) + kMaxNev * sizeof(int) + 256;
}

cudaError_t syev_lowest(const double* S, int lds, int m, int nev, double* theta, double* V, int ldv, bool f64,
                        cudaStream_t s) {
  if (m < 1 || m > kMaxM || nev < 1 || nev > kMaxNev || nev > m) return cudaErrorInvalidValue;
  const size_t smem = syev_smem(m);
  static const cudaError_t attr = [] {
    cudaError_t e = cudaFuncSetAttribute(k_syev_lowest<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)syev_smem(kMaxM));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_syev_lowest<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)syev_smem(kMaxM));
    return e;
  }();
  if (attr != cudaSuccess) return attr;
  if (f64)
    k_syev_lowest<true><<<1, 512, smem, s>>>(S, lds, m, nev, theta, V, ldv);
  else
    k_syev_lowest<false><<<1, 512, smem, s>>>(S, lds, m, nev, theta, V, ldv);
  count_launch();
  return cudaGetLastError();
}

cudaError_t to_df(const double* x, float2* y, int count, double scale, bool f64, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_to_df<<<(count + 255) / 256, 256, 0, s>>>(x, y, count, scale, f64); count_launch();
  return cudaGetLastError();
}

}  // namespace sppc
