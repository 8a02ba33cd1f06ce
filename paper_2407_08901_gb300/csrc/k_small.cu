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
#include "fp64_fast.cuh"
#include "val.cuh"

namespace sppc {

namespace {

constexpr int kMaxM = 144;
constexpr int kMaxNev = 16;

__global__ void k_chol_rinv(const double* __restrict__ G, int ldg, int kk, int kp, double shift_rel,
                            double* __restrict__ R, float2* __restrict__ Rinv_df, int* status, bool f64) {
  __shared__ double A[16][17];
  __shared__ double Ri[16][17];
  __shared__ double rdiag[16];  // 1 / R_jj (fast reciprocal: a few ulps)
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
  // right-looking Cholesky A = R^T R, R upper; thread i owns column i.  The
  // square roots and reciprocals take the fast FP64 forms (fp64_fast.cuh): this
  // serial chain runs twice per appended block
  for (int j = 0; j < kk; ++j) {
    if (t == 0) {
      const double d = A[j][j];
      if (!(d > 0.0)) {
        if (!bad) bad = j + 1;
        A[j][j] = 1.0;
        rdiag[j] = 1.0;
      } else {
        const double rs = rsqrt64(d);
        A[j][j] = d * rs;
        rdiag[j] = recip64(A[j][j]);
      }
    }
    __syncthreads();
    if (t > j && t < kk) A[j][t] *= rdiag[j];
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
      Ri[i][t] = s * rdiag[i];
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

// Eigenvalues of the symmetric tridiagonal T (diagonal d, squared
// off-diagonal e2) below x: the sign changes along the leading principal
// minors p_0 = 1, p_1, ..., p_m of T - x I (Sturm sequence property), from
// p_{i+1} = (d_i - x) p_i - e2_{i-1} p_{i-1}: three FP64 operations a step and
// no division (on this GPU every FP64 instruction is expensive, so the
// division of the ratio form dominates it).  Rounding perturbs d_i - x and
// e2_i by a few ulps, as in the ratio form.  A minor that is exactly zero is
// replaced by a tiny one of the sign opposite to its predecessor's (a
// perturbation of d_i far below its rounding); the pair is rescaled by a power
// of two (exact) when the larger magnitude leaves [2^-256, 2^256].  Signs,
// zeros and exponents are read from the high words with integer operations.
__device__ int sturm_count_minors(const double* d, const double* e2, int m, double x) {
  double pm = 1.0, p = __dsub_rn(d[0], x);
  int hm = __double2hiint(pm), cnt = 0;
#pragma unroll 2
  for (int i = 0;; ++i) {
    const double dn = i + 1 < m ? d[i + 1] : 0.0, en = i + 1 < m ? e2[i] : 0.0;
    int hi = __double2hiint(p);
    if (((hi & 0x7FFFFFFF) | __double2loint(p)) == 0) {
      p = __dmul_rn(pm, -0x1p-300);
      hi = __double2hiint(p);
    }
    cnt += ((hi ^ hm) < 0) ? 1 : 0;
    if (i + 1 >= m) break;
    const int ep = (hi >> 20) & 0x7FF, em = (hm >> 20) & 0x7FF, mx = ep > em ? ep : em;
    if (mx > 1023 + 256 || mx < 1023 - 256) {
      const double sc = __hiloint2double((2046 - mx) << 20, 0);
      p = __dmul_rn(p, sc);
      pm = __dmul_rn(pm, sc);
    }
    const double pn = __fma_rn(__dsub_rn(dn, x), p, -__dmul_rn(en, pm));
    pm = p;
    p = pn;
    hm = __double2hiint(pm);
  }
  return cnt;
}

// Narrow [lo, hi] for index w by 33-section in FP64: 32 Sturm counts per round
// (one per lane, at the same cost as one), every lane takes the same decision.
// Stops when hi - lo <= rel * max(|lo|,|hi|) + abs_tol.
__device__ void multisect64(const double* d, const double* e2, int m, int w, double rel, double abs_tol,
                            int max_rounds, double& lo_io, double& hi_io) {
  const int lane = threadIdx.x & 31;
  double lo = lo_io, hi = hi_io;
  for (int it = 0; it < max_rounds; ++it) {
    if (hi - lo <= rel * fmax(fabs(lo), fabs(hi)) + abs_tol) break;
    const double h = (hi - lo) * (1.0 / 33.0);
    const int c = sturm_count_minors(d, e2, m, lo + h * static_cast<double>(lane + 1));
    const unsigned ball = __ballot_sync(0xffffffffu, c > w);
    const int f = ball ? __ffs(ball) - 1 : 32;  // first section point above index w
    const double nlo = f > 0 ? lo + h * static_cast<double>(f) : lo;
    const double nhi = f < 32 ? lo + h * static_cast<double>(f + 1) : hi;
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

__device__ __forceinline__ float recip_of(float x) { return 1.f / x; }
__device__ __forceinline__ double recip_of(double x) { return recip64(x); }

// Solve (T - sigma I) y = y in place for the tridiagonal (d, e), with partial
// pivoting; an exactly zero pivot is set to eps_piv.  One reciprocal per row
// (of the pivot), used by the elimination and kept (rdu) for the
// back-substitution.
template <typename T>
__device__ void tri_shift_solve(const T* d, const T* e, int m, T sigma, T eps_piv, T* y, T* rdu, T* u1, T* u2, T* lm,
                                unsigned char* piv) {
  const T reps = recip_of(eps_piv);
  // 1 / the back-substitution's divisor: the pivot, or +-eps_piv below that
  auto rback = [&](T pv, T r) { return fabs(pv) < eps_piv ? (pv < T(0) ? -reps : reps) : r; };
  T a0 = d[0] - sigma, b0 = (m > 1) ? e[0] : T(0);
  for (int i = 0; i + 1 < m; ++i) {
    const T c = e[i];
    const T a1 = d[i + 1] - sigma;
    const T b1 = (i + 2 < m) ? e[i + 1] : T(0);
    if (fabs(c) > fabs(a0)) {
      piv[i] = 1;
      const T r = recip_of(c);
      rdu[i] = rback(c, r);
      u1[i] = a1;
      u2[i] = b1;
      const T l = a0 * r;
      lm[i] = l;
      a0 = b0 - l * a1;
      b0 = -l * b1;
    } else {
      piv[i] = 0;
      if (a0 == T(0)) a0 = eps_piv;
      const T r = recip_of(a0);
      rdu[i] = rback(a0, r);
      u1[i] = b0;
      u2[i] = T(0);
      const T l = c * r;
      lm[i] = l;
      a0 = a1 - l * b0;
      b0 = b1;
    }
  }
  {
    const T pv = (a0 == T(0)) ? eps_piv : a0;
    rdu[m - 1] = rback(pv, recip_of(pv));
  }
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
    y[i] = sv * rdu[i];
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

// ---- the projected eigensolve on a cluster of kSyC CTAs (one per SM)
//
// The FP64 pipe of this GPU issues one warp instruction in tens of cycles, so a
// single SM spends most of an m = 128 eigensolve in the O(m^3) Householder
// steps.  Here they run over a thread-block cluster: CTA r holds rows r, r + C,
// r + 2C, ... of the matrix, each step's reflector and matrix-vector products
// travel through distributed shared memory, two cluster barriers a step.
constexpr int kSyC = 8;
constexpr int kSyThreads = 512;
constexpr int kSyWarps = kSyThreads / 32;

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// the shared::cluster address of `p` (in this CTA's shared memory) in CTA `rank`
__device__ __forceinline__ uint32_t at_rank(const void* p, unsigned rank) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ float2 ld_cluster(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}

// Shared-memory layout of one CTA (byte offsets), the same in every CTA.
struct SyevLayout {
  int al, vb, pb, wb, kb, red, tau, refl, yd, d, e, e2, y, lo, hi, ev, d32, e232, crowd, total;
  __host__ __device__ explicit SyevLayout(int m) {
    const int rows = (m + kSyC - 1) / kSyC;
    int o = 0;
    auto take = [&](int bytes) {
      const int at = o;
      o += (bytes + 15) & ~15;
      return at;
    };
    al = take(8 * rows * m);           // this CTA's rows
    vb = take(8 * 2 * kMaxM);          // the step's reflector, two buffers
    pb = take(8 * kMaxM);              // p = tau A v, all trailing rows
    wb = take(8 * kMaxM);              // w = p - K v
    kb = take(8 * kSyC);               // the CTAs' parts of p . v
    red = take(8 * 40);
    tau = take(8 * kMaxM);
    refl = take(8 * (m * (m - 1) / 2 + 1));  // reflector j: m - 1 - j slots
    yd = take(8 * kMaxNev * m);
    d = take(8 * m);
    e = take(8 * m);
    e2 = take(8 * m);
    y = take(8 * kMaxNev * m);
    lo = take(8 * kMaxNev);
    hi = take(8 * kMaxNev);
    ev = take(8 * kMaxNev);
    d32 = take(4 * m);
    e232 = take(4 * m);
    crowd = take(4 * kMaxNev);
    total = o;
  }
};

__host__ __device__ inline int refl_off(int j, int m) { return j * (m - 1) - j * (j - 1) / 2; }

// Symmetric eigensolve of the projected matrix, nev lowest pairs.
//  1. Householder tridiagonalisation (Golub and Van Loan, Alg. 8.3.1) in the
//     slot format (double-float, or FP64 for the native FP64 path), distributed
//     over the cluster by rows; every CTA then gathers all reflectors.
//  2. Eigenvalue brackets by Sturm-count multisection in FP32 to ~1e-5; indices
//     whose brackets crowd a neighbour are narrowed further in FP64
//     (division-free counts, 33-section).
//  3. Eigenvectors of the tridiagonal matrix by inverse iteration, one thread
//     per vector: three FP32 steps, then FP64 steps.  Isolated eigenvalues: FP32
//     Rayleigh-quotient shifts, one FP64 step at the FP64 Rayleigh quotient.
//     Crowded groups: shifts at the bracket midpoints (FP64 brackets ~1e-13
//     wide), two FP64 steps, then modified Gram-Schmidt over the crowded
//     vectors.  The eigenvalue is the final Rayleigh quotient.  Every CTA that
//     owns a wanted vector computes all of them (lanes of one warp: the same
//     time as one).
//  4. Back-transformation through the reflectors in the slot format: CTA r
//     takes the vectors c = r (mod C), a warp each.
template <bool F64>
__global__ void __cluster_dims__(kSyC, 1, 1) __launch_bounds__(kSyThreads, 1)
    k_syev_lowest(const double* __restrict__ S, int lds, int m, int nev, double* __restrict__ theta,
                  double* __restrict__ V, int ldv) {
  using AR = Ar<F64>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const SyevLayout L(m);
  float2* Al = reinterpret_cast<float2*>(smraw + L.al);
  float2* vb = reinterpret_cast<float2*>(smraw + L.vb);
  float2* pb = reinterpret_cast<float2*>(smraw + L.pb);
  float2* wb = reinterpret_cast<float2*>(smraw + L.wb);
  float2* kb = reinterpret_cast<float2*>(smraw + L.kb);
  float2* red = reinterpret_cast<float2*>(smraw + L.red);
  float2* tau = reinterpret_cast<float2*>(smraw + L.tau);
  float2* refl = reinterpret_cast<float2*>(smraw + L.refl);
  float2* Yd = reinterpret_cast<float2*>(smraw + L.yd);
  double* d = reinterpret_cast<double*>(smraw + L.d);
  double* e = reinterpret_cast<double*>(smraw + L.e);
  double* e2 = reinterpret_cast<double*>(smraw + L.e2);
  double* Y = reinterpret_cast<double*>(smraw + L.y);
  double* lo = reinterpret_cast<double*>(smraw + L.lo);
  double* hi = reinterpret_cast<double*>(smraw + L.hi);
  double* ev = reinterpret_cast<double*>(smraw + L.ev);
  float* d32 = reinterpret_cast<float*>(smraw + L.d32);
  float* e232 = reinterpret_cast<float*>(smraw + L.e232);
  int* crowd = reinterpret_cast<int*>(smraw + L.crowd);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int rank = static_cast<int>(cluster_rank());
  const int nloc = rank < m ? (m - rank + kSyC - 1) / kSyC : 0;  // rows rank + C li, li < nloc
  for (int x = t; x < nloc * m; x += kSyThreads) {
    const int li = x / m, l = x % m, i = rank + kSyC * li;
    Al[x] = AR::from_d(0.5 * (S[static_cast<int64_t>(i) * lds + l] + S[static_cast<int64_t>(l) * lds + i]));
  }
  __syncthreads();
  // ---- 1. Householder tridiagonalisation over the cluster
  for (int j = 0; j + 2 < m; ++j) {
    const int len = m - j - 1;
    float2* vcur = vb + (j & 1) * kMaxM;
    if (rank == j % kSyC) {
      // the reflector from row j (= column j below the diagonal); it stays in
      // row j, columns j + 1 .., for the back-transformation
      float2* row = Al + (j / kSyC) * m;
      if (warp == 0) {
        typename AR::Acc sa;
        AR::zero(sa);
        for (int l = lane; l < len; l += 32) AR::mac(sa, row[j + 1 + l], row[j + 1 + l]);
        const float2 s2 = warp_sum<F64>(AR::get(sa));
        if (lane == 0) {
          const float2 x0 = row[j + 1];
          float2 tj = make_float2(0.f, 0.f), v0 = x0;
          double ej = 0.0;
          if constexpr (F64) {
            // |v|^2 = 2 (s2 + |x0| ||x||), so tau = 2 / |v|^2 = 1 / (s2 + |x0| ||x||)
            const double s2d = slot_d(s2), x0d = slot_d(x0);
            if (s2d > 0.0) {
              const double nr = s2d * rsqrt64(s2d);
              const double al = x0d >= 0.0 ? -nr : nr;
              v0 = d_slot(x0d - al);
              tj = d_slot(recip64(__fma_rn(fabs(x0d), nr, s2d)));
              ej = al;
            }
          } else {
            const float2 nrm = slot_sqrt<F64>(s2);
            if (AR::lead(nrm) != 0.0) {
              const float2 alpha = (AR::lead(x0) >= 0.0) ? AR::neg(nrm) : nrm;
              v0 = AR::sub(x0, alpha);
              const float2 vtv = AR::add(AR::sub(s2, AR::mul(x0, x0)), AR::mul(v0, v0));
              tj = AR::div(AR::from_d(2.0), vtv);
              ej = AR::to_d(alpha);
            }
          }
          row[j + 1] = v0;
          red[34] = tj;
          red[35] = d_slot(ej);
          red[36] = d_slot(AR::to_d(row[j]));
        }
      }
      __syncthreads();
      for (int x = t; x < kSyC * len; x += kSyThreads) {
        const int q = x / len, l = x % len;
        st_cluster(at_rank(vcur + l, q), row[j + 1 + l]);
      }
      if (t < kSyC) {
        st_cluster(at_rank(tau + j, t), red[34]);
        st_cluster(at_rank(e + j, t), slot_d(red[35]));
        st_cluster(at_rank(d + j, t), slot_d(red[36]));
      }
    }
    cluster_sync();  // the reflector, tau_j, d_j, e_j everywhere
    const float2 tj = tau[j];
    const bool active = AR::lead(tj) != 0.0;
    const int li0 = j + 1 <= rank ? 0 : (j + 1 - rank + kSyC - 1) / kSyC;  // this CTA's trailing rows
    if (active) {
      // p_i = tau_j (A v)_i, a warp per row, sent to every CTA; this CTA's part of p . v
      typename AR::Acc kd;
      AR::zero(kd);
      for (int li = li0 + warp; li < nloc; li += kSyWarps) {
        const int ii = rank + kSyC * li - j - 1;
        const float2* row = Al + li * m + (j + 1);
        typename AR::Acc pa;
        AR::zero(pa);
        for (int l = lane; l < len; l += 32) AR::mac(pa, row[l], vcur[l]);
        const float2 pr = AR::mul(tj, warp_sum<F64>(AR::get(pa)));
        if (lane < kSyC) st_cluster(at_rank(pb + ii, lane), pr);
        AR::mac(kd, pr, vcur[ii]);
      }
      if (lane == 0) red[warp] = AR::get(kd);
      __syncthreads();
      if (warp == 0) {  // the warps' parts summed by a butterfly over lanes 0-15
        float2 k = lane < kSyWarps ? red[lane] : make_float2(0.f, 0.f);
#pragma unroll
        for (int o = kSyWarps / 2; o > 0; o >>= 1) k = AR::add(k, shfl_xor_df(k, o));
        if (lane < kSyC) st_cluster(at_rank(kb + rank, lane), k);
      }
    }
    cluster_sync();  // p and the parts of p . v everywhere
    if (active) {
      if (warp == 0) {
        float2 k = lane < kSyC ? kb[lane] : make_float2(0.f, 0.f);
#pragma unroll
        for (int o = kSyC / 2; o > 0; o >>= 1) k = AR::add(k, shfl_xor_df(k, o));
        if (lane == 0) red[37] = AR::mul(AR::mul(AR::from_d(0.5), tj), k);
      }
      __syncthreads();
      const float2 K = red[37];
      for (int l = t; l < len; l += kSyThreads) wb[l] = AR::sub(pb[l], AR::mul(K, vcur[l]));  // w
      __syncthreads();
      // A -= v w^T + w v^T on this CTA's trailing rows
      for (int li = li0 + warp; li < nloc; li += kSyWarps) {
        const int ii = rank + kSyC * li - j - 1;
        const float2 vi = vcur[ii], wi = wb[ii];
        float2* row = Al + li * m + (j + 1);
        for (int l = lane; l < len; l += 32) {
          if constexpr (F64)
            row[l] = d_slot(__fma_rn(-slot_d(wi), slot_d(vcur[l]), __fma_rn(-slot_d(vi), slot_d(wb[l]), slot_d(row[l]))));
          else
            row[l] = AR::sub(row[l], AR::add(AR::mul(vi, wb[l]), AR::mul(wi, vcur[l])));
        }
      }
    }
    __syncthreads();
  }
  // the last diagonal entries and off-diagonal from their rows' owners
  if (m >= 2) {
    if (rank == (m - 2) % kSyC && t < kSyC) {
      const float2* row = Al + ((m - 2) / kSyC) * m;
      st_cluster(at_rank(d + (m - 2), t), AR::to_d(row[m - 2]));
      st_cluster(at_rank(e + (m - 2), t), AR::to_d(row[m - 1]));
      st_cluster(at_rank(tau + (m - 2), t), make_float2(0.f, 0.f));
    }
    if (rank == (m - 1) % kSyC && t < kSyC) {
      const float2* row = Al + ((m - 1) / kSyC) * m;
      st_cluster(at_rank(d + (m - 1), t), AR::to_d(row[m - 1]));
      st_cluster(at_rank(tau + (m - 1), t), make_float2(0.f, 0.f));
    }
  } else if (rank == 0 && t == 0) {
    d[0] = AR::to_d(Al[0]);
    tau[0] = make_float2(0.f, 0.f);
  }
  cluster_sync();
  // every CTA gathers the reflectors (row j, columns j + 1 .., of CTA j mod C)
  for (int j = warp; j + 2 < m; j += kSyWarps) {
    const uint32_t src = at_rank(Al + (j / kSyC) * m + (j + 1), j % kSyC);
    const int len = m - j - 1, o = refl_off(j, m);
    for (int l = lane; l < len; l += 32) refl[o + l] = ld_cluster(src + 8u * l);
  }
  cluster_sync();  // no CTA leaves while another reads its rows
  if (rank >= nev) return;  // no vector to back-transform here

  for (int i = t; i < m; i += kSyThreads) {
    e2[i] = (i + 1 < m) ? e[i] * e[i] : 0.0;
    d32[i] = static_cast<float>(d[i]);
    e232[i] = static_cast<float>(e2[i]);
  }
  __shared__ double gl, gu, tnorm;
  if (warp == 0) {  // Gershgorin bounds and ||T||: lanes over rows, then a butterfly
    double l0 = 1e300, h0 = -1e300, mx = 0.0;
    for (int i = lane; i < m; i += 32) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
      l0 = fmin(l0, d[i] - r);
      h0 = fmax(h0, d[i] + r);
      mx = fmax(mx, fabs(d[i]) + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
      l0 = fmin(l0, __shfl_xor_sync(0xffffffffu, l0, o));
      h0 = fmax(h0, __shfl_xor_sync(0xffffffffu, h0, o));
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
      tnorm = fmax(mx, 1e-300);
      const double pad = 1e-6 * tnorm + 1e-300;
      gl = l0 - pad;
      gu = h0 + pad;
    }
  }
  __syncthreads();
  // ---- 2. brackets: FP32 multisection, then FP64 for crowded indices
  for (int w = warp; w < nev; w += kSyWarps) {
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
  for (int w = warp; w < nev; w += kSyWarps) {
    if (!crowd[w]) continue;
    // start from the FP32 bracket widened well past the FP32 Sturm error
    // (about m * 2^-24 * ||T||); if the FP64 counts disagree, from the whole interval
    double l0 = lo[w] - 4e-5 * tnorm, h0 = hi[w] + 4e-5 * tnorm;
    const int c = sturm_count_minors(d, e2, m, lane == 0 ? l0 : h0);
    const int cl = __shfl_sync(0xffffffffu, c, 0), ch = __shfl_sync(0xffffffffu, c, 1);
    if (!(cl <= w && ch > w)) {
      l0 = gl;
      h0 = gu;
    }
    multisect64(d, e2, m, w, 1e-13, 1e-15 * tnorm, 24, l0, h0);
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
    // the group below).
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
  // crowded vectors: modified Gram-Schmidt in index order (warp 0, lanes over rows)
  if (warp == 0) {
    for (int c = 0; c < nev; ++c) {
      if (!crowd[c]) continue;
      double* yc = Y + c * m;
      for (int b = 0; b < c; ++b) {
        if (!crowd[b]) continue;
        const double* yb = Y + b * m;
        double dot = 0.0, nb = 0.0;
        for (int i = lane; i < m; i += 32) {
          dot = fma(yb[i], yc[i], dot);
          nb = fma(yb[i], yb[i], nb);
        }
        for (int o = 16; o > 0; o >>= 1) {
          dot += __shfl_xor_sync(0xffffffffu, dot, o);
          nb += __shfl_xor_sync(0xffffffffu, nb, o);
        }
        const double f = dot / nb;
        for (int i = lane; i < m; i += 32) yc[i] -= f * yb[i];
        __syncwarp();
      }
    }
  }
  __syncthreads();
  // normalise, Rayleigh quotient on T (the eigenvalue): a warp per vector
  for (int c = warp; c < nev; c += kSyWarps) {
    double* y = Y + c * m;
    double nn = 0.0;
    for (int i = lane; i < m; i += 32) nn = fma(y[i], y[i], nn);
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    const double inv = 1.0 / sqrt(nn);
    double num = 0.0;
    for (int i = lane; i < m; i += 32) {
      double ty = d[i] * y[i];
      if (i > 0) ty = fma(e[i - 1], y[i - 1], ty);
      if (i + 1 < m) ty = fma(e[i], y[i + 1], ty);
      num = fma(y[i], ty, num);
    }
    for (int o = 16; o > 0; o >>= 1) num += __shfl_xor_sync(0xffffffffu, num, o);
    __syncwarp();
    for (int i = lane; i < m; i += 32) Yd[c * m + i] = AR::from_d(y[i] * inv);
    if (lane == 0) ev[c] = num / nn;
  }
  __syncthreads();
  // ---- 4. back-transform y <- H_0 H_1 ... H_{m-3} y (slot format): vectors
  // c = rank (mod C), a warp each, no block barrier (the reflectors are read only)
  const int c = rank + kSyC * warp;
  if (c < nev) {
    float2* yv = Yd + c * m;
    for (int j = m - 3; j >= 0; --j) {
      const float2 tj = tau[j];
      if (AR::lead(tj) == 0.0) continue;
      const int len = m - j - 1;
      const float2* v = refl + refl_off(j, m);
      typename AR::Acc pa;
      AR::zero(pa);
      for (int i = lane; i < len; i += 32) AR::mac(pa, v[i], yv[j + 1 + i]);
      const float2 sdot = AR::mul(tj, warp_sum<F64>(AR::get(pa)));
      for (int i = lane; i < len; i += 32) yv[j + 1 + i] = AR::sub(yv[j + 1 + i], AR::mul(sdot, v[i]));
      __syncwarp();
    }
    for (int i = lane; i < m; i += 32) V[static_cast<int64_t>(i) * ldv + c] = AR::to_d(yv[i]);
    if (lane == 0) theta[c] = ev[c];
  }
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

cudaError_t syev_lowest(const double* S, int lds, int m, int nev, double* theta, double* V, int ldv, bool f64,
                        cudaStream_t s) {
  if (m < 1 || m > kMaxM || nev < 1 || nev > kMaxNev || nev > m) return cudaErrorInvalidValue;
  const int smem = SyevLayout(m).total;
  static const cudaError_t attr = [] {
    const int most = SyevLayout(kMaxM).total;
    cudaError_t e = cudaFuncSetAttribute(k_syev_lowest<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_syev_lowest<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    return e;
  }();
  if (attr != cudaSuccess) return attr;
  if (f64)
    k_syev_lowest<true><<<kSyC, kSyThreads, smem, s>>>(S, lds, m, nev, theta, V, ldv);
  else
    k_syev_lowest<false><<<kSyC, kSyThreads, smem, s>>>(S, lds, m, nev, theta, V, ldv);
  count_launch();
  return cudaGetLastError();
}

cudaError_t to_df(const double* x, float2* y, int count, double scale, bool f64, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_to_df<<<(count + 255) / 256, 256, 0, s>>>(x, y, count, scale, f64); count_launch();
  return cudaGetLastError();
}

}  // namespace sppc
