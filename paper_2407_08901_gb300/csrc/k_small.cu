// Small dense FP64 kernels, one CTA each: the k x k Cholesky factor and its
// inverse for CholeskyQR (Eq. QR), and the symmetric eigensolve of the projected
// matrix Q^T H Q (Eqs. tilde_H, proj; at most k(p_max+1) <= 144 rows).
//
// The eigensolve reduces the matrix to tridiagonal form with Householder
// reflections (Golub and Van Loan, Alg. 8.3.1), finds the nev lowest eigenvalues
// by Sturm-count multisection, their vectors by inverse iteration on the
// tridiagonal matrix (Wilkinson), cleans the nev vectors with a Rayleigh-Ritz
// step on their span (Jacobi on the nev x nev matrix), and back-transforms
// through the stored reflectors.
#include <math.h>

#include "df.cuh"
#include "sppc_internal.h"

namespace sppc {

namespace {

constexpr int kMaxM = 144;
constexpr int kMaxNev = 16;

__global__ void k_chol_rinv(const double* __restrict__ G, int ldg, int kk, int kp, double shift_rel,
                            double* __restrict__ R, float2* __restrict__ Rinv_df, int* status) {
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
    Rinv_df[e] = in ? df_from_double(Ri[i][j]) : make_float2(0.f, 0.f);
  }
  if (t == 0) status[0] = bad;
}

// Sturm count: number of eigenvalues of the tridiagonal (d, e) below x.
__device__ int sturm_count(const double* d, const double* e2, int m, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0) ++cnt;
  for (int i = 1; i < m; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
  }
  return cnt;
}

__global__ void __launch_bounds__(512) k_syev_lowest(const double* __restrict__ S, int lds, int m, int nev,
                                                     double* __restrict__ theta, double* __restrict__ V, int ldv) {
  extern __shared__ double sm[];
  double* A = sm;                    // m x m (row stride m), reflectors stored below the diagonal
  double* tau = A + m * m;           // m
  double* d = tau + m;               // m
  double* e = d + m;                 // m
  double* e2 = e + m;                // m
  double* vec = e2 + m;              // m  (Householder vector work)
  double* p = vec + m;               // m
  double* Y = p + m;                 // m x nev (column c at Y[c*m])
  double* ev = Y + m * kMaxNev;      // nev
  double* red = ev + kMaxNev;        // 32 reduction slots
  double* G = red + 32;              // nev x nev (Rayleigh-Ritz)
  double* Gv = G + kMaxNev * kMaxNev;  // nev x nev eigenvectors
  double* J = Gv + kMaxNev * kMaxNev;  // nev x nev Jacobi work
  const int t = threadIdx.x, nt = blockDim.x;
  const int lane = t & 31, warp = t >> 5, nwarp = nt >> 5;
  for (int x = t; x < m * m; x += nt) {
    const int i = x / m, j = x % m;
    A[x] = 0.5 * (S[i * lds + j] + S[j * lds + i]);
  }
  __syncthreads();
  // ---- Householder tridiagonalisation
  for (int j = 0; j + 2 < m; ++j) {
    const int len = m - j - 1;
    // norm of x = A[j+1:, j]
    double part = 0.0;
    for (int i = t; i < len; i += nt) {
      const double xv = A[(j + 1 + i) * m + j];
      part += xv * xv;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
      for (int w = 0; w < nwarp; ++w) s += red[w];
      const double x0 = A[(j + 1) * m + j];
      const double nrm = sqrt(s);
      if (nrm == 0.0) {
        tau[j] = 0.0;
        e[j] = 0.0;
        red[31] = 0.0;
      } else {
        const double alpha = (x0 >= 0.0) ? -nrm : nrm;
        const double v0 = x0 - alpha;
        // v = x - alpha e1, tau = 2 / (v^T v) with v^T v = s - x0^2 + v0^2
        const double vtv = s - x0 * x0 + v0 * v0;
        tau[j] = 2.0 / vtv;
        e[j] = alpha;
        red[31] = v0;
      }
    }
    __syncthreads();
    const double tj = tau[j];
    for (int i = t; i < len; i += nt) vec[i] = (i == 0) ? red[31] : A[(j + 1 + i) * m + j];
    __syncthreads();
    if (tj != 0.0) {
      // p = tau * A22 v
      for (int i = t; i < len; i += nt) {
        const double* row = A + (j + 1 + i) * m + (j + 1);
        double s = 0.0;
        for (int l = 0; l < len; ++l) s += row[l] * vec[l];
        p[i] = tj * s;
      }
      __syncthreads();
      double pv = 0.0;
      for (int i = t; i < len; i += nt) pv += p[i] * vec[i];
      for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
      if (lane == 0) red[warp] = pv;
      __syncthreads();
      if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < nwarp; ++w) s += red[w];
        red[30] = 0.5 * tj * s;
      }
      __syncthreads();
      const double K = red[30];
      for (int i = t; i < len; i += nt) p[i] = p[i] - K * vec[i];  // w
      __syncthreads();
      for (int x = t; x < len * len; x += nt) {
        const int i = x / len, l = x % len;
        A[(j + 1 + i) * m + (j + 1 + l)] -= vec[i] * p[l] + p[i] * vec[l];
      }
    }
    __syncthreads();
    for (int i = t; i < len; i += nt) A[(j + 1 + i) * m + j] = vec[i];  // keep v for the back-transform
    if (t == 0) d[j] = A[j * m + j];
    __syncthreads();
  }
  if (t == 0) {
    if (m >= 2) {
      d[m - 2] = A[(m - 2) * m + (m - 2)];
      d[m - 1] = A[(m - 1) * m + (m - 1)];
      e[m - 2] = A[(m - 1) * m + (m - 2)];
      tau[m - 2] = 0.0;
    } else {
      d[0] = A[0];
    }
    for (int i = 0; i + 1 < m; ++i) e2[i] = e[i] * e[i];
  }
  __syncthreads();
  // ---- Gershgorin bounds and multisection for eigenvalues 0..nev-1
  __shared__ double gl, gu, pivmin;
  if (t == 0) {
    double lo = 1e300, hi = -1e300, mx = 0.0;
    for (int i = 0; i < m; ++i) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
      lo = fmin(lo, d[i] - r);
      hi = fmax(hi, d[i] + r);
      mx = fmax(mx, fabs(d[i]) + r);
    }
    const double pad = 2.2e-16 * mx * m + 1e-300;
    gl = lo - pad;
    gu = hi + pad;
    pivmin = fmax(1e-290, 2.2e-16 * 2.2e-16 * fmax(mx * mx, 1e-300));
  }
  __syncthreads();
  for (int w = warp; w < nev; w += nwarp) {
    double lo = gl, hi = gu;
    for (int it = 0; it < 40; ++it) {
      if (hi - lo <= 2.2e-16 * fmax(fabs(lo), fabs(hi)) * 2.0 + pivmin) break;
      const double x = lo + (hi - lo) * (lane + 1) / 33.0;
      const int c = sturm_count(d, e2, m, x, pivmin);
      // first point whose count exceeds w bounds the eigenvalue from above
      const unsigned ball = __ballot_sync(0xffffffffu, c > w);
      double nlo = lo, nhi = hi;
      if (ball) {
        const int f = __ffs(ball) - 1;
        nhi = lo + (hi - lo) * (f + 1) / 33.0;
        if (f > 0) nlo = lo + (hi - lo) * f / 33.0;
      } else {
        nlo = lo + (hi - lo) * 32 / 33.0;
      }
      lo = __shfl_sync(0xffffffffu, nlo, 0);
      hi = __shfl_sync(0xffffffffu, nhi, 0);
    }
    if (lane == 0) ev[w] = 0.5 * (lo + hi);
  }
  __syncthreads();
  // ---- inverse iteration on T - ev I (thread c handles vector c), vectors in Y
  if (t < nev) {
    double* y = Y + t * m;
    const double lam = ev[t];
    double du[kMaxM], u1[kMaxM], u2[kMaxM], lm[kMaxM];
    unsigned char piv[kMaxM];
    double tnorm = 0.0;
    for (int i = 0; i < m; ++i) tnorm = fmax(tnorm, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0));
    const double eps_piv = 2.2e-16 * fmax(tnorm, 1e-300);
    // factor (T - lam I) = P L U, U with diagonals du, u1, u2
    double a0 = d[0] - lam, b0 = (m > 1) ? e[0] : 0.0;
    for (int i = 0; i + 1 < m; ++i) {
      const double c = e[i];                          // subdiagonal element of row i+1
      const double a1 = d[i + 1] - lam;
      const double b1 = (i + 2 < m) ? e[i + 1] : 0.0;
      if (fabs(c) > fabs(a0)) {
        piv[i] = 1;
        du[i] = c;
        u1[i] = a1;
        u2[i] = b1;
        const double l = a0 / c;
        lm[i] = l;
        a0 = b0 - l * a1;
        b0 = -l * b1;
      } else {
        piv[i] = 0;
        if (a0 == 0.0) a0 = eps_piv;
        du[i] = a0;
        u1[i] = b0;
        u2[i] = 0.0;
        const double l = c / a0;
        lm[i] = l;
        a0 = a1 - l * b0;
        b0 = b1;
      }
    }
    du[m - 1] = (a0 == 0.0) ? eps_piv : a0;
    // start vector: a fixed non-symmetric pattern, then 3 iterations
    for (int i = 0; i < m; ++i) y[i] = 1.0 + 0.1 * (double)((i * 7 + t * 3) % 11);
    for (int iter = 0; iter < 3; ++iter) {
      // forward: apply P and L
      for (int i = 0; i + 1 < m; ++i) {
        if (piv[i]) {
          const double tmp = y[i];
          y[i] = y[i + 1];
          y[i + 1] = tmp - lm[i] * y[i];
        } else {
          y[i + 1] -= lm[i] * y[i];
        }
      }
      // backward: U
      for (int i = m - 1; i >= 0; --i) {
        double s = y[i];
        if (i + 1 < m) s -= u1[i] * y[i + 1];
        if (i + 2 < m) s -= u2[i] * y[i + 2];
        double di = du[i];
        if (fabs(di) < eps_piv) di = (di < 0 ? -eps_piv : eps_piv);
        y[i] = s / di;
      }
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) nrm = fmax(nrm, fabs(y[i]));
      for (int i = 0; i < m; ++i) y[i] /= nrm;
    }
  }
  __syncthreads();
  // ---- modified Gram-Schmidt over the nev vectors (parallel over rows)
  for (int c = 0; c < nev; ++c) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int b = 0; b <= c; ++b) {
        double part = 0.0;
        for (int i = t; i < m; i += nt) part += Y[b * m + i] * Y[c * m + i];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        double s = 0.0;
        for (int w = 0; w < nwarp; ++w) s += red[w];
        __syncthreads();
        if (b < c) {
          for (int i = t; i < m; i += nt) Y[c * m + i] -= s * Y[b * m + i];
        } else {
          const double inv = 1.0 / sqrt(s);
          for (int i = t; i < m; i += nt) Y[c * m + i] *= inv;
        }
        __syncthreads();
      }
    }
  }
  // ---- Rayleigh-Ritz on span(Y): G = Y^T T Y (T tridiagonal), Jacobi, rotate
  for (int x = t; x < nev * nev; x += nt) {
    const int a = x / nev, b = x % nev;
    double s = 0.0;
    for (int i = 0; i < m; ++i) {
      double ty = d[i] * Y[b * m + i];
      if (i > 0) ty += e[i - 1] * Y[b * m + i - 1];
      if (i + 1 < m) ty += e[i] * Y[b * m + i + 1];
      s += Y[a * m + i] * ty;
    }
    G[a * kMaxNev + b] = s;
  }
  __syncthreads();
  if (t == 0) {
    for (int a = 0; a < nev; ++a)
      for (int b = 0; b < nev; ++b) {
        const double sym = 0.5 * (G[a * kMaxNev + b] + G[b * kMaxNev + a]);
        J[a * kMaxNev + b] = sym;
        Gv[a * kMaxNev + b] = (a == b) ? 1.0 : 0.0;
      }
    // cyclic Jacobi on the nev x nev matrix in p
    for (int sweep = 0; sweep < 30; ++sweep) {
      double off = 0.0, tot = 0.0;
      for (int a = 0; a < nev; ++a)
        for (int b = 0; b < nev; ++b) {
          const double v = J[a * kMaxNev + b] * J[a * kMaxNev + b];
          tot += v;
          if (a != b) off += v;
        }
      if (off <= 1e-34 * tot || off == 0.0) break;
      for (int a = 0; a < nev - 1; ++a)
        for (int b = a + 1; b < nev; ++b) {
          const double apq = J[a * kMaxNev + b];
          if (apq == 0.0) continue;
          const double app = J[a * kMaxNev + a], aqq = J[b * kMaxNev + b];
          const double th = 0.5 * (aqq - app) / apq;
          const double tt = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
          const double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
          for (int r = 0; r < nev; ++r) {
            const double xa = J[r * kMaxNev + a], xb = J[r * kMaxNev + b];
            J[r * kMaxNev + a] = c * xa - s * xb;
            J[r * kMaxNev + b] = s * xa + c * xb;
          }
          for (int r = 0; r < nev; ++r) {
            const double xa = J[a * kMaxNev + r], xb = J[b * kMaxNev + r];
            J[a * kMaxNev + r] = c * xa - s * xb;
            J[b * kMaxNev + r] = s * xa + c * xb;
          }
          for (int r = 0; r < nev; ++r) {
            const double xa = Gv[r * kMaxNev + a], xb = Gv[r * kMaxNev + b];
            Gv[r * kMaxNev + a] = c * xa - s * xb;
            Gv[r * kMaxNev + b] = s * xa + c * xb;
          }
        }
    }
    // sort ascending (selection sort on the diagonal, permuting Gv columns)
    for (int a = 0; a < nev; ++a) ev[a] = J[a * kMaxNev + a];
    for (int a = 0; a < nev; ++a) {
      int best = a;
      for (int b = a + 1; b < nev; ++b)
        if (ev[b] < ev[best]) best = b;
      if (best != a) {
        const double tv = ev[a];
        ev[a] = ev[best];
        ev[best] = tv;
        for (int r = 0; r < nev; ++r) {
          const double tg = Gv[r * kMaxNev + a];
          Gv[r * kMaxNev + a] = Gv[r * kMaxNev + best];
          Gv[r * kMaxNev + best] = tg;
        }
      }
    }
  }
  __syncthreads();
  // rotate Y by Gv into the back-transform buffer (vec..p area reused: use G region)
  // Yr[c][i] = sum_b Y[b][i] Gv[b][c]; computed row by row into Y in place via a temp per row
  for (int i = t; i < m; i += nt) {
    double tmp[kMaxNev];
    for (int c = 0; c < nev; ++c) {
      double s = 0.0;
      for (int b = 0; b < nev; ++b) s += Y[b * m + i] * Gv[b * kMaxNev + c];
      tmp[c] = s;
    }
    for (int c = 0; c < nev; ++c) Y[c * m + i] = tmp[c];
  }
  __syncthreads();
  // ---- back-transform: y <- H_0 H_1 ... H_{m-3} y, H_j = I - tau_j v_j v_j^T on rows j+1..
  for (int j = m - 3; j >= 0; --j) {
    const double tj = tau[j];
    if (tj == 0.0) continue;
    const int len = m - j - 1;
    for (int c = warp; c < nev; c += nwarp) {
      double part = 0.0;
      for (int i = lane; i < len; i += 32) part += A[(j + 1 + i) * m + j] * Y[c * m + j + 1 + i];
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      const double s = tj * part;
      for (int i = lane; i < len; i += 32) Y[c * m + j + 1 + i] -= s * A[(j + 1 + i) * m + j];
    }
    __syncthreads();
  }
  for (int x = t; x < m * nev; x += nt) {
    const int i = x / nev, c = x % nev;
    V[i * ldv + c] = Y[c * m + i];
  }
  if (t < nev) theta[t] = ev[t];
}

__global__ void k_to_df(const double* __restrict__ x, float2* __restrict__ y, int count, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) y[i] = df_from_double(scale * x[i]);
}

}  // namespace

cudaError_t chol_rinv(const double* G, int ldg, int kk, int kp, double shift_rel, double* R, float2* Rinv_df,
                      int* status, cudaStream_t s) {
  if (kk < 1 || kk > 16 || kp > 16) return cudaErrorInvalidValue;
  k_chol_rinv<<<1, 32, 0, s>>>(G, ldg, kk, kp, shift_rel, R, Rinv_df, status); count_launch();
  return cudaGetLastError();
}

static size_t syev_smem(int m) {
  return sizeof(double) * ((size_t)m * m + 6 * (size_t)m + (size_t)m * kMaxNev + kMaxNev + 32 +
                           3 * kMaxNev * kMaxNev) + 1024;
}

cudaError_t syev_lowest(const double* S, int lds, int m, int nev, double* theta, double* V, int ldv,
                        cudaStream_t s) {
  if (m < 1 || m > kMaxM || nev < 1 || nev > kMaxNev || nev > m) return cudaErrorInvalidValue;
  const size_t smem = syev_smem(m);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_syev_lowest, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)syev_smem(kMaxM));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_syev_lowest<<<1, 512, smem, s>>>(S, lds, m, nev, theta, V, ldv); count_launch();
  return cudaGetLastError();
}

cudaError_t to_df(const double* x, float2* y, int count, double scale, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_to_df<<<(count + 255) / 256, 256, 0, s>>>(x, y, count, scale); count_launch();
  return cudaGetLastError();
}

cudaError_t negate_to_df(const double* x, float2* y, int count, cudaStream_t s) { return to_df(x, y, count, -1.0, s); }

}  // namespace sppc
