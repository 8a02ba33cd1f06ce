// Persistent MINRES for the k shifted small-space systems of Eq. (sm_lin_proj):
// (H0_hat - E_k^(0)) x1 = b1 on the complement of psi_hat_k, all k columns at
// once, one cooperative launch per solve.
//
// MINRES (Paige and Saunders, 1975): the Lanczos three-term recurrence on the
// projected operator P (H0_hat - E) P, P = I - psi psi^T, builds the Krylov
// basis; the tridiagonal least-squares problem is kept in QR form by one Givens
// rotation per step; the iterate is updated through the three-term recurrence of
// the search directions w.  The Lanczos step follows the order of the oracle:
// with y = (H0_hat - E) v and the dots (v,y), (psi,y), (v,psi), (v,v_prev),
// s = psi^T y, alpha = v^T (P y - beta v_prev), p = P y - beta v_prev - alpha v.
//
// Schedule per iteration (two grid-wide barriers):
//   A  per owned row: apply the previous step's Givens update to w and x,
//      v_new = p / beta, y = (H0_hat p - E p) / beta (the SpMM gathers p, which
//      is final), partial dots -> barrier
//   B  reduce the dots (every CTA, same order), p = y - s psi - beta v_prev -
//      alpha v, partial ||p||^2 -> barrier
//   C  reduce ||p||^2, Givens rotation, convergence, coefficients of the next A.
// Rows are owned by the warp whose SpMM slice holds them (two lanes per row),
// so all row updates are local.  Every CTA computes the same scalars from the
// same partial sums, so no broadcast is needed.  The grid barrier spins with a
// bound (about a second); on time-out it raises an error flag and every CTA
// leaves at its next barrier.
#include <cooperative_groups.h>

#include "spmm_core.cuh"

namespace sppc {

namespace {

constexpr int kMinresThreads = 512;  // 16 warps: few CTAs keep barriers and reductions short
constexpr int kMinresWarps = kMinresThreads / 32;

struct MinresKernelArgs {
  SellDev A;
  int k;
  const float2* negE;  // -E_k^(0) per column, double-float
  const float2* psi;   // n1 x kp
  float2* P;           // in: b1; work: unnormalised Lanczos vector
  float2* V;
  float2* VP;
  float2* Y;
  float2* W1;
  float2* W2;
  float2* X;           // out: solution
  double tol;
  int maxit;
  float2* partials;    // [G][32] double-float
  unsigned* bar;       // [0] arrival count, [1] generation
  int* status;         // [0] error flag, [1] iterations run, [2 + j] iterations of column j
};

__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      bar[0] = 0;
      __threadfence();
      atomicExch(bar + 1, g + 1);
    } else {
      unsigned spins = 0;
      while (*gen == g) {
        if (++spins > (1u << 24) || *reinterpret_cast<volatile int*>(err)) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *reinterpret_cast<volatile int*>(err) == 0;
}

// Deterministic grid reduction of nout (<= 32) double-float values: every CTA
// reads all CTAs' partials in the same order (warp w sums CTAs w, w+16, ...;
// the 16 warp sums are then added in order).  Result in red_out (shared).
__device__ void reduce_partials(const float2* partials, int nout, float2* sred /*[16][32]*/, float2* red_out) {
  const int t = threadIdx.x;
  const int o = t & 31, part = t >> 5;
  if (o < nout) {
    float sh = 0.f, sl = 0.f;
    for (int g = part; g < (int)gridDim.x; g += kMinresWarps) {
      acc_add(sh, sl, partials[static_cast<int64_t>(g) * 32 + o]);
      acc_norm(sh, sl);
    }
    sred[part * 32 + o] = acc_get(sh, sl);
  }
  __syncthreads();
  if (t < nout) {
    float2 r = sred[t];
    for (int w = 1; w < kMinresWarps; ++w) r = df_add(r, sred[w * 32 + t]);
    red_out[t] = r;
  }
  __syncthreads();
}

template <int KP>
__global__ void __launch_bounds__(kMinresThreads) k_minres(MinresKernelArgs a) {
  constexpr int CPL = KP / 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rl = lane >> 1;
  const int off = (lane & 1) * CPL;
  const int64_t gw = static_cast<int64_t>(blockIdx.x) * kMinresWarps + warp;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * kMinresWarps;
  const uint64_t pol = policy_keep();
  int* err = a.status;

  __shared__ float2 sred[kMinresWarps * 32];
  __shared__ float2 sdot[32];
  __shared__ float2 wred[kMinresWarps][32];
  // per-column MINRES state (identical in every CTA)
  __shared__ double st_beta[8], st_cp[8], st_cc[8], st_sp[8], st_sc[8], st_eta[8], st_rn[8], st_b1[8], st_alpha[8];
  __shared__ int st_done[8], st_it[8];
  // coefficients (double-float) of the row updates
  __shared__ float2 c_invb[8], c_wa[8], c_w2[8], c_w1[8], c_x[8], c_s[8], c_beta[8], c_alpha[8];
  __shared__ int s_dow, s_all;

  float2 *P = a.P, *V = a.V, *VP = a.VP, *W1 = a.W1, *W2 = a.W2;

  // block-level dot accumulation helpers: lane holds CPL columns of one row
  auto zero_acc = [](float (&h)[4][CPL], float (&l)[4][CPL]) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < CPL; ++c) h[q][c] = l[q][c] = 0.f;
  };
  // write this CTA's partial of nq dots (columns 0..KP-1) to partials[blockIdx]
  auto flush = [&](float (&h)[4][CPL], float (&l)[4][CPL], int nq) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q >= nq) break;
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        float2 v = acc_get(h[q][c], l[q][c]);
        // sum over the 16 rows of the warp (lanes of equal parity)
#pragma unroll
        for (int m = 2; m < 32; m <<= 1) v = df_add(v, shfl_xor_df(v, m));
        if (lane < 2) wred[warp][q * 8 + off + c] = v;
      }
    }
    __syncthreads();
    if (threadIdx.x < nq * 8) {
      float2 sacc = wred[0][threadIdx.x];
      for (int w = 1; w < kMinresWarps; ++w) sacc = df_add(sacc, wred[w][threadIdx.x]);
      a.partials[static_cast<int64_t>(blockIdx.x) * 32 + threadIdx.x] = sacc;
    }
    __syncthreads();
  };

  for (int t = threadIdx.x; t < kMinresWarps * 32; t += kMinresThreads)
    wred[t / 32][t % 32] = make_float2(0.f, 0.f);
  __syncthreads();
  float dh[4][CPL], dl[4][CPL];
  // ---- init: zero V, VP, W1, W2, X on owned rows; ||b1||^2 partial
  zero_acc(dh, dl);
  for (int64_t s = gw; s < a.A.nslices; s += nw) {
    const int row = a.A.slice_rows[s * kSliceH + rl];
    if (row < 0) continue;
    const int64_t b = static_cast<int64_t>(row) * KP + off;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const float2 z = make_float2(0.f, 0.f);
      V[b + c] = z;
      VP[b + c] = z;
      W1[b + c] = z;
      W2[b + c] = z;
      a.X[b + c] = z;
      const float2 pv = P[b + c];
      acc_mac(dh[0][c], dl[0][c], pv, pv);
    }
  }
  flush(dh, dl, 1);
  if (!grid_barrier(a.bar, err)) return;
  reduce_partials(a.partials, 8, sred, sdot);
  if (threadIdx.x < 8) {
    const int j = threadIdx.x;
    const double b1 = (j < a.k) ? sqrt(fmax(df_to_double(sdot[j]), 0.0)) : 0.0;
    st_beta[j] = b1;
    st_b1[j] = b1;
    st_eta[j] = b1;
    st_rn[j] = b1;
    st_cp[j] = st_cc[j] = 1.0;
    st_sp[j] = st_sc[j] = 0.0;
    st_done[j] = (b1 > 0.0) ? 0 : 1;
    st_it[j] = 0;
    c_invb[j] = st_done[j] ? make_float2(0.f, 0.f) : df_from_double(1.0 / b1);
  }
  if (threadIdx.x == 0) {
    s_dow = 0;
    s_all = 0;
  }
  __syncthreads();

  int it = 0;
  bool finish = false;
  while (true) {
    // ---- phase A
    zero_acc(dh, dl);
    for (int64_t s = gw; s < a.A.nslices; s += nw) {
      const int row = a.A.slice_rows[s * kSliceH + rl];
      float ah[CPL], al[CPL];
      if (!finish) slice_rowsum<KP>(a.A, s, rl, off, P, pol, ah, al);
      if (row < 0) continue;
      const int64_t b = static_cast<int64_t>(row) * KP + off;
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = off + c;
        const float2 vold = V[b + c];
        if (s_dow) {
          // w_new = (v - rho3 w2 - rho2 w1) / rho1 ; x += c eta w_new
          float2 wn = df_mul(c_wa[j], vold);
          wn = df_add(wn, df_mul(c_w2[j], W2[b + c]));
          wn = df_add(wn, df_mul(c_w1[j], W1[b + c]));
          W2[b + c] = wn;  // W2's buffer becomes w_new (roles swap below)
          a.X[b + c] = df_add(a.X[b + c], df_mul(c_x[j], wn));
        }
        if (finish) continue;
        const float2 pv = P[b + c];
        const float2 vn = df_mul(c_invb[j], pv);
        VP[b + c] = vn;  // VP's buffer becomes v_new (roles swap below)
        // y = (H0_hat p - E p) / beta
        float2 y = df_add(acc_get(ah[c], al[c]), df_mul(a.negE[j], pv));
        y = df_mul(c_invb[j], y);
        a.Y[b + c] = y;
        const float2 ps = a.psi[b + c];
        acc_mac(dh[0][c], dl[0][c], vn, y);
        acc_mac(dh[1][c], dl[1][c], ps, y);
        acc_mac(dh[2][c], dl[2][c], vn, ps);
        acc_mac(dh[3][c], dl[3][c], vn, vold);
      }
    }
    if (s_dow) {
      float2* t = W2;
      W2 = W1;
      W1 = t;
    }
    if (finish) break;
    {
      float2* t = VP;
      VP = V;
      V = t;
    }
    flush(dh, dl, 4);
    if (!grid_barrier(a.bar, err)) return;
    // ---- phase B
    reduce_partials(a.partials, 32, sred, sdot);
    if (threadIdx.x < 8) {
      const int j = threadIdx.x;
      double s = 0.0, al = 0.0;
      if (!st_done[j]) {
        s = df_to_double(sdot[8 + j]);
        al = df_to_double(sdot[j]) - s * df_to_double(sdot[16 + j]) - st_beta[j] * df_to_double(sdot[24 + j]);
      }
      st_alpha[j] = al;
      c_s[j] = df_from_double(-s);
      c_beta[j] = df_from_double(st_done[j] ? 0.0 : -st_beta[j]);
      c_alpha[j] = df_from_double(-al);
    }
    __syncthreads();
    zero_acc(dh, dl);
    for (int64_t s = gw; s < a.A.nslices; s += nw) {
      const int row = a.A.slice_rows[s * kSliceH + rl];
      if (row < 0) continue;
      const int64_t b = static_cast<int64_t>(row) * KP + off;
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = off + c;
        float2 pn = a.Y[b + c];
        pn = df_add(pn, df_mul(c_s[j], a.psi[b + c]));
        pn = df_add(pn, df_mul(c_beta[j], VP[b + c]));
        pn = df_add(pn, df_mul(c_alpha[j], V[b + c]));
        P[b + c] = pn;
        acc_mac(dh[0][c], dl[0][c], pn, pn);
      }
    }
    flush(dh, dl, 1);
    if (!grid_barrier(a.bar, err)) return;
    // ---- phase C
    reduce_partials(a.partials, 8, sred, sdot);
    ++it;
    if (threadIdx.x < 8) {
      const int j = threadIdx.x;
      const float2 z = make_float2(0.f, 0.f);
      if (st_done[j]) {
        c_wa[j] = c_w2[j] = c_w1[j] = c_x[j] = c_invb[j] = z;
      } else {
        const double bn = sqrt(fmax(df_to_double(sdot[j]), 0.0));
        const double al = st_alpha[j], be = st_beta[j];
        const double delta = st_cc[j] * al - st_cp[j] * st_sc[j] * be;
        const double rho1 = hypot(delta, bn);
        const double rho2 = st_sc[j] * al + st_cp[j] * st_cc[j] * be;
        const double rho3 = st_sp[j] * be;
        st_it[j] += 1;
        if (rho1 == 0.0) {
          st_done[j] = 1;
          c_wa[j] = c_w2[j] = c_w1[j] = c_x[j] = c_invb[j] = z;
        } else {
          const double cn = delta / rho1, sn = bn / rho1;
          c_wa[j] = df_from_double(1.0 / rho1);
          c_w2[j] = df_from_double(-rho3 / rho1);
          c_w1[j] = df_from_double(-rho2 / rho1);
          c_x[j] = df_from_double(cn * st_eta[j]);
          st_rn[j] = fabs(sn) * st_rn[j];
          st_eta[j] = -sn * st_eta[j];
          st_cp[j] = st_cc[j];
          st_cc[j] = cn;
          st_sp[j] = st_sc[j];
          st_sc[j] = sn;
          const bool conv = (st_rn[j] <= a.tol * st_b1[j]) || (bn == 0.0);
          if (conv) st_done[j] = 1;
          c_invb[j] = conv ? z : df_from_double(1.0 / bn);
        }
        st_beta[j] = bn;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int all = 1;
      for (int j = 0; j < a.k; ++j) all &= st_done[j];
      s_all = all;
      s_dow = 1;
    }
    __syncthreads();
    if (s_all || it >= a.maxit) finish = true;  // one more phase A applies the last w/x update
  }
  if (blockIdx.x == 0 && threadIdx.x < 8) {
    a.status[2 + threadIdx.x] = st_it[threadIdx.x];
    if (threadIdx.x == 0) a.status[1] = s_all ? it : -it;
  }
}

}  // namespace

// Buffers: P holds b1 on entry (overwritten); V, VP, Y, W1, W2 are scratch;
// X receives the solution.  All n1 x kp double-float.  status (host-visible via
// a copy): [0] time-out flag, [1] iterations (negative: limit reached),
// [2+j] iterations of column j.  bar: two zeroed unsigned words.
cudaError_t minres_persistent(const SellDev& A, int k, int kp, const float2* negE, const float2* psi, float2* P,
                              float2* V, float2* VP, float2* Y, float2* W1, float2* W2, float2* X, double tol,
                              int maxit, float2* partials, int64_t partial_cap, unsigned* bar, int* status,
                              cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return cudaErrorNotSupported;
  const void* fn = nullptr;
  switch (kp) {
    case 2: fn = reinterpret_cast<const void*>(k_minres<2>); break;
    case 4: fn = reinterpret_cast<const void*>(k_minres<4>); break;
    case 6: fn = reinterpret_cast<const void*>(k_minres<6>); break;
    case 8: fn = reinterpret_cast<const void*>(k_minres<8>); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMinresThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (A.nslices + kMinresWarps - 1) / kMinresWarps;
  const int64_t gmax = static_cast<int64_t>(sms) * per_sm;
  if (grid > gmax) grid = gmax;
  if (grid < 1) grid = 1;
  if (grid * 32 > partial_cap) return cudaErrorInvalidValue;
  e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(status, 0, 10 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  MinresKernelArgs args{A, k, negE, psi, P, V, VP, Y, W1, W2, X, tol, maxit, partials, bar, status};
  void* params[] = {&args};
  count_launch();
  return cudaLaunchCooperativeKernel(fn, dim3(static_cast<unsigned>(grid)), dim3(kMinresThreads), params, 0, s);
}

}  // namespace sppc
