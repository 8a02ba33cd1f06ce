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
//   A  per owned element: apply the previous step's Givens update to w and x,
//      v_new = p / beta, y = (H0_hat p - E p) / beta (the SpMM gathers p, which
//      is final), partial dots -> barrier
//   B  reduce the dots (every CTA, same order), p = y - s psi - beta v_prev -
//      alpha v, partial ||p||^2 -> barrier
//   C  reduce ||p||^2, Givens rotation, convergence, coefficients of the next A.
//
// Work split: a row of H0_hat (CSR) is handled by 8 lanes, 4 rows per warp at a
// time.  For the product the 8 lanes are 4 entry segments (entries seg, seg+4,
// ...) x 2 column halves (a half row of p is one 256-bit gather for kp = 8);
// after the segment sums are combined by shuffles, lane (half, seg) owns the
// single element (row, half*kp/2 + seg) for every vector update.  A lane therefore
// reads and writes only its own elements of v, w, x, y, and only p is exchanged
// between CTAs; p is gathered with coherent loads, ordered by the barrier's
// release and acquire operations.  Every CTA computes the same scalars from the
// same partial sums, so no broadcast is needed; the partials of consecutive
// phases go to two alternating buffers, so none is rewritten before every CTA
// has read it.  The grid barrier polls with a bound (default a few seconds,
// opts.spin_cap); on time-out it raises an error flag and every CTA leaves at
// its next barrier.
#include <cooperative_groups.h>

#include "spmm_core.cuh"  // policy_keep, val.cuh

namespace sppc {

namespace {

constexpr int kMinresThreads = 512;  // 16 warps: few CTAs keep barriers and reductions short
constexpr int kMinresWarps = kMinresThreads / 32;

struct MinresKernelArgs {
  CsrDev A;
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
  float2* partials;    // 2 x [32][G] double-float (alternate phases)
  unsigned* bar;       // [0] arrival count, [1] generation
  int* status;         // [0] error flag, [1] iterations run, [2 + j] iterations of column j
  unsigned spin_limit; // polls after which a grid barrier gives up
};

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier: bar[0] counts arrivals and is never reset (barrier b takes the
// values b G .. b G + G - 1, G CTAs), bar[1] holds the number of completed
// barriers.  One thread per CTA arrives with an acquire-release add; the last
// arriver of barrier b publishes b + 1 with a release store, the others poll
// bar[1] with acquire loads.  The CTA barriers on both sides extend the
// ordering to the CTA's other threads.  The poll is bounded (a few seconds); on
// time-out, or when another CTA has raised the error flag, it raises the flag
// and the CTA leaves (the others leave at their next barrier).
constexpr unsigned kSpinLimit = 1u << 22;  // default poll bound (a few seconds)

__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, unsigned limit) {
  __shared__ int s_bar_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned G = gridDim.x;
    const unsigned old = atom_add_acq_rel(bar, 1u);
    const unsigned gen = old / G + 1;
    int ok = 1;
    if (old % G == G - 1) {
      st_release_u32(bar + 1, gen);
    } else {
      unsigned spins = 0;
      while (static_cast<int>(ld_acquire_u32(bar + 1) - gen) < 0) {
        ++spins;
        if (spins > limit || ((spins & 255u) == 0 && *reinterpret_cast<volatile int*>(err))) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
      }
    }
    s_bar_ok = ok;
  }
  __syncthreads();
  return s_bar_ok != 0;
}

// Deterministic grid reduction of nout (<= 32) double-float values.  The
// partials are stored output-major (partials[o * G + g], G CTAs), so the 16
// lanes of a half-warp that share output o = t / 16 read 16 consecutive CTAs'
// values at once.  Lane (o, part) adds CTAs part, part + 16, ... in order, and
// the 16 lane sums are combined by a fixed shuffle tree.  Every CTA computes the
// same result; it lands in red_out (shared).
constexpr int kMaxPartialsPerWarp = 16;  // gridDim.x <= 16 * kMinresWarps
template <class V>
__device__ void reduce_partials(const float2* partials, int nout, float2* red_out) {
  const int t = threadIdx.x;
  const int o = t >> 4, part = t & 15;
  const int G = static_cast<int>(gridDim.x);
  typename V::Acc sa;
  V::zero(sa);
  if (o < nout) {
    float2 v[kMaxPartialsPerWarp];
#pragma unroll
    for (int i = 0; i < kMaxPartialsPerWarp; ++i) {
      const int g = part + i * 16;
      v[i] = (g < G) ? __ldcg(partials + static_cast<int64_t>(o) * G + g) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < kMaxPartialsPerWarp; ++i) {
      V::acc(sa, v[i]);
      V::norm(sa);
    }
  }
  float2 r = V::get(sa);
#pragma unroll
  for (int m = 8; m > 0; m >>= 1) r = V::add(r, shfl_xor_df(r, m));
  if (part == 0 && o < nout) red_out[o] = r;
  __syncthreads();
}

// Coherent gather of the CPL-column half row of p at row cidx (p is rewritten by
// other CTAs between barriers, so the read-only path must not be used).
template <int KP>
__device__ __forceinline__ void gather_p(const float2* X, int cidx, int off, float2 (&x)[KP / 2], uint64_t pol) {
  const float2* p = X + static_cast<int64_t>(cidx) * KP + off;
  if constexpr (KP == 8) {
    float4 a, b;
    asm volatile("ld.global.L2::cache_hint.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p), "l"(pol)
                 : "memory");
    x[0] = make_float2(a.x, a.y);
    x[1] = make_float2(a.z, a.w);
    x[2] = make_float2(b.x, b.y);
    x[3] = make_float2(b.z, b.w);
  } else if constexpr (KP == 4) {
    float4 a;
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w)
                 : "l"(p), "l"(pol)
                 : "memory");
    x[0] = make_float2(a.x, a.y);
    x[1] = make_float2(a.z, a.w);
  } else {
#pragma unroll
    for (int j = 0; j < KP / 2; ++j)
      asm volatile("ld.global.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;"
                   : "=f"(x[j].x), "=f"(x[j].y)
                   : "l"(p + j), "l"(pol)
                   : "memory");
  }
}

// Row sums of H0_hat p for one row: this lane's segment (entries seg, seg+4, ...),
// columns [off, off + CPL), in batches of 4 independent gathers, then the
// segment sums combined across the 4 lanes of the half (all 32 lanes call it).
template <int KP, class V>
__device__ __forceinline__ void row_product(const CsrDev& A, int64_t row, bool valid, int seg, int off,
                                            const float2* P, uint64_t pol, float2 (&out)[KP / 2]) {
  constexpr int CPL = KP / 2;
  typename V::Acc acc[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) V::zero(acc[c]);
  if (valid) {
    const int64_t rb = __ldg(A.rowptr + row), re = __ldg(A.rowptr + row + 1);
    for (int64_t e = rb + seg; e < re; e += 16) {
      int cc[4];
      float2 vv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t ee = e + 4 * u;
        cc[u] = (ee < re) ? __ldg(A.col + ee) : -1;
        vv[u] = (ee < re) ? __ldg(A.val + ee) : make_float2(0.f, 0.f);
      }
      float2 xx[4][CPL];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (cc[u] >= 0) {
          gather_p<KP>(P, cc[u], off, xx[u], pol);
        } else {
#pragma unroll
          for (int c = 0; c < CPL; ++c) xx[u][c] = make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < CPL; ++c) V::mac(acc[c], vv[u], xx[u][c]);
#pragma unroll
      for (int c = 0; c < CPL; ++c) V::norm(acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    float2 v = V::get(acc[c]);
    v = V::add(v, shfl_xor_df(v, 1));
    v = V::add(v, shfl_xor_df(v, 2));
    out[c] = v;
  }
}

template <int KP, class V>
__global__ void __launch_bounds__(kMinresThreads, 1) k_minres(MinresKernelArgs a) {
  using Acc = typename V::Acc;
  constexpr int CPL = KP / 2;
  constexpr int kRowsPerWarp = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rq = lane >> 3;             // row of the warp's group of 4
  const int half = (lane >> 2) & 1;     // column half
  const int seg = lane & 3;             // entry segment; element column in the half
  const int off = half * CPL;
  const int j = off + seg;              // owned element column (valid if seg < CPL)
  const bool has_col = seg < CPL;
  const int64_t n = a.A.nrows;
  const int64_t row0 = (static_cast<int64_t>(blockIdx.x) * kMinresWarps + warp) * kRowsPerWarp;
  const int64_t rstride = static_cast<int64_t>(gridDim.x) * kMinresWarps * kRowsPerWarp;
  const uint64_t pol = policy_keep();
  int* err = a.status;

  __shared__ float2 sdot[32];
  __shared__ float2 wred[kMinresWarps][32];
  // per-column MINRES state (identical in every CTA)
  __shared__ double st_beta[8], st_cp[8], st_cc[8], st_sp[8], st_sc[8], st_eta[8], st_rn[8], st_b1[8], st_alpha[8];
  __shared__ int st_done[8], st_it[8];
  // coefficients (double-float) of the element updates
  __shared__ float2 c_invb[8], c_wa[8], c_w2[8], c_w1[8], c_x[8], c_s[8], c_beta[8], c_alpha[8];
  __shared__ int s_dow, s_all;

  float2 *P = a.P, *Vv = a.V, *VP = a.VP, *W1 = a.W1, *W2 = a.W2;

  // Two partial buffers, used by alternate phases (init and B: 1, A: 0): a CTA
  // rewrites a buffer only after the next grid barrier, which every CTA reaches
  // after its reads of that buffer.
  float2* const pbuf[2] = {a.partials, a.partials + static_cast<int64_t>(32) * gridDim.x};
  // write this CTA's partial of nq dots (columns 0..KP-1) to buf[o * G + blockIdx]
  auto flush = [&](Acc (&d)[4], int nq, float2* buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q >= nq) break;
      float2 v = has_col ? V::get(d[q]) : make_float2(0.f, 0.f);
      // sum over the 4 rows of the warp (lanes with equal half and seg)
      v = V::add(v, shfl_xor_df(v, 8));
      v = V::add(v, shfl_xor_df(v, 16));
      if (lane < 8 && has_col) wred[warp][q * 8 + j] = v;
    }
    __syncthreads();
    {
      // the 16 warps' values of output o, combined by a fixed shuffle tree
      static_assert(kMinresWarps == 16, "one half-warp per output");
      const int o = threadIdx.x >> 4, w = threadIdx.x & 15;
      float2 v = (o < nq * 8) ? wred[w][o] : make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 8; m > 0; m >>= 1) v = V::add(v, shfl_xor_df(v, m));
      if (w == 0 && o < nq * 8) buf[static_cast<int64_t>(o) * gridDim.x + blockIdx.x] = v;
    }
    __syncthreads();
  };
  auto zero4 = [](Acc (&d)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) V::zero(d[q]);
  };

  for (int t = threadIdx.x; t < kMinresWarps * 32; t += kMinresThreads)
    wred[t / 32][t % 32] = make_float2(0.f, 0.f);
  __syncthreads();
  Acc dd[4];
  // ---- init: zero V, VP, W1, W2, X on owned elements; ||b1||^2 partial
  zero4(dd);
  for (int64_t r0 = row0; r0 < n; r0 += rstride) {
    const int64_t row = r0 + rq;
    if (row >= n || !has_col) continue;
    const int64_t b = row * KP + j;
    const float2 z = make_float2(0.f, 0.f);
    Vv[b] = z;
    VP[b] = z;
    W1[b] = z;
    W2[b] = z;
    a.X[b] = z;
    const float2 pv = P[b];
    V::mac(dd[0], pv, pv);
    V::norm(dd[0]);
  }
  flush(dd, 1, pbuf[1]);
  if (!grid_barrier(a.bar, err, a.spin_limit)) return;
  reduce_partials<V>(pbuf[1], 8, sdot);
  if (threadIdx.x < 8) {
    const int jj = threadIdx.x;
    const double b1 = (jj < a.k) ? sqrt(fmax(V::to_d(sdot[jj]), 0.0)) : 0.0;
    st_beta[jj] = b1;
    st_b1[jj] = b1;
    st_eta[jj] = b1;
    st_rn[jj] = b1;
    st_cp[jj] = st_cc[jj] = 1.0;
    st_sp[jj] = st_sc[jj] = 0.0;
    st_done[jj] = (b1 > 0.0) ? 0 : 1;
    st_it[jj] = 0;
    c_invb[jj] = st_done[jj] ? make_float2(0.f, 0.f) : V::from_d(1.0 / b1);
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
    zero4(dd);
    for (int64_t r0 = row0; r0 < n; r0 += rstride) {
      const int64_t row = r0 + rq;
      const bool valid = row < n;
      float2 hp[CPL];
      if (!finish) row_product<KP, V>(a.A, row, valid, seg, off, P, pol, hp);
      if (!valid || !has_col) continue;
      const int64_t b = row * KP + j;
      const float2 vold = Vv[b];
      if (s_dow) {
        // w_new = (v - rho3 w2 - rho2 w1) / rho1 ; x += c eta w_new
        float2 wn = V::mul(c_wa[j], vold);
        wn = V::add(wn, V::mul(c_w2[j], W2[b]));
        wn = V::add(wn, V::mul(c_w1[j], W1[b]));
        W2[b] = wn;  // W2's buffer becomes w_new (roles swap below)
        a.X[b] = V::add(a.X[b], V::mul(c_x[j], wn));
      }
      if (finish) continue;
      float2 hj = hp[0];
#pragma unroll
      for (int c = 1; c < CPL; ++c)
        if (c == seg) hj = hp[c];
      const float2 pv = P[b];
      const float2 vn = V::mul(c_invb[j], pv);
      VP[b] = vn;  // VP's buffer becomes v_new (roles swap below)
      // y = (H0_hat p - E p) / beta
      float2 y = V::add(hj, V::mul(a.negE[j], pv));
      y = V::mul(c_invb[j], y);
      a.Y[b] = y;
      const float2 ps = __ldg(a.psi + b);
      V::mac(dd[0], vn, y);
      V::mac(dd[1], ps, y);
      V::mac(dd[2], vn, ps);
      V::mac(dd[3], vn, vold);
#pragma unroll
      for (int q = 0; q < 4; ++q) V::norm(dd[q]);
    }
    if (s_dow) {
      float2* t = W2;
      W2 = W1;
      W1 = t;
    }
    if (finish) break;
    {
      float2* t = VP;
      VP = Vv;
      Vv = t;
    }
    flush(dd, 4, pbuf[0]);
    if (!grid_barrier(a.bar, err, a.spin_limit)) return;
    // ---- phase B
    reduce_partials<V>(pbuf[0], 32, sdot);
    if (threadIdx.x < 8) {
      const int jj = threadIdx.x;
      double s = 0.0, al = 0.0;
      if (!st_done[jj]) {
        s = V::to_d(sdot[8 + jj]);
        al = V::to_d(sdot[jj]) - s * V::to_d(sdot[16 + jj]) - st_beta[jj] * V::to_d(sdot[24 + jj]);
      }
      st_alpha[jj] = al;
      c_s[jj] = V::from_d(-s);
      c_beta[jj] = V::from_d(st_done[jj] ? 0.0 : -st_beta[jj]);
      c_alpha[jj] = V::from_d(-al);
    }
    __syncthreads();
    zero4(dd);
    for (int64_t r0 = row0; r0 < n; r0 += rstride) {
      const int64_t row = r0 + rq;
      if (row >= n || !has_col) continue;
      const int64_t b = row * KP + j;
      float2 pn = a.Y[b];
      pn = V::add(pn, V::mul(c_s[j], __ldg(a.psi + b)));
      pn = V::add(pn, V::mul(c_beta[j], VP[b]));
      pn = V::add(pn, V::mul(c_alpha[j], Vv[b]));
      P[b] = pn;
      V::mac(dd[0], pn, pn);
      V::norm(dd[0]);
    }
    flush(dd, 1, pbuf[1]);
    if (!grid_barrier(a.bar, err, a.spin_limit)) return;
    // ---- phase C
    reduce_partials<V>(pbuf[1], 8, sdot);
    ++it;
    if (threadIdx.x < 8) {
      const int jj = threadIdx.x;
      const float2 z = make_float2(0.f, 0.f);
      if (st_done[jj]) {
        c_wa[jj] = c_w2[jj] = c_w1[jj] = c_x[jj] = c_invb[jj] = z;
      } else {
        const double bn = sqrt(fmax(V::to_d(sdot[jj]), 0.0));
        const double al = st_alpha[jj], be = st_beta[jj];
        const double delta = st_cc[jj] * al - st_cp[jj] * st_sc[jj] * be;
        // delta and beta are of the order of ||H0_hat||: no overflow guard needed
        const double rho1 = sqrt(delta * delta + bn * bn);
        const double rho2 = st_sc[jj] * al + st_cp[jj] * st_cc[jj] * be;
        const double rho3 = st_sp[jj] * be;
        st_it[jj] += 1;
        if (rho1 == 0.0) {
          st_done[jj] = 1;
          c_wa[jj] = c_w2[jj] = c_w1[jj] = c_x[jj] = c_invb[jj] = z;
        } else {
          const double inv = 1.0 / rho1;  // one division, the rest are products
          const double cn = delta * inv, sn = bn * inv;
          c_wa[jj] = V::from_d(inv);
          c_w2[jj] = V::from_d(-rho3 * inv);
          c_w1[jj] = V::from_d(-rho2 * inv);
          c_x[jj] = V::from_d(cn * st_eta[jj]);
          st_rn[jj] = fabs(sn) * st_rn[jj];
          st_eta[jj] = -sn * st_eta[jj];
          st_cp[jj] = st_cc[jj];
          st_cc[jj] = cn;
          st_sp[jj] = st_sc[jj];
          st_sc[jj] = sn;
          const bool conv = (st_rn[jj] <= a.tol * st_b1[jj]) || (bn == 0.0);
          if (conv) st_done[jj] = 1;
          c_invb[jj] = conv ? z : V::from_d(1.0 / bn);
        }
        st_beta[jj] = bn;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int all = 1;
      for (int jj = 0; jj < a.k; ++jj) all &= st_done[jj];
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
// X receives the solution.  All n1 x kp value slots in A's format; with fp32 the
// iteration runs in FP32 on the slots' leading words and writes FP32 values
// (a double-float slot with a zero low word).  status (host-visible via
// a copy): [0] time-out flag, [1] iterations (negative: limit reached),
// [2+j] iterations of column j.  bar: two zeroed unsigned words.
cudaError_t minres_persistent(const CsrDev& A, int k, int kp, const float2* negE, const float2* psi, float2* P,
                              float2* V, float2* VP, float2* Y, float2* W1, float2* W2, float2* X, double tol,
                              int maxit, float2* partials, int64_t partial_cap, unsigned* bar, int* status,
                              cudaStream_t s, int max_ctas, int spin_cap, bool fp32) {
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return cudaErrorNotSupported;
  const void* fn = nullptr;
  // arithmetic: FP32 on request, else the matrix's slot format
  const int fmt = fp32 ? 2 : (A.f64 ? 1 : 0);
  switch (kp * 4 + fmt) {
    case 8: fn = reinterpret_cast<const void*>(k_minres<2, Ar<false>>); break;
    case 9: fn = reinterpret_cast<const void*>(k_minres<2, Ar<true>>); break;
    case 10: fn = reinterpret_cast<const void*>(k_minres<2, ArF32>); break;
    case 16: fn = reinterpret_cast<const void*>(k_minres<4, Ar<false>>); break;
    case 17: fn = reinterpret_cast<const void*>(k_minres<4, Ar<true>>); break;
    case 18: fn = reinterpret_cast<const void*>(k_minres<4, ArF32>); break;
    case 24: fn = reinterpret_cast<const void*>(k_minres<6, Ar<false>>); break;
    case 25: fn = reinterpret_cast<const void*>(k_minres<6, Ar<true>>); break;
    case 26: fn = reinterpret_cast<const void*>(k_minres<6, ArF32>); break;
    case 32: fn = reinterpret_cast<const void*>(k_minres<8, Ar<false>>); break;
    case 33: fn = reinterpret_cast<const void*>(k_minres<8, Ar<true>>); break;
    case 34: fn = reinterpret_cast<const void*>(k_minres<8, ArF32>); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMinresThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t rows_per_cta = static_cast<int64_t>(kMinresWarps) * 4;
  int64_t grid = (A.nrows + rows_per_cta - 1) / rows_per_cta;
  const int64_t gmax = static_cast<int64_t>(sms) * per_sm;
  if (grid > gmax) grid = gmax;
  if (grid < 1) grid = 1;
  if (grid > static_cast<int64_t>(kMaxPartialsPerWarp) * kMinresWarps) grid = kMaxPartialsPerWarp * kMinresWarps;
  if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
  if (grid * 64 > partial_cap) return cudaErrorInvalidValue;
  e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(status, 0, 10 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const unsigned spin_limit = spin_cap > 0 ? static_cast<unsigned>(spin_cap) : kSpinLimit;
  MinresKernelArgs args{A, k, negE, psi, P, V, VP, Y, W1, W2, X, tol, maxit, partials, bar, status, spin_limit};
  void* params[] = {&args};
  count_launch();
  return cudaLaunchCooperativeKernel(fn, dim3(static_cast<unsigned>(grid)), dim3(kMinresThreads), params, 0, s);
}

}  // namespace sppc
