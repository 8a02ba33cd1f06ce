// SpMM Y = H X over the level-blocked SELL-16 layout, in double-float or native
// FP64 arithmetic (the matrix's slot format, val.cuh).
//
// The product with H is the dominant cost of SPPC: k SpMVs per order (paper
// Sec. 4.2-4.3), plus the products with the leading block H0_hat inside the
// small solves.  One warp owns a 16-row slice, two lanes per row, so the row
// reduction needs no shuffles; the 16 rows' t-th entries are contiguous, so
// column indices (4 B) and double-float values (8 B) stream in coalesced 64 B /
// 128 B transactions with an evict-first hint (they are read once).  Each entry
// gathers one row of X (kp double-float values, 16-64 B); the two lanes of a row
// each fetch half of it, so one warp load touches 16 rows (one L1 wavefront per
// row) instead of 32 rows four times over.  Gathers run one entry ahead with
// an L2 evict-last hint; slices follow the level order, so a wave of warps
// gathers from one window of levels of X.
#include <atomic>

#include "spmm_core.cuh"

namespace sppc {

namespace {

// SELL-16: a warp owns a 16-row slice, two lanes per row (slice_rowsum); the
// epilogue writes, accumulates (column tiles) or finishes Y.
// Seven resident CTAs per SM (<= 73 registers): measured fastest for the
// 8-column instance (a 64-register cap spills and is 6% slower).
template <int KP, bool EPI, bool F64>
__global__ void __launch_bounds__(128, 7) k_spmm_sell(SellDev A, int64_t s0, int64_t s1, int q,
                                                   const float2* __restrict__ X, float2* __restrict__ Y, Epi epi) {
  static_assert(KP % 2 == 0 && KP <= 8, "kp must be 2, 4, 6 or 8");
  using V = Ar<F64>;
  constexpr int CPL = KP / 2;
  const int lane = threadIdx.x & 31;
  const int rl = lane >> 1;
  const int off = (lane & 1) * CPL;
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const uint64_t pol = policy_keep();
  for (int64_t s = s0 + gw; s < s1; s += nw) {
    const int row = A.slice_rows[s * kSliceH + rl];
    float2 sum[CPL];
    slice_rowsum<KP, F64>(A, s, rl, off, X, pol, sum);
    if (row < 0) continue;
    const int64_t base = static_cast<int64_t>(row) * KP + off;
    // the first chunk of a row writes, later chunks accumulate, the last applies the epilogue
    const bool first = (A.nchunks == 1) || (A.row_first[row] == q);
    const bool last = !EPI || (A.nchunks == 1) || (A.row_last[row] == q);
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      float2 r = sum[c];
      if (!first) r = V::add(r, Y[base + c]);
      if (EPI && last) {
        if (epi.alpha) r = V::mul(epi.alpha[off + c], r);
        if (epi.beta) r = V::add(r, V::mul(epi.beta[off + c], X[base + c]));
        if (epi.gamma) r = V::add(r, V::mul(epi.gamma[off + c], epi.Z[base + c]));
      }
      Y[base + c] = r;
    }
  }
}

// Product with a short CSR matrix (the n1-row H0_hat): 8 lanes per row (4
// entry segments x 2 column halves), 4 rows per warp.  A segment takes entries
// seg, seg + 4, ... and issues its gathers 4 at a time, so a row of m entries
// costs about m / 16 dependent L2 round trips; in the SELL kernel a lane pair
// walks a whole slice row (about m / 2 of them), which sets the time of a
// product over a few thousand rows.  The segment sums combine by shuffles in a
// fixed order; lane (half, seg) then owns element (row, half * KP/2 + seg).
template <int KP, bool EPI, bool F64>
__device__ __forceinline__ void csr_rows(const CsrDev& A, const float2* __restrict__ X, float2* __restrict__ Y,
                                         const Epi& epi) {
  using V = Ar<F64>;
  constexpr int CPL = KP / 2;
  constexpr int NP = CPL / 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rq = lane >> 3, half = (lane >> 2) & 1, seg = lane & 3;
  const int off = half * CPL;
  const int64_t row = (static_cast<int64_t>(blockIdx.x) * 4 + warp) * 4 + rq;
  const bool valid = row < A.nrows;
  const uint64_t pol = policy_keep();
  typename V::Acc2 pa[NP > 0 ? NP : 1];
#pragma unroll
  for (int c = 0; c < NP; ++c) V::zero(pa[c]);
  typename V::Acc oa;  // odd last column
  V::zero(oa);
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
          gather_half<KP>(X, cc[u], off, xx[u], pol);
        } else {
#pragma unroll
          for (int c = 0; c < CPL; ++c) xx[u][c] = make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int c = 0; c < NP; ++c) V::mac2(pa[c], vv[u], xx[u][2 * c], xx[u][2 * c + 1]);
        if constexpr (CPL % 2 == 1) V::mac(oa, vv[u], xx[u][CPL - 1]);
      }
#pragma unroll
      for (int c = 0; c < NP; ++c) V::norm(pa[c]);
      if constexpr (CPL % 2 == 1) V::norm(oa);
    }
  }
  float2 out[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    float2 v;
    if (c < 2 * NP)
      v = (c & 1) ? V::get1(pa[c / 2]) : V::get0(pa[c / 2]);
    else
      v = V::get(oa);
    v = V::add(v, shfl_xor_df(v, 1));
    v = V::add(v, shfl_xor_df(v, 2));
    out[c] = v;
  }
  if (!valid || seg >= CPL) return;
  float2 r = out[0];
#pragma unroll
  for (int c = 1; c < CPL; ++c)
    if (c == seg) r = out[c];
  const int64_t b = row * KP + off + seg;
  if (EPI) {
    const int j = off + seg;
    if (epi.alpha) r = V::mul(epi.alpha[j], r);
    if (epi.beta) r = V::add(r, V::mul(epi.beta[j], X[b]));
    if (epi.gamma) r = V::add(r, V::mul(epi.gamma[j], epi.Z[b]));
  }
  Y[b] = r;
}

template <int KP, bool EPI, bool F64>
__global__ void __launch_bounds__(128) k_spmm_csr(CsrDev A, const float2* __restrict__ X, float2* __restrict__ Y,
                                                  Epi epi) {
  csr_rows<KP, EPI, F64>(A, X, Y, epi);
}

// Two blocks in one launch (blockIdx.y picks the block): the same rows and sums
// as two k_spmm_csr launches, with twice the warps in flight for these
// latency-bound products.
struct CsrPair {
  const float2* X[2];
  float2* Y[2];
  const float2* Z[2];
};
template <int KP, bool EPI, bool F64>
__global__ void __launch_bounds__(128) k_spmm_csr2(CsrDev A, CsrPair P, Epi epi) {
  const int b = blockIdx.y;
  epi.Z = P.Z[b];
  csr_rows<KP, EPI, F64>(A, P.X[b], P.Y[b], epi);
}

std::atomic<long long> g_launches{0};

// Calls f.template operator()<KP, EPI, F64>() for the run-time column count,
// epilogue and value format.
template <class F>
cudaError_t dispatch_spmm(int kp, bool epi, bool f64, F&& f) {
  auto fmt = [&]<int KP, bool EPI>() {
    if (f64)
      f.template operator()<KP, EPI, true>();
    else
      f.template operator()<KP, EPI, false>();
  };
  switch (kp * 2 + (epi ? 1 : 0)) {
    case 4: fmt.template operator()<2, false>(); break;
    case 5: fmt.template operator()<2, true>(); break;
    case 8: fmt.template operator()<4, false>(); break;
    case 9: fmt.template operator()<4, true>(); break;
    case 12: fmt.template operator()<6, false>(); break;
    case 13: fmt.template operator()<6, true>(); break;
    case 16: fmt.template operator()<8, false>(); break;
    case 17: fmt.template operator()<8, true>(); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

int spmm_default_grid() {
  // computed once (thread-safe static initialisation: handles may solve on several host threads)
  static const int grid = [] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm_sell<8, false, false>, 128, 0);
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
  }();
  return grid;
}

cudaError_t spmm(const SellDev& A, int kp, const float2* X, float2* Y, const Epi& epi, cudaStream_t s) {
  if (A.nslices == 0) return cudaSuccess;
  if (kp == 8 && A.tma && !A.f64) return spmm_tma8(A, X, Y, epi, s);
  const int64_t gmax = spmm_default_grid();
  for (int q = 0; q < A.nchunks; ++q) {
    const int64_t s0 = A.nchunks == 1 ? 0 : A.chunk_slice[q];
    const int64_t s1 = A.nchunks == 1 ? A.nslices : A.chunk_slice[q + 1];
    if (s1 <= s0) continue;
    int64_t grid = (s1 - s0 + 3) / 4;
    if (grid > gmax) grid = gmax;
    const bool has_epi = epi.alpha || epi.beta || epi.gamma;
    const unsigned g = (unsigned)grid;
    const cudaError_t e0 = dispatch_spmm(kp, has_epi, A.f64, [&]<int KP, bool EPI, bool F>() {
      k_spmm_sell<KP, EPI, F><<<g, 128, 0, s>>>(A, s0, s1, q, X, Y, epi);
    });
    if (e0 != cudaSuccess) return e0;
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t spmm_csr2(const CsrDev& A, int kp, const float2* const X[2], float2* const Y[2], const float2* const Z[2],
                      const Epi& epi, cudaStream_t s) {
  if (A.nrows == 0) return cudaSuccess;
  const dim3 g(static_cast<unsigned>((A.nrows + 15) / 16), 2);
  const bool has_epi = epi.alpha || epi.beta || epi.gamma;
  CsrPair P{{X[0], X[1]}, {Y[0], Y[1]}, {Z ? Z[0] : nullptr, Z ? Z[1] : nullptr}};
  const cudaError_t e0 = dispatch_spmm(kp, has_epi, A.f64, [&]<int KP, bool EPI, bool F>() {
    k_spmm_csr2<KP, EPI, F><<<g, 128, 0, s>>>(A, P, epi);
  });
  if (e0 != cudaSuccess) return e0;
  count_launch();
  return cudaGetLastError();
}

cudaError_t spmm_csr(const CsrDev& A, int kp, const float2* X, float2* Y, const Epi& epi, cudaStream_t s) {
  if (A.nrows == 0) return cudaSuccess;
  const unsigned g = static_cast<unsigned>((A.nrows + 15) / 16);
  const bool has_epi = epi.alpha || epi.beta || epi.gamma;
  const cudaError_t e0 = dispatch_spmm(kp, has_epi, A.f64, [&]<int KP, bool EPI, bool F>() {
    k_spmm_csr<KP, EPI, F><<<g, 128, 0, s>>>(A, X, Y, epi);
  });
  if (e0 != cudaSuccess) return e0;
  count_launch();
  return cudaGetLastError();
}

}  // namespace sppc
