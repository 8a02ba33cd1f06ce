// Tall-skinny dense kernels on row-major n x kp double-float blocks:
// Gram products A^T B (block Gram-Schmidt Eq. blkGS, CholeskyQR Eq. QR, the
// border of the projected matrix Eq. proj), block updates X - A C (blkGS, the
// recycled H Psi of Eq. HPsip, Ritz vectors), diagonal combinations (right-hand
// side of Eq. exp_seq2) and the Ritz residual norms of Eq. rrn.
//
// Reductions over rows are two-stage and deterministic: each CTA writes its
// partial sums, a finishing kernel adds the partials in a fixed order.  Every
// kernel is instantiated for both slot formats (val.cuh): double-float (F64 =
// false) and native FP64 (F64 = true); the host wrappers take the format.
#include "fp64_fast.cuh"
#include "sppc_internal.h"
#include "val.cuh"

namespace sppc {

namespace {

constexpr int kChunk = 2048;  // rows per CTA in the reductions over long blocks

// The preconditioned residual r / (diag(H) - theta) of the Ritz pass: one
// division per element.  In FP64 a division costs about ten FP64 operations on
// this GPU, which made the elementwise pass DFMA-bound (n x 8 divisions); the
// fast reciprocal (fp64_fast.cuh, within a few ulps) and a product take four.
template <bool F64>
__device__ __forceinline__ float2 precond_div(float2 num, float2 den) {
  if constexpr (F64)
    return d_slot(slot_d(num) * recip64(slot_d(den)));
  else
    return Ar<false>::div(num, den);
}

// Rows per CTA of a reduction over `rows` rows: about eight CTAs per SM (so
// that four resident CTAs of 8 warps run two full waves), in multiples of 32
// rows, between 128 and kChunk.
inline int64_t chunk_rows(int64_t rows) {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  int64_t c = (rows + 8 * sms - 1) / (8 * sms);
  c = (c + 31) / 32 * 32;
  return c < 128 ? 128 : (c > kChunk ? kChunk : c);
}

// One warp per output: lane l adds the partials of chunks l, l+32, ... in order,
// then the 32 lane sums are combined by a fixed butterfly (deterministic).
template <bool F64>
__global__ void k_finish(const float2* __restrict__ partials, int64_t nchunks, int nout, double* __restrict__ out) {
  using A = Ar<F64>;
  const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (o >= nout) return;
  typename A::Acc s;
  A::zero(s);
  for (int64_t c = lane; c < nchunks; c += 32) {
    A::acc(s, partials[c * nout + o]);
    A::norm(s);
  }
  const float2 t = warp_sum<F64>(A::get(s));
  if (lane == 0) out[o] = A::to_d(t);
}

// One CTA = 8 warps and `chunk` rows.  A warp covers 32/KP rows at a time, lane
// (row u, column i) with i = lane % KP: the A block rows are read contiguously
// and the lanes of one row share (broadcast) its B row.  Each lane accumulates
// the KP dots (i, j); lanes with equal i and the 8 warps are then combined.
template <int KP, bool F64>
__global__ void __launch_bounds__(256) k_gram(BlockList A, const float2* __restrict__ B, int64_t r0, int64_t r1,
                                              int64_t chunk, float2* __restrict__ partials) {
  using V = Ar<F64>;
  constexpr int RPW = 32 / KP;   // rows per warp step (KP = 6 leaves 2 lanes idle)
  __shared__ float2 red[8][KP * KP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = lane % KP, u = lane / KP;
  const bool active = u < RPW;
  const int64_t c0 = r0 + static_cast<int64_t>(blockIdx.x) * chunk;
  const int64_t c1 = min(c0 + chunk, r1);
  const int nout = A.n * KP * KP;
  for (int a = 0; a < A.n; ++a) {
    const float2* __restrict__ Aa = A.p[a];
    typename V::Acc acc[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) V::zero(acc[j]);
    int cnt = 0;
    if (active) {
      // two rows per iteration, loads issued before the multiply-adds
      int64_t r = c0 + warp * RPW + u;
      for (; r + 8 * RPW < c1; r += 16 * RPW) {
        const int64_t r2 = r + 8 * RPW;
        const float2 av = Aa[r * KP + i];
        const float2 av2 = Aa[r2 * KP + i];
        float4 b[KP / 2], b2[KP / 2];
        const float4* br = reinterpret_cast<const float4*>(B + r * KP);
        const float4* br2 = reinterpret_cast<const float4*>(B + r2 * KP);
#pragma unroll
        for (int q = 0; q < KP / 2; ++q) {
          b[q] = br[q];
          b2[q] = br2[q];
        }
#pragma unroll
        for (int q = 0; q < KP / 2; ++q) {
          V::mac(acc[2 * q], av, make_float2(b[q].x, b[q].y));
          V::mac(acc[2 * q + 1], av, make_float2(b[q].z, b[q].w));
        }
#pragma unroll
        for (int q = 0; q < KP / 2; ++q) {
          V::mac(acc[2 * q], av2, make_float2(b2[q].x, b2[q].y));
          V::mac(acc[2 * q + 1], av2, make_float2(b2[q].z, b2[q].w));
        }
        if (((++cnt) & 7) == 0) {
#pragma unroll
          for (int j = 0; j < KP; ++j) V::norm(acc[j]);
        }
      }
      if (r < c1) {
        const float2 av = Aa[r * KP + i];
        const float4* br = reinterpret_cast<const float4*>(B + r * KP);
#pragma unroll
        for (int q = 0; q < KP / 2; ++q) {
          const float4 b = br[q];
          V::mac(acc[2 * q], av, make_float2(b.x, b.y));
          V::mac(acc[2 * q + 1], av, make_float2(b.z, b.w));
        }
      }
    }
    // combine the RPW row-lanes of column i inside the warp (fixed order)
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      float2 v = active ? V::get(acc[j]) : make_float2(0.f, 0.f);
      for (int uu = 1; uu < RPW; ++uu) {
        const float2 o = make_float2(__shfl_sync(0xffffffffu, v.x, lane + uu * KP < 32 ? lane + uu * KP : lane),
                                     __shfl_sync(0xffffffffu, v.y, lane + uu * KP < 32 ? lane + uu * KP : lane));
        if (u == 0) v = V::add(v, o);
      }
      if (u == 0 && lane < KP) red[warp][i * KP + j] = v;
    }
    __syncthreads();
    if (threadIdx.x < KP * KP) {
      float2 t = red[0][threadIdx.x];
      for (int w = 1; w < 8; ++w) t = V::add(t, red[w][threadIdx.x]);
      const int ii = threadIdx.x / KP, jj = threadIdx.x % KP;
      partials[static_cast<int64_t>(blockIdx.x) * nout + (a * KP + ii) * KP + jj] = t;
    }
    __syncthreads();
  }
}

// Symmetric Gram A^T A of one n x 8 block (CholeskyQR, Eq. QR): the 36 pairs
// i <= j instead of all 64 products.  Lane (rho, c) = (lane / 4, lane % 4)
// takes row rho of the warp's 8 and holds the row rotated by c, b[k] =
// a[(k + c) mod 8], so that its nine pairs are fixed positions of b: (b[0],
// b[d]) and (b[4], b[4 + d]) for d = 0 .. 3, i.e. (c, c + d) and (c + 4, c + 4 +
// d), and (b[0], b[4]) = (c, c + 4); the four classes c cover the 36 pairs once.
// Lanes of one class are combined by shuffles, the 8 warps in shared memory;
// the CTA writes all 64 entries (mirrored) as its partial.
template <bool F64>
__global__ void __launch_bounds__(256) k_gram_sym8(const float2* __restrict__ A, int64_t r0, int64_t r1,
                                                   int64_t chunk, float2* __restrict__ partials) {
  using V = Ar<F64>;
  __shared__ float2 red[8][4][9];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rho = lane >> 2, c = lane & 3;
  const int64_t c0 = r0 + static_cast<int64_t>(blockIdx.x) * chunk;
  const int64_t c1 = min(c0 + chunk, r1);
  typename V::Acc acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) V::zero(acc[q]);
  int cnt = 0;
  for (int64_t r = c0 + warp * 8 + rho; r < c1; r += 64) {
    float2 b[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) b[k] = A[r * 8 + ((k + c) & 7)];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      V::mac(acc[2 * d], b[0], b[d]);
      V::mac(acc[2 * d + 1], b[4], b[(4 + d) & 7]);
    }
    V::mac(acc[8], b[0], b[4]);
    if (((++cnt) & 7) == 0) {
#pragma unroll
      for (int q = 0; q < 9; ++q) V::norm(acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    float2 v = V::get(acc[q]);
#pragma unroll
    for (int m = 4; m < 32; m <<= 1) v = V::add(v, shfl_xor_df(v, m));
    if (rho == 0) red[warp][c][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < 64) {
    const int i = threadIdx.x >> 3, j = threadIdx.x & 7;
    // the class and slot holding pair (min, max): (cc, cc + dd) with dd = j - i mod 8
    const int lo = i < j ? i : j, hi = i < j ? j : i, dd = hi - lo;
    int cc, q;
    if (dd == 4) {
      cc = lo;
      q = 8;
    } else if (dd < 4) {  // (cc, cc + dd) or (cc + 4, cc + 4 + dd) with cc < 4
      cc = lo & 3;
      q = 2 * dd + (lo >= 4 ? 1 : 0);
    } else {  // hi + (8 - dd) = lo (mod 8): the pair read from hi
      const int e = 8 - dd;
      cc = hi & 3;
      q = 2 * e + (hi >= 4 ? 1 : 0);
    }
    float2 t = red[0][cc][q];
    for (int w = 1; w < 8; ++w) t = V::add(t, red[w][cc][q]);
    partials[static_cast<int64_t>(blockIdx.x) * 64 + threadIdx.x] = t;
  }
}

// TRI: one block and an upper triangular coef (CholeskyQR's R^-1): the products
// with its zero entries (i > j) are skipped, which leaves every sum unchanged.
template <int KP, bool F64, bool TRI = false>
__global__ void __launch_bounds__(256) k_update(float2* Y, const float2* X, const float2* __restrict__ alpha,
                                                BlockList A, const float2* __restrict__ coef, int64_t r0, int64_t r1) {
  using V = Ar<F64>;
  extern __shared__ float2 scoef[];
  const int ncoef = A.n * KP * KP;
  for (int t = threadIdx.x; t < ncoef; t += blockDim.x) scoef[t] = coef[t];
  __shared__ float2 salpha[8];
  if (threadIdx.x < KP) salpha[threadIdx.x] = alpha ? alpha[threadIdx.x] : make_float2(0.f, 0.f);
  __syncthreads();
  const int64_t r = r0 + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= r1) return;
  typename V::Acc acc[KP];
#pragma unroll
  for (int j = 0; j < KP; ++j) V::zero(acc[j]);
  if (X && alpha) {
#pragma unroll
    for (int j = 0; j < KP; ++j) V::set(acc[j], V::mul(salpha[j], X[r * KP + j]));
  }
  for (int a = 0; a < A.n; ++a) {
    const float4* ar = reinterpret_cast<const float4*>(A.p[a] + r * KP);
    float2 av[KP];
#pragma unroll
    for (int q = 0; q < KP / 2; ++q) {
      const float4 t = ar[q];
      av[2 * q] = make_float2(t.x, t.y);
      av[2 * q + 1] = make_float2(t.z, t.w);
    }
    const float2* ca = scoef + a * KP * KP;
#pragma unroll
    for (int i = 0; i < KP; ++i) {
#pragma unroll
      for (int j = 0; j < KP; ++j)
        if (!TRI || i <= j) V::mac(acc[j], av[i], ca[i * KP + j]);
    }
#pragma unroll
    for (int j = 0; j < KP; ++j) V::norm(acc[j]);
  }
#pragma unroll
  for (int j = 0; j < KP; ++j) Y[r * KP + j] = V::get(acc[j]);
}

// Short blocks: one thread per element (row r, column j) instead of per row,
// the same sum in the same order as k_update.
template <int KP, bool F64, bool TRI = false>
__global__ void __launch_bounds__(256) k_update_el(float2* Y, const float2* X, const float2* __restrict__ alpha,
                                                   BlockList A, const float2* __restrict__ coef, int64_t r0,
                                                   int64_t r1) {
  using V = Ar<F64>;
  extern __shared__ float2 scoef[];
  const int ncoef = A.n * KP * KP;
  for (int t = threadIdx.x; t < ncoef; t += blockDim.x) scoef[t] = coef[t];
  __syncthreads();
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t r = r0 + t / KP;
  const int j = static_cast<int>(t % KP);
  if (r >= r1) return;
  typename V::Acc acc;
  V::zero(acc);
  if (X && alpha) V::set(acc, V::mul(alpha[j], X[r * KP + j]));
  for (int a = 0; a < A.n; ++a) {
    const float2* ar = A.p[a] + r * KP;
    const float2* ca = scoef + a * KP * KP + j;
#pragma unroll
    for (int i = 0; i < KP; ++i)
      if (!TRI || i <= j) V::mac(acc, ar[i], ca[i * KP]);
    V::norm(acc);
  }
  __syncwarp();
  Y[r * KP + j] = V::get(acc);
}

template <int KP, bool F64>
__global__ void __launch_bounds__(256) k_combine_diag(float2* Y, const float2* X, const float2* __restrict__ alpha,
                                                      BlockList A, const float2* __restrict__ coef, int64_t r0,
                                                      int64_t r1) {
  using V = Ar<F64>;
  __shared__ float2 sc[kMaxBlocks * 8];
  __shared__ float2 salpha[8];
  for (int t = threadIdx.x; t < A.n * 8; t += blockDim.x) sc[t] = coef[t];
  if (threadIdx.x < KP) salpha[threadIdx.x] = alpha ? alpha[threadIdx.x] : make_float2(0.f, 0.f);
  __syncthreads();
  const int64_t r = r0 + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= r1) return;
  typename V::Acc acc[KP];
#pragma unroll
  for (int j = 0; j < KP; ++j) {
    V::zero(acc[j]);
    if (X && alpha) V::set(acc[j], V::mul(salpha[j], X[r * KP + j]));
  }
  for (int b = 0; b < A.n; ++b) {
    const float2* ab = A.p[b] + r * KP;
#pragma unroll
    for (int j = 0; j < KP; ++j) V::mac(acc[j], sc[b * 8 + j], ab[j]);
  }
#pragma unroll
  for (int j = 0; j < KP; ++j) Y[r * KP + j] = V::get(acc[j]);
}

struct Pairs {
  const float2* a[4];
  const float2* b[4];
};

// NQ pairs: only NQ * KP accumulators live (more resident warps for the
// one-pair calls); rows read as 16-byte vectors.  The same sums in the same
// order for every NQ.
template <int KP, bool F64, int NQ>
__global__ void __launch_bounds__(256) k_coldots(Pairs P, int64_t r0, int64_t r1, int64_t chunk,
                                                 float2* partials) {
  using V = Ar<F64>;
  __shared__ float2 red[8][NQ * KP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = r0 + static_cast<int64_t>(blockIdx.x) * chunk;
  const int64_t c1 = min(c0 + chunk, r1);
  typename V::Acc acc[NQ * KP];
#pragma unroll
  for (int t = 0; t < NQ * KP; ++t) V::zero(acc[t]);
  for (int64_t r = c0 + threadIdx.x; r < c1; r += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float4* ar = reinterpret_cast<const float4*>(P.a[q] + r * KP);
      const float4* br = reinterpret_cast<const float4*>(P.b[q] + r * KP);
#pragma unroll
      for (int h = 0; h < KP / 2; ++h) {
        const float4 x = ar[h], y = br[h];
        V::mac(acc[q * KP + 2 * h], make_float2(x.x, x.y), make_float2(y.x, y.y));
        V::mac(acc[q * KP + 2 * h + 1], make_float2(x.z, x.w), make_float2(y.z, y.w));
      }
    }
  }
  constexpr int nout = NQ * KP;
#pragma unroll
  for (int t = 0; t < nout; ++t) {
    const float2 v = warp_sum<F64>(V::get(acc[t]));
    if (lane == 0) red[warp][t] = v;
  }
  __syncthreads();
  if (threadIdx.x < nout) {
    float2 s = red[0][threadIdx.x];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s = V::add(s, red[w][threadIdx.x]);
    partials[static_cast<int64_t>(blockIdx.x) * nout + threadIdx.x] = s;
  }
}

// Two threads per row, each owning half of the KP columns (halves the
// accumulator registers, so twice the warps fit per SM).
template <int KP, bool F64>
__global__ void __launch_bounds__(256) k_ritz_resid(BlockList Q, BlockList Wb, const float2* __restrict__ Y,
                                                    const float2* __restrict__ theta, int64_t n, float2* partials,
                                                    double* Zout, int64_t ldz, int ncols, float2* Tout,
                                                    const float2* __restrict__ diag, float clamp, float2* Zlead,
                                                    float2* Rlead, int64_t nlead) {
  using V = Ar<F64>;
  constexpr int CH = KP / 2;
  extern __shared__ float2 sy[];
  const int ny = Q.n * KP * KP;
  for (int t = threadIdx.x; t < ny; t += blockDim.x) sy[t] = Y[t];
  __shared__ float2 sth[8];
  __shared__ float2 red[8][8];
  if (threadIdx.x < KP) sth[threadIdx.x] = theta[threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int half = threadIdx.x & 1;
  const int j0 = half * CH;
  typename V::Acc racc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) V::zero(racc[c]);
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * kChunk;
  const int64_t c1 = min(c0 + kChunk, n);
  for (int64_t r = c0 + (threadIdx.x >> 1); r < c1; r += blockDim.x >> 1) {
    typename V::Acc za[CH], ha[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      V::zero(za[c]);
      V::zero(ha[c]);
    }
    for (int a = 0; a < Q.n; ++a) {
      const float4* qa = reinterpret_cast<const float4*>(Q.p[a] + r * KP);
      const float4* wa = reinterpret_cast<const float4*>(Wb.p[a] + r * KP);
      const float2* ya = sy + a * KP * KP + j0;
#pragma unroll
      for (int q = 0; q < KP / 2; ++q) {
        const float4 qv = qa[q], wv = wa[q];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const float2 y0 = ya[(2 * q) * KP + c], y1 = ya[(2 * q + 1) * KP + c];
          V::mac(za[c], make_float2(qv.x, qv.y), y0);
          V::mac(ha[c], make_float2(wv.x, wv.y), y0);
          V::mac(za[c], make_float2(qv.z, qv.w), y1);
          V::mac(ha[c], make_float2(wv.z, wv.w), y1);
        }
      }
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        V::norm(za[c]);
        V::norm(ha[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int j = j0 + c;
      const float2 z = V::get(za[c]);
      const float2 d = V::sub(V::get(ha[c]), V::mul(sth[j], z));
      V::mac(racc[c], d, d);
      if (Zout && j < ncols) Zout[r * ldz + j] = V::to_d(z);
      if (Zlead && r < nlead) {
        Zlead[r * KP + j] = z;
        Rlead[r * KP + j] = d;
      }
      if (Tout) {
        // preconditioned residual d / (H_rr - theta_j), denominator clamped to |.| >= clamp
        float2 t = d;
        if (diag) t = precond_div<F64>(d, V::clamp_den(V::sub(diag[r], sth[j]), clamp));
        Tout[r * KP + j] = t;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    float2 v = V::get(racc[c]);
    // sum over the lanes of equal half (butterfly over the row bits)
#pragma unroll
    for (int m = 2; m < 32; m <<= 1) v = V::add(v, shfl_xor_df(v, m));
    if (lane < 2) red[warp][j0 + c] = v;
  }
  __syncthreads();
  if (threadIdx.x < KP) {
    float2 s = red[0][threadIdx.x];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s = V::add(s, red[w][threadIdx.x]);
    partials[static_cast<int64_t>(blockIdx.x) * KP + threadIdx.x] = s;
  }
}

template <bool F64>
__global__ void k_f64_to_df(const double* __restrict__ X, int64_t ldx, int ncols, float2* __restrict__ Y, int kp,
                            int64_t r0, int64_t r1) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t r = r0 + t / kp;
  const int c = static_cast<int>(t % kp);
  if (r >= r1) return;
  Y[r * kp + c] = (c < ncols) ? Ar<F64>::from_d(X[r * ldx + c]) : make_float2(0.f, 0.f);
}

template <bool F64>
__global__ void k_df_to_f64(const float2* __restrict__ X, int kp, double* __restrict__ Y, int64_t ldy, int ncols,
                            int64_t r0, int64_t r1) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t r = r0 + t / ncols;
  const int c = static_cast<int>(t % ncols);
  if (r >= r1) return;
  Y[r * ldy + c] = Ar<F64>::to_d(X[r * kp + c]);
}

__global__ void k_zero(float2* Y, int64_t count) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < count) Y[t] = make_float2(0.f, 0.f);
}

inline unsigned nblk(int64_t work, int threads) { return static_cast<unsigned>((work + threads - 1) / threads); }

// Calls f.template operator()<KP, F64>() for the run-time column count and format.
template <class F>
cudaError_t dispatch(int kp, bool f64, F&& f) {
  switch (kp * 2 + (f64 ? 1 : 0)) {
    case 4: f.template operator()<2, false>(); break;
    case 5: f.template operator()<2, true>(); break;
    case 8: f.template operator()<4, false>(); break;
    case 9: f.template operator()<4, true>(); break;
    case 12: f.template operator()<6, false>(); break;
    case 13: f.template operator()<6, true>(); break;
    case 16: f.template operator()<8, false>(); break;
    case 17: f.template operator()<8, true>(); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t finish(const float2* partials, int64_t nchunks, int nout, double* out, bool f64, cudaStream_t s) {
  if (f64)
    k_finish<true><<<nblk((int64_t)nout * 32, 256), 256, 0, s>>>(partials, nchunks, nout, out);
  else
    k_finish<false><<<nblk((int64_t)nout * 32, 256), 256, 0, s>>>(partials, nchunks, nout, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t gram(const BlockList& A, const float2* B, int kp, int64_t r0, int64_t r1, double* out,
                 float2* partials, int64_t partial_cap, bool f64, cudaStream_t s) {
  const int nout = A.n * kp * kp;
  if (r1 <= r0 || A.n == 0) {
    return cudaMemsetAsync(out, 0, sizeof(double) * nout, s);
  }
  int64_t chunk = chunk_rows(r1 - r0);
  int64_t nchunks = (r1 - r0 + chunk - 1) / chunk;
  if (nchunks * nout > partial_cap) {  // fall back to the coarse cut if the finer one does not fit
    chunk = kChunk;
    nchunks = (r1 - r0 + chunk - 1) / chunk;
  }
  if (nchunks * nout > partial_cap) return cudaErrorInvalidValue;
  const unsigned g = static_cast<unsigned>(nchunks);
  cudaError_t e = dispatch(kp, f64, [&]<int KP, bool F>() { k_gram<KP, F><<<g, 256, 0, s>>>(A, B, r0, r1, chunk, partials); });
  if (e != cudaSuccess) return e;
  return finish(partials, nchunks, nout, out, f64, s);
}

// A^T A for one n x kp block, the same contract as gram(one block, A); kp = 8
// takes the symmetric kernel (36 pairs), other kp the general one.
cudaError_t gram_sym(const float2* A, int kp, int64_t r0, int64_t r1, double* out, float2* partials,
                     int64_t partial_cap, bool f64, cudaStream_t s) {
  BlockList L;
  L.p[0] = A;
  L.n = 1;
  if (kp != 8) return gram(L, A, kp, r0, r1, out, partials, partial_cap, f64, s);
  if (r1 <= r0) return cudaMemsetAsync(out, 0, sizeof(double) * 64, s);
  int64_t chunk = chunk_rows(r1 - r0);
  int64_t nchunks = (r1 - r0 + chunk - 1) / chunk;
  if (nchunks * 64 > partial_cap) {
    chunk = kChunk;
    nchunks = (r1 - r0 + chunk - 1) / chunk;
  }
  if (nchunks * 64 > partial_cap) return cudaErrorInvalidValue;
  const unsigned g = static_cast<unsigned>(nchunks);
  if (f64)
    k_gram_sym8<true><<<g, 256, 0, s>>>(A, r0, r1, chunk, partials);
  else
    k_gram_sym8<false><<<g, 256, 0, s>>>(A, r0, r1, chunk, partials);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return finish(partials, nchunks, 64, out, f64, s);
}

// The finishing sum of gram() for partial results written by another kernel
// (k_gram_tc.cu): out[o] = sum over c of partials[c * nout + o], fixed order.
cudaError_t gram_finish(const float2* partials, int64_t nchunks, int nout, double* out, bool f64, cudaStream_t s) {
  return finish(partials, nchunks, nout, out, f64, s);
}

namespace {
template <bool F64>
__global__ void k_ritz_precond(const float2* __restrict__ D, const float2* __restrict__ theta,
                               const float2* __restrict__ diag, float clamp, float2* __restrict__ T, int kp,
                               int64_t n) {
  using V = Ar<F64>;
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n * kp) return;
  const int64_t r = e / kp;
  const int j = static_cast<int>(e - r * kp);
  float2 t = D[e];
  if (diag) t = precond_div<F64>(t, V::clamp_den(V::sub(diag[r], theta[j]), clamp));
  T[e] = t;
}
}  // namespace

// The preconditioned residual block of the Ritz pass (the division k_ritz_resid
// applies), from a residual block computed elsewhere.
cudaError_t ritz_precond(const float2* D, const float2* theta, const float2* diag, float clamp, float2* T, int kp,
                         int64_t n, bool f64, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = nblk(n * kp, 256);
  if (f64)
    k_ritz_precond<true><<<g, 256, 0, s>>>(D, theta, diag, clamp, T, kp, n);
  else
    k_ritz_precond<false><<<g, 256, 0, s>>>(D, theta, diag, clamp, T, kp, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t update(float2* Y, const float2* X, const float2* alpha, const BlockList& A, const float2* coef, int kp,
                   int64_t r0, int64_t r1, bool f64, cudaStream_t s) {
  if (r1 <= r0) return cudaSuccess;
  const size_t smem = sizeof(float2) * (size_t)(A.n > 0 ? A.n : 1) * kp * kp;
  if (r1 - r0 < static_cast<int64_t>(kChunk) * 64) {
    // short blocks (the leading block): one thread per element for parallelism
    const unsigned ge = nblk((r1 - r0) * kp, 256);
    return dispatch(kp, f64,
                    [&]<int KP, bool F>() { k_update_el<KP, F><<<ge, 256, smem, s>>>(Y, X, alpha, A, coef, r0, r1); });
  }
  const unsigned g = nblk(r1 - r0, 256);
  return dispatch(kp, f64, [&]<int KP, bool F>() { k_update<KP, F><<<g, 256, smem, s>>>(Y, X, alpha, A, coef, r0, r1); });
}

// Y = A coef for one block A and an upper triangular kp x kp coef (CholeskyQR's
// T R^-1): update() without the products with coef's zero lower entries.
cudaError_t update_tri(float2* Y, const float2* A, const float2* coef, int kp, int64_t r0, int64_t r1, bool f64,
                       cudaStream_t s) {
  if (r1 <= r0) return cudaSuccess;
  BlockList L;
  L.p[0] = A;
  L.n = 1;
  const size_t smem = sizeof(float2) * kp * kp;
  if (r1 - r0 < static_cast<int64_t>(kChunk) * 64) {
    const unsigned ge = nblk((r1 - r0) * kp, 256);
    return dispatch(kp, f64, [&]<int KP, bool F>() {
      k_update_el<KP, F, true><<<ge, 256, smem, s>>>(Y, nullptr, nullptr, L, coef, r0, r1);
    });
  }
  const unsigned g = nblk(r1 - r0, 256);
  return dispatch(kp, f64, [&]<int KP, bool F>() {
    k_update<KP, F, true><<<g, 256, smem, s>>>(Y, nullptr, nullptr, L, coef, r0, r1);
  });
}

cudaError_t combine_diag(float2* Y, const float2* X, const float2* alpha, const BlockList& A, const float2* coef,
                         int kp, int64_t r0, int64_t r1, bool f64, cudaStream_t s) {
  if (r1 <= r0) return cudaSuccess;
  const unsigned g = nblk(r1 - r0, 256);
  return dispatch(kp, f64,
                  [&]<int KP, bool F>() { k_combine_diag<KP, F><<<g, 256, 0, s>>>(Y, X, alpha, A, coef, r0, r1); });
}

cudaError_t coldots(const float2* const* A, const float2* const* B, int nq, int kp, int64_t r0, int64_t r1,
                    double* out, float2* partials, int64_t partial_cap, bool f64, cudaStream_t s) {
  if (nq < 1 || nq > 4) return cudaErrorInvalidValue;
  const int nout = nq * kp;
  if (r1 <= r0) return cudaMemsetAsync(out, 0, sizeof(double) * nout, s);
  Pairs P{};
  for (int q = 0; q < nq; ++q) {
    P.a[q] = A[q];
    P.b[q] = B[q];
  }
  int64_t chunk = chunk_rows(r1 - r0);
  int64_t nchunks = (r1 - r0 + chunk - 1) / chunk;
  if (nchunks * nout > partial_cap) {
    chunk = kChunk;
    nchunks = (r1 - r0 + chunk - 1) / chunk;
  }
  if (nchunks * nout > partial_cap) return cudaErrorInvalidValue;
  const unsigned g = static_cast<unsigned>(nchunks);
  cudaError_t e = dispatch(kp, f64, [&]<int KP, bool F>() {
    switch (nq) {
      case 1: k_coldots<KP, F, 1><<<g, 256, 0, s>>>(P, r0, r1, chunk, partials); break;
      case 2: k_coldots<KP, F, 2><<<g, 256, 0, s>>>(P, r0, r1, chunk, partials); break;
      case 3: k_coldots<KP, F, 3><<<g, 256, 0, s>>>(P, r0, r1, chunk, partials); break;
      default: k_coldots<KP, F, 4><<<g, 256, 0, s>>>(P, r0, r1, chunk, partials); break;
    }
  });
  if (e != cudaSuccess) return e;
  return finish(partials, nchunks, nout, out, f64, s);
}

cudaError_t ritz_resid(const BlockList& Q, const BlockList& Wb, const float2* Y, const float2* theta, int kp,
                       int64_t n, double* out, float2* partials, int64_t partial_cap, double* Zout, int64_t ldz,
                       int ncols, float2* Tout, const float2* diag, float clamp, bool f64, cudaStream_t s,
                       float2* Zlead, float2* Rlead, int64_t nlead) {
  const int64_t nchunks = (n + kChunk - 1) / kChunk;
  if (nchunks * kp > partial_cap) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float2) * (size_t)Q.n * kp * kp;
  const unsigned g = static_cast<unsigned>(nchunks);
  cudaError_t e = dispatch(kp, f64, [&]<int KP, bool F>() {
    k_ritz_resid<KP, F><<<g, 256, smem, s>>>(Q, Wb, Y, theta, n, partials, Zout, ldz, ncols, Tout, diag, clamp, Zlead,
                                             Rlead, nlead);
  });
  if (e != cudaSuccess) return e;
  return finish(partials, nchunks, kp, out, f64, s);
}

cudaError_t f64_to_df(const double* X, int64_t ldx, int ncols, float2* Y, int kp, int64_t r0, int64_t r1, bool f64,
                      cudaStream_t s) {
  if (r1 <= r0) return cudaSuccess;
  if (f64)
    k_f64_to_df<true><<<nblk((r1 - r0) * kp, 256), 256, 0, s>>>(X, ldx, ncols, Y, kp, r0, r1);
  else
    k_f64_to_df<false><<<nblk((r1 - r0) * kp, 256), 256, 0, s>>>(X, ldx, ncols, Y, kp, r0, r1);
  count_launch();
  return cudaGetLastError();
}

cudaError_t df_to_f64(const float2* X, int kp, double* Y, int64_t ldy, int ncols, int64_t r0, int64_t r1, bool f64,
                      cudaStream_t s) {
  if (r1 <= r0 || ncols <= 0) return cudaSuccess;
  if (f64)
    k_df_to_f64<true><<<nblk((r1 - r0) * ncols, 256), 256, 0, s>>>(X, kp, Y, ldy, ncols, r0, r1);
  else
    k_df_to_f64<false><<<nblk((r1 - r0) * ncols, 256), 256, 0, s>>>(X, kp, Y, ldy, ncols, r0, r1);
  count_launch();
  return cudaGetLastError();
}

cudaError_t fill_zero(float2* Y, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_zero<<<nblk(count, 256), 256, 0, s>>>(Y, count); count_launch();
  return cudaGetLastError();
}

}  // namespace sppc
