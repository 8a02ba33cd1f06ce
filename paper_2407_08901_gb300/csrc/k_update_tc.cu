// Block updates Y = alpha X + [Q_0 ... Q_{na-1}] C against the orthonormal basis
// on the tensor cores (tcgen05), with FP64-grade accuracy from exact integer
// digit products.
//
// The subtractions of block Gram-Schmidt (Eq. blkGS: T = S - Q C) and the
// restart's Q Y are block updates whose contraction runs over the basis columns
// i: Y[r][j] = alpha_j X[r][j] + sum_i Q[r][i] C[i][j].  The basis digits come
// from the tiles k_qcut stored for the Gram products (tc_digits.cuh): an atom
// holds 8 basis columns x 16 rows, rows contiguous, so for this contraction it
// is an MN-major operand (M = rows, K = basis columns).  C (8 na x 8) is cut
// once per CTA into balanced digits with one power of two per column j
// (2^g_j > max_i |C[i][j]|) and laid out as shifted windows, as in the Gram: C's
// digit t of K step ks sits in tile 7 + t, and the window from tile 7 - s holds,
// at level L, C's digit L - s, so the eight MMAs D += Q_s window_s (M = 128 rows,
// N = 80 = (level, column), K = 16 basis columns) of a K step accumulate every
// level L = s + t <= 9 in one tensor-memory region.  A level's sum over at most
// 128 basis columns and 8 digit pairs stays within 2^24, exact in FP32.
//
// Per CTA (one per SM, 384 threads), tiles of 128 rows; per tile the K steps
// (two blocks each) stream through five shared-memory stages: warp 1 copies a
// step's eight 16-row chunks (cp.async.bulk, the two blocks' 4 KB of a chunk
// each), warp 0 issues its eight MMAs into the tile's region (two regions
// alternate between tiles), and two groups of four warps (4-7 for the even
// tiles, 8-11 for the odd ones, so that two tiles' epilogues overlap) read a
// finished tile back (tcgen05.ld, one row per thread), turn each column's level
// sums into one value by integer arithmetic (tc_digits.cuh: an exact 128-bit
// sum, rounded once), add alpha X (when X and alpha are given, as update() does;
// the X row is loaded before the tile's MMAs are waited for) and store Y.  Y may
// alias X (a row is read and written by one thread).  Errors: a
// non-finite coefficient sets bit 0 of *err, a timed-out wait (about a second)
// bit 1; after a time-out the kernel waits (bounded) for its copies and MMAs in
// flight and frees its tensor memory.
#include <cstdint>

#include "tc_digits.cuh"

namespace sppc {

namespace {

using namespace tc;

constexpr int kUThreads = 384;                          // warps: 0 MMA, 1 copies, 4-7 and 8-11 read-back
constexpr int kTileRows = 128;                          // rows per tile: the MMA's M
constexpr int kTileChunks = kTileRows / kTcRows;        // 8 digit chunks per tile
constexpr int kChunkStride = 2 * kBlockChunk;           // a chunk's two blocks of one K step in a stage
constexpr int kStepBytes = kTileChunks * kChunkStride;  // 32 KB
constexpr int kUStages = 5;
constexpr int kCoefTiles = 17;                          // tiles 0-6 and 15-16 zero, 7 + t = digit t
constexpr int kMaxSteps = 8;                            // K steps of a launch (16 blocks)
constexpr int kCoefBytes = kMaxSteps * kCoefTiles * kAtom;
constexpr int kUSmem = kUStages * kStepBytes + kCoefBytes + 1024;  // + alignment slack
constexpr int kUTmemCols = 256;                         // two regions of 128 columns

// MN-major operand (the basis digits of a K step): atoms of 16 rows x 8 basis
// columns; the leading byte offset steps along M (the next 16 rows, 4 KB on in a
// stage), the stride byte offset along K (the next 8 basis columns, the other
// block, 2 KB on).
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t addr) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>(kChunkStride >> 4) << 16) |
         (static_cast<uint64_t>(kBlockChunk >> 4) << 32) | (1ull << 46) | (6ull << 61);
}

// Qd: digits of blocks 0 .. na - 1 (na <= 16) of one group; coef: 8 na x 8 slots,
// row (8 a + i); rowexp: null (blocks cut at 2^61) or the blocks' column
// exponents e (cut at 2^(61 - e)), one per coefficient row, folded into the
// coefficients; xmode 0: no X term, 1: alpha X (alpha: 8 slots), 2: X.
template <bool F64>
__global__ void __launch_bounds__(kUThreads, 1)
    k_update_tc(const unsigned char* __restrict__ Qd, int na, const float2* __restrict__ coef,
                const int* __restrict__ rowexp, const float2* __restrict__ alpha, const float2* X, int xmode,
                float2* Y, int64_t n, int64_t rows_per_cta, int* __restrict__ err) {
  using V = Ar<F64>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kUStages], mma_bar[kUStages], acc_bar[2], free_bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int gexp[8];
  __shared__ int abort_flag, bad_flag;
  __shared__ int armed[kUStages], committed[kUStages];  // [0]: units armed / committed, for the error path
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* ctiles = smem + kUStages * kStepBytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * rows_per_cta;
  const int64_t c1 = min(c0 + rows_per_cta, n);
  const int64_t nck = (c1 - c0 + kTcRows - 1) / kTcRows;   // digit chunks of this CTA
  const int64_t ntiles = (nck + kTileChunks - 1) / kTileChunks;
  const int ksteps = (na + 1) / 2;
  const int64_t nunits = ntiles * ksteps;
  const int64_t gc0 = c0 / kTcRows;
  volatile int* abort = &abort_flag;

  // every stage and coefficient tile starts at zero (stale stage data is then
  // always finite digits, which a missing block meets with zero coefficients)
  for (int i = tid; i < (kUStages * kStepBytes + kCoefBytes) / 16; i += kUThreads)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  if (tid < 8) gexp[tid] = -100000;
  if (tid == 0) {
    for (int st = 0; st < kUStages; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[st])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_bar[st])) : "memory");
      armed[st] = committed[st] = 0;
    }
    for (int r = 0; r < 2; ++r) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_bar[r])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&free_bar[r])) : "memory");
    }
    abort_flag = 0;
    bad_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kUTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  // C's column exponents, then its digits into the window tiles of each K step
  const int ncoef = 64 * na;
  auto row_e = [&](int i) -> int { return rowexp ? (rowexp[i] < -5000 ? 0 : rowexp[i]) : 0; };
  for (int e = tid; e < ncoef; e += kUThreads) {
    const int eb = exp_bound<F64>(coef[e]);
    atomicMax(&gexp[e & 7], eb < -5000 ? eb : eb + row_e(e >> 3));
  }
  __syncthreads();
  {
    bool bad = false;
    for (int e = tid; e < ncoef; e += kUThreads) {
      const int i = e >> 3, j = e & 7, ks = i >> 4, il = i & 15;
      const int g = gexp[j] < -5000 ? 0 : gexp[j];
      uint64_t x;
      bool ng;
      if (!to_fixed<F64>(coef[e], kQShift - g + row_e(i), x, ng)) {
        bad = true;
        x = 0;
      }
      const Digits dg = spread_balanced(x);
      const uint32_t S1 = sign_s(ng, ng), T1 = sign_t(ng, ng);
      uint32_t h[4];
#pragma unroll
      for (int w = 0; w < 4; ++w) h[w] = hfma2(dg.w[w], S1, T1);
      unsigned char* dst = ctiles + (ks * kCoefTiles + 7) * kAtom + atom_off(j, il);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const uint32_t word = h[digit_word(t)];
        *reinterpret_cast<uint16_t*>(dst + t * kAtom) =
            static_cast<uint16_t>(digit_high(t) ? (word >> 16) : (word & 0xFFFFu));
      }
    }
    if (bad) atomicOr(&bad_flag, 1);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 1) {
    // ---- copies: unit u = (tile u / ksteps, K step u % ksteps) into stage u % kUStages
    if (elect_one()) {
      // stage st used for the wraps-th time; unit = (tile, K step ks) (32-bit counters)
      int st = 0, ks = 0, tile = 0, armed_total = 0;
      uint32_t wraps = 0;
      for (int u = 0; u < static_cast<int>(nunits); ++u) {
        if (wraps > 0 && !role_wait(smem_u32(&mma_bar[st]), (wraps - 1) & 1u, abort)) break;
        const int64_t ch0 = static_cast<int64_t>(tile) * kTileChunks;
        const int nch = static_cast<int>(nck - ch0 < kTileChunks ? nck - ch0 : kTileChunks);
        const int nb = na - 2 * ks < 2 ? na - 2 * ks : 2;
        const uint32_t bar = smem_u32(&full_bar[st]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(static_cast<uint32_t>(nch * nb * kBlockChunk))
                     : "memory");
        const uint32_t dst = smem_u32(smem + st * kStepBytes);
        const unsigned char* src = Qd + (gc0 + ch0) * kGroupChunk + 2 * ks * kBlockChunk;
        for (int c = 0; c < nch; ++c)
          bulk_g2s(dst + c * kChunkStride, src + static_cast<int64_t>(c) * kGroupChunk, nb * kBlockChunk, bar);
        ++armed_total;
        if (++st == kUStages) {
          st = 0;
          ++wraps;
        }
        if (++ks == ksteps) {
          ks = 0;
          ++tile;
        }
      }
      armed[0] = armed_total;
    }
    __syncwarp();
  } else if (warp == 0) {
    // ---- MMAs: a unit's eight into its tile's region; a tile's first unit waits
    // until the region's previous tile is read back
    if (elect_one()) {
      const uint32_t idesc = instr_desc(kDCols, true);
      int st = 0, ks = 0, tile = 0, committed_total = 0;
      uint32_t ph = 0;
      for (int u = 0; u < static_cast<int>(nunits); ++u) {
        const int r = tile & 1;
        if (ks == 0 && tile >= 2 &&
            !role_wait(smem_u32(&free_bar[r]), static_cast<uint32_t>((tile >> 1) - 1) & 1u, abort))
          break;
        if (!role_wait(smem_u32(&full_bar[st]), ph, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(smem + st * kStepBytes);
        const uint32_t cb = smem_u32(ctiles + ks * kCoefTiles * kAtom);
#pragma unroll
        for (int s = 0; s < 8; ++s)
          mma_f16(tmem + static_cast<uint32_t>(r * 128), smem_desc_mn(a0 + s * kAtom),
                  smem_desc_sw32(cb + (7 - s) * kAtom, kAtom), idesc, (ks > 0 || s > 0) ? 1u : 0u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&mma_bar[st]))
                     : "memory");
        ++committed_total;
        if (ks == ksteps - 1)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&acc_bar[r]))
                       : "memory");
        if (++st == kUStages) {
          st = 0;
          ph ^= 1u;
        }
        if (++ks == ksteps) {
          ks = 0;
          ++tile;
        }
      }
      committed[0] = committed_total;
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ---- read-back and epilogue: group r = (warp - 4) / 4 takes the tiles of
    // region r, row 32 q + lane of each (tensor-memory lanes 32 q .., q = warp % 4)
    const int q = warp & 3, r = (warp - 4) >> 2;
    const uint32_t taddr = tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(r * 128);
    int g[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) g[j] = gexp[j] < -5000 ? 0 : gexp[j];
    float2 al[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) al[j] = xmode == 1 ? alpha[j] : V::from_d(1.0);
    for (int64_t tile = r; tile < ntiles; tile += 2) {
      const int64_t row = c0 + tile * kTileRows + 32 * q + lane;
      // X's row first: its load flies while the tile's MMAs finish
      float4 xr[4];
      if (xmode && row < c1) {
        const float4* xp = reinterpret_cast<const float4*>(X + row * 8);
#pragma unroll
        for (int h = 0; h < 4; ++h) xr[h] = xp[h];
      }
      if (!role_wait(smem_u32(&acc_bar[r]), static_cast<uint32_t>((tile >> 1) & 1), abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      long long acc[8][4];
#pragma unroll
      for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[j][c] = 0;
      read_levels<0>(taddr, acc);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&free_bar[r]));
      if (row < c1) {
        float2 x[8];
        if (xmode) {
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            x[2 * h] = make_float2(xr[h].x, xr[h].y);
            x[2 * h + 1] = make_float2(xr[h].z, xr[h].w);
          }
        }
        float2 y[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float2 t = levels_to_slot<F64>(acc[j], g[j]);
          if (xmode) t = V::add(V::mul(al[j], x[j]), t);
          y[j] = t;
        }
        float4* yp = reinterpret_cast<float4*>(Y + row * 8);
#pragma unroll
        for (int h = 0; h < 4; ++h) yp[h] = make_float4(y[2 * h].x, y[2 * h].y, y[2 * h + 1].x, y[2 * h + 1].y);
      }
    }
  }
  __syncthreads();
  if (abort_flag) {
    if (tid == 0) {
      for (int st = 0; st < kUStages; ++st) {
        // phases of stage st started: the units u < total with u % kUStages == st
        const int a = armed[0] / kUStages + (st < armed[0] % kUStages ? 1 : 0);
        const int c = committed[0] / kUStages + (st < committed[0] % kUStages ? 1 : 0);
        volatile int never = 0;
        if (a > 0) role_wait(smem_u32(&full_bar[st]), static_cast<uint32_t>((a - 1) & 1), &never);
        never = 0;
        if (c > 0) role_wait(smem_u32(&mma_bar[st]), static_cast<uint32_t>((c - 1) & 1), &never);
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (bad_flag) atomicOr(err, 1);
    if (abort_flag) atomicOr(err, 2);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kUTmemCols) : "memory");
  }
}

}  // namespace

// Rows per CTA: one CTA per SM, multiples of the 128-row tile.
cudaError_t update_tc(const unsigned char* Qd, int nblocks, const float2* coef, const float2* alpha, const float2* X,
                      float2* Y, int64_t n, bool f64, int* err, cudaStream_t s, const int* rowexp) {
  if (nblocks < 0 || nblocks > kMaxBlocks) return cudaErrorInvalidValue;
  if (n <= 0) return cudaSuccess;
  static const int sms = [] {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_update_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUSmem);
    cudaFuncSetAttribute(k_update_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUSmem);
    return c > 0 ? c : 1;
  }();
  int64_t ctas = (n + 4 * kTileRows - 1) / (4 * kTileRows);
  if (ctas > sms) ctas = sms;
  if (ctas < 1) ctas = 1;
  int64_t per = (n + ctas - 1) / ctas;
  per = (per + kTileRows - 1) / kTileRows * kTileRows;
  ctas = (n + per - 1) / per;
  const int64_t gb = qdigits_group_bytes(n);
  if (nblocks == 0) {
    // Y = alpha X (or 0): the CUDA-core update with no blocks does exactly that
    BlockList none;
    return update(Y, X, alpha, none, coef, 8, 0, n, f64, s);
  }
  // groups of at most 16 blocks; later groups add onto Y
  for (int a0 = 0; a0 < nblocks; a0 += 16) {
    const int na = nblocks - a0 < 16 ? nblocks - a0 : 16;
    const float2* x = a0 == 0 ? X : Y;
    const int xmode = a0 == 0 ? (X && alpha ? 1 : 0) : 2;
    const unsigned char* q = Qd + (a0 / 16) * gb;
    const unsigned g = static_cast<unsigned>(ctas);
    const int* re = rowexp ? rowexp + a0 * 8 : nullptr;
    if (f64)
      k_update_tc<true><<<g, kUThreads, kUSmem, s>>>(q, na, coef + a0 * 64, re, alpha, x, xmode, Y, n, per, err);
    else
      k_update_tc<false><<<g, kUThreads, kUSmem, s>>>(q, na, coef + a0 * 64, re, alpha, x, xmode, Y, n, per, err);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sppc
