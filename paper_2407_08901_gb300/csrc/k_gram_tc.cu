// Gram products Q^T B against the orthonormal basis on the tensor cores
// (tcgen05), with FP64-grade accuracy from exact integer digit products.
//
// The projections of block Gram-Schmidt (Eq. blkGS) and the border of the
// projected matrix (Eq. proj) are Gram products G = A^T B with A = the basis
// blocks [Q_0 ... Q_{na-1}] (n x 8 na, entries |q| < 2 because the columns are
// orthonormal) and B one n x 8 block, both in value slots (double-float pairs or
// IEEE doubles).  Scheme (the splitting of Ozaki et al. into exact integer
// products):
//   - q -> sign * X_q, X_q = round(|q| 2^61) < 2^62 (fixed point, one scale for
//     all of Q); b in column j -> sign * X_b, X_b = round(|b| 2^(61 - f_j)) with
//     2^f_j > max |b_j| over all rows;
//   - X = sum_s d_s 256^(7 - s) with balanced digits d_s in [-128, 127] (the
//     bytes of X + 0x80...80, each minus 128), so that
//     q b = sum_{s,t} (+-d_s)(+-c_t) 2^(f_j - 10 - 8 (s + t));
//   - each digit is exact in FP16 and each digit product (|.| <= 2^14) exact in
//     the FP32 accumulator; the sum over one level L = s + t (at most 8 pairs)
//     and 64 rows stays below 2^23, exact as well;
//   - levels L <= 9 are kept: the dropped part of a product is below
//     2^(f_j - 71), far under the 2^-53 |q| |b| of one FP64 rounding.
//
// All MMAs of a chunk accumulate into one tensor-memory region D (128 lanes =
// basis columns, 80 columns = (level L, B column j)): with C the tile of B's
// digits padded by zero tiles, C[7 + t] = digit t of the chunk's B rows, the
// window of C starting at tile 7 - s holds, at level L, B's digit L - s, so
// D += Q_s^T window_s over the Q digits s gives every level at once.  (An MMA
// into a different region than the previous one costs several hundred cycles
// on this part; consecutive MMAs into one region issue back to back.)
//
// The basis is cut once per block (k_qcut, when a Gram first needs the block):
// its digits are stored as FP16 in exactly the shared-memory order the MMA
// reads.  Per group of 16 blocks and 16-row chunk c, block a's 2 KB lie at
// (c * 16 + a) * 2048: digit plane s at + 256 s, one 32-byte-swizzled 8 x 16
// core-matrix atom (row i = basis column at 32 i, its two 16-byte halves = rows
// 0-7 and 8-15 of the chunk, swapped when i >= 4).  A Gram needs no
// per-element work on Q: per chunk one bulk copy (cp.async.bulk) brings the na
// blocks' 2 KB pieces, another the chunk's 16 x 8 slots of B.  Per CTA (one per
// SM, 384 threads) six stages rotate: the copies of chunks k + 1 .. k + 4 fly
// while 128 threads cut B's values of chunk k (in shared memory) into C and one
// thread issues the chunk's eight MMAs (M = 128, N = 80, K = 16), committed to
// the stage's mbarrier.  With at most 8 blocks (64 basis columns) the A tile's
// upper half is idle, so a second copy of the pieces, shifted by one digit plane,
// fills it: one MMA then takes digit 2p in lanes 0-63 and digit 2p + 1 in lanes
// 64-127 against digit 2p's window (the upper lanes land one level higher and
// are read back as such), four MMAs a chunk instead of eight.  B's column exponents f_j come from a separate pass over
// B (k_colexp).  Every 64 rows D is read back (tcgen05.ld) and added into 64-bit
// integers, three levels to a word (exact).  At the end each column's words are
// scaled and added in FP64 and written as the CTA's partial result for the
// fixed-order cross-CTA sum of k_dense.cu.
// Errors: |q| >= 2 or a non-finite value sets bit 0 of *err, a timed-out wait
// (about a second) bit 1; after a time-out the kernel still waits (bounded) for
// its copies and MMAs in flight and frees its tensor memory.
#include <cstdint>

#include "tc_digits.cuh"

namespace sppc {

namespace {

using namespace tc;

constexpr int kTcThreads = 384;                 // 12 warps: MMA, copies, 4 cutters, 4 read-back
constexpr int kTcGroupChunks = 4;                // chunks summed in tensor memory before a read-back (64 rows)
constexpr int kABytes = kGroupChunk;             // A tiles of a stage
constexpr int kBRaw = kTcRows * 8 * 8;           // B's 16 x 8 slots of a chunk: 1 KB
constexpr int kCTiles = 17;                      // C: tiles 0-6 and 15-16 zero, 7 + t = B's digit t
constexpr int kStageBytes = kABytes + kBRaw + kCTiles * kAtom;  // 38,144
constexpr int kStages = 6;                       // copies run kStages - 2 chunks ahead
constexpr int kTcSmem = kStages * kStageBytes + 1024;   // + alignment slack: one CTA per SM
constexpr int kTmemCols = 256;                  // two D regions of 128 columns
// Stacked mode (na <= 8): a second copy of a chunk's digit pieces, without its
// first plane (block 0's digit 0, never read there), lands at A row group 8 so
// that row group 8 + a reads block a one digit plane further on.
constexpr int kStackCopy = 8 * kBlockChunk;
static_assert(2 * 128 <= kTmemCols, "two accumulator regions");
static_assert(7 + kLevels <= kCTiles, "C windows");

// One basis block (n rows x 8 columns of slots) cut into its digit tiles at
// out (= the group's digits + 2048 a for block a of the group), in fixed point
// 2^61 (colexp null: |v| < 2) or 2^(61 - colexp[i]) per column i (|v| <
// 2^colexp[i], the column exponents of a block of H Q): thread u handles
// chunk u / 16, rows 8 ((u / 8) % 2) .. + 7 of the chunk, column i = u % 8, and
// writes 16 bytes (the half (u / 8) % 2 of atom row i) per digit plane.  Rows
// >= n get zero digits.
template <bool F64>
__global__ void __launch_bounds__(256) k_qcut(const float2* __restrict__ Q, int64_t n, int64_t nchunks,
                                              const int* __restrict__ colexp, unsigned char* __restrict__ out,
                                              int* __restrict__ err) {
  const int64_t u = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (u >= nchunks * 16) return;
  const int64_t c = u >> 4;
  const int kq = static_cast<int>((u >> 3) & 1), i = static_cast<int>(u & 7);
  int shift = kQShift;  // per column: X = round(|v| 2^(61 - e_i)) when |v| < 2^e_i
  if (colexp) shift -= colexp[i] < -5000 ? 0 : colexp[i];
  uint64_t x[8];
  bool ng[8];
  bool bad = false;
#pragma unroll
  for (int rr = 0; rr < 8; ++rr) {
    const int64_t r = c * kTcRows + kq * 8 + rr;
    const float2 v = r < n ? Q[r * 8 + i] : make_float2(0.f, 0.f);
    if (!to_fixed<F64>(v, shift, x[rr], ng[rr])) {
      bad = true;
      x[rr] = 0;
    }
  }
  Digits dg[8];
#pragma unroll
  for (int rr = 0; rr < 8; ++rr) dg[rr] = spread_balanced(x[rr]);
  uint32_t S2[4], T2[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    S2[q] = sign_s(ng[2 * q], ng[2 * q + 1]);
    T2[q] = sign_t(ng[2 * q], ng[2 * q + 1]);
  }
  unsigned char* dst = out + c * kGroupChunk + atom_off(i, kq * 8);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int w = digit_word(s);
    const uint32_t sel = digit_high(s) ? 0x7632u : 0x5410u;
    uint4 o;
    o.x = hfma2(__byte_perm(dg[0].w[w], dg[1].w[w], sel), S2[0], T2[0]);
    o.y = hfma2(__byte_perm(dg[2].w[w], dg[3].w[w], sel), S2[1], T2[1]);
    o.z = hfma2(__byte_perm(dg[4].w[w], dg[5].w[w], sel), S2[2], T2[2]);
    o.w = hfma2(__byte_perm(dg[6].w[w], dg[7].w[w], sel), S2[3], T2[3]);
    *reinterpret_cast<uint4*>(dst + s * kAtom) = o;
  }
  if (bad) atomicOr(err, 1);
}

// Column exponents of B (n x 8 slots): fexp[j] = max over rows of e with
// |b| < 2^e (fexp preset to a very negative value).
template <bool F64>
__global__ void __launch_bounds__(256) k_colexp(const float2* __restrict__ B, int64_t n, int* __restrict__ fexp) {
  __shared__ int red[8];
  if (threadIdx.x < 8) red[threadIdx.x] = -100000;
  __syncthreads();
  int e = -100000;
  const int j = threadIdx.x & 7;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 3);
  int64_t r = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 3) + (threadIdx.x >> 3);
  for (; r + 3 * stride < n; r += 4 * stride) {  // four loads in flight
    const float2 v0 = B[r * 8 + j], v1 = B[(r + stride) * 8 + j], v2 = B[(r + 2 * stride) * 8 + j],
                 v3 = B[(r + 3 * stride) * 8 + j];
    e = max(max(e, max(exp_bound<F64>(v0), exp_bound<F64>(v1))), max(exp_bound<F64>(v2), exp_bound<F64>(v3)));
  }
  for (; r < n; r += stride) e = max(e, exp_bound<F64>(B[r * 8 + j]));
  atomicMax(&red[j], e);
  __syncthreads();
  if (threadIdx.x < 8) atomicMax(&fexp[threadIdx.x], red[threadIdx.x]);
}

// Qd: the digits of a group of 16 blocks (the first na <= 16 used); B: n x 8
// slots; fexp: B's column exponents (k_colexp); rows [0, n), CTA x takes rows
// [x rows_per_cta, ...), rows_per_cta a multiple of 16.  Roles: warp 0 issues
// the MMAs, warp 1 the copies, warps 4-7 cut B's values, warps 8-11 read D back
// (warp 8 + q: tensor-memory lanes 32 q ..); chunk k uses stage k % kStages,
// 64-row group g the D region g % 2.  Handshakes (mbarriers): full (copies
// landed) -> cut (128 cutter arrivals) -> mma (MMAs done: the stage is free
// again) and, per group, acc (its MMAs done) -> free (128 read-back arrivals:
// the region may be overwritten).
template <bool F64>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gram_tc(const unsigned char* __restrict__ Qd, int na, const float2* __restrict__ B,
              const int* __restrict__ fexp, int64_t n, int64_t rows_per_cta, float2* __restrict__ partials,
              int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kStages], cut_bar[kStages], mma_bar[kStages], acc_bar[2], free_bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, bad_flag;
  __shared__ int armed[kStages], committed[kStages];  // [0]: chunks armed / committed, for the error path
  // stages from a 1024-byte boundary (the swizzle atoms need 256-byte alignment)
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int M = na * 8;
  // up to 8 blocks: digits 2p and 2p + 1 share an MMA (A rows 0-63 and 64-127)
  const bool stack = na <= 8;
  const int64_t c0 = static_cast<int64_t>(blockIdx.x) * rows_per_cta;
  const int64_t c1 = min(c0 + rows_per_cta, n);
  const int64_t nck = (c1 - c0 + kTcRows - 1) / kTcRows;
  const int64_t ngroups = (nck + kTcGroupChunks - 1) / kTcGroupChunks;
  const int64_t gc0 = c0 / kTcRows;  // first global chunk
  volatile int* abort = &abort_flag;

  // the zero tiles of C (0-6 and 15-16) in every stage; A rows >= M are never
  // read back, so A needs no clearing
  for (int st = 0; st < kStages; ++st) {
    uint4* z = reinterpret_cast<uint4*>(smem + st * kStageBytes + kABytes + kBRaw);
    for (int i = tid; i < kCTiles * kAtom / 16; i += kTcThreads) {
      const int tile = i / (kAtom / 16);
      if (tile < 7 || tile >= 15) z[i] = make_uint4(0, 0, 0, 0);
    }
  }
  if (tid == 0) {
    for (int st = 0; st < kStages; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[st])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&cut_bar[st])), "r"(8 * kTcRows)
                   : "memory");
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
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  long long acc[8][4];  // read-back warps: A column 32 (warp - 8) + lane, all B columns
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[j][c] = 0;

  if (warp == 1) {
    // ---- copies: chunk k into stage k % kStages once the MMAs of chunk k - kStages are done
    if (elect_one()) {
      // stage st, used for the wraps-th time (32-bit counters stepped per chunk)
      int st = 0, armed_total = 0;
      uint32_t wraps = 0;
      for (int k = 0; k < static_cast<int>(nck); ++k) {
        if (wraps > 0 && !role_wait(smem_u32(&mma_bar[st]), (wraps - 1) & 1u, abort)) break;
        const uint32_t bar = smem_u32(&full_bar[st]);
        const int64_t base = c0 + k * kTcRows;
        const int rows = static_cast<int>(c1 - base < kTcRows ? c1 - base : kTcRows);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(static_cast<uint32_t>((stack ? 2 * na * kBlockChunk - kAtom : na * kBlockChunk) + rows * 64))
                     : "memory");
        const uint32_t dst = smem_u32(smem + st * kStageBytes);
        const unsigned char* src = Qd + (gc0 + k) * kGroupChunk;
        bulk_g2s(dst, src, na * kBlockChunk, bar);
        if (stack) bulk_g2s(dst + kStackCopy, src + kAtom, na * kBlockChunk - kAtom, bar);
        bulk_g2s(dst + kABytes, B + base * 8, rows * 64, bar);
        ++armed_total;
        if (++st == kStages) {
          st = 0;
          ++wraps;
        }
      }
      armed[0] = armed_total;
    }
    __syncwarp();
  } else if (warp == 0) {
    // ---- MMAs: chunk k's eight into its group's region once it is cut (and,
    // for a group's first chunk, once the region's previous group is read back)
    if (elect_one()) {
      const uint32_t idesc = instr_desc(kDCols);
      // stage st and its phase parity, group g and the chunk's place gi in it
      int st = 0, gi = 0, g = 0, committed_total = 0;
      uint32_t ph = 0;
      for (int k = 0; k < static_cast<int>(nck); ++k) {
        const int r = g & 1;
        const bool first = gi == 0;
        if (first && g >= 2 && !role_wait(smem_u32(&free_bar[r]), static_cast<uint32_t>((g >> 1) - 1) & 1u, abort))
          break;
        if (!role_wait(smem_u32(&cut_bar[st]), ph, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(smem + st * kStageBytes), cb = a0 + kABytes + kBRaw;
        if (stack) {
          // digits 2p (rows 0-63 of A) and 2p + 1 (rows 64-127, from the second
          // copy) in one MMA, both against digit 2p's window
#pragma unroll
          for (int p = 0; p < 4; ++p)
            mma_f16(tmem + static_cast<uint32_t>(r * 128), smem_desc_sw32(a0 + 2 * p * kAtom, kBlockChunk),
                    smem_desc_sw32(cb + (7 - 2 * p) * kAtom, kAtom), idesc, (!first || p > 0) ? 1u : 0u);
        } else {
#pragma unroll
          for (int s = 0; s < 8; ++s)
            mma_f16(tmem + static_cast<uint32_t>(r * 128), smem_desc_sw32(a0 + s * kAtom, kBlockChunk),
                    smem_desc_sw32(cb + (7 - s) * kAtom, kAtom), idesc, (!first || s > 0) ? 1u : 0u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&mma_bar[st]))
                     : "memory");
        ++committed_total;
        if (gi == kTcGroupChunks - 1 || k + 1 == static_cast<int>(nck))
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&acc_bar[r]))
                       : "memory");
        if (++st == kStages) {
          st = 0;
          ph ^= 1u;
        }
        if (++gi == kTcGroupChunks) {
          gi = 0;
          ++g;
        }
      }
      committed[0] = committed_total;
    }
    __syncwarp();
  } else if (warp >= 4 && warp < 8) {
    // ---- cutters: value (row ct / 8, column ct % 8) of each chunk into C's tiles 7 .. 14
    const int ct = tid - 128, kr = ct >> 3, jb = ct & 7;
    int fb = fexp[jb];
    if (fb < -5000) fb = 0;  // an all-zero column
    bool bad = false;
    // value of chunk k (stage st) into its C tiles
    auto cut = [&](int k, int st) {
      unsigned char* sg = smem + st * kStageBytes;
      const float2 v = c0 + static_cast<int64_t>(k) * kTcRows + kr < c1
                           ? reinterpret_cast<const float2*>(sg + kABytes)[ct]
                           : make_float2(0.f, 0.f);
      uint64_t x;
      bool ng;
      if (!to_fixed<F64>(v, kQShift - fb, x, ng)) {
        bad = true;
        x = 0;
      }
      const Digits dg = spread_balanced(x);
      const uint32_t S1 = sign_s(ng, ng), T1 = sign_t(ng, ng);
      uint32_t h[4];
#pragma unroll
      for (int w = 0; w < 4; ++w) h[w] = hfma2(dg.w[w], S1, T1);
      unsigned char* dst = sg + kABytes + kBRaw + 7 * kAtom + atom_off(jb, kr);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const uint32_t word = h[digit_word(t)];
        *reinterpret_cast<uint16_t*>(dst + t * kAtom) =
            static_cast<uint16_t>(digit_high(t) ? (word >> 16) : (word & 0xFFFFu));
      }
    };
    int st = 0;
    uint32_t ph = 0;
    for (int k = 0; k < static_cast<int>(nck); ++k) {
      if (!role_wait(smem_u32(&full_bar[st]), ph, abort)) break;
      cut(k, st);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&cut_bar[st]));
      if (++st == kStages) {
        st = 0;
        ph ^= 1u;
      }
    }
    if (bad) atomicOr(&bad_flag, 1);
  } else if (warp >= 8) {
    // ---- read-back: group g's region once its MMAs are done
    const int q = warp - 8;
    const uint32_t taddr = tmem + (static_cast<uint32_t>(32 * q) << 16);
    for (int64_t g = 0; g < ngroups; ++g) {
      const int r = static_cast<int>(g & 1);
      if (!role_wait(smem_u32(&acc_bar[r]), static_cast<uint32_t>((g >> 1) & 1), abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!stack) {
        if (32 * q < M) read_levels<0>(taddr + static_cast<uint32_t>(r * 128), acc);
      } else if (q < 2) {
        if (32 * q < M) read_levels<0>(taddr + static_cast<uint32_t>(r * 128), acc);
      } else {
        // digit 2p + 1 against digit 2p's window: one level up (up to level 10)
        if (32 * (q - 2) < M) read_levels<1>(taddr + static_cast<uint32_t>(r * 128), acc);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&free_bar[r]));
    }
  }
  __syncthreads();
  if (abort_flag) {
    // copies and MMAs in flight end (bounded) before the tensor memory is freed
    // and the CTA leaves
    if (tid == 0) {
      for (int st = 0; st < kStages; ++st) {
        // phases of stage st started: the chunks k < total with k % kStages == st
        const int a = armed[0] / kStages + (st < armed[0] % kStages ? 1 : 0);
        const int c = committed[0] / kStages + (st < committed[0] % kStages ? 1 : 0);
        volatile int never = 0;
        if (a > 0) role_wait(smem_u32(&full_bar[st]), static_cast<uint32_t>((a - 1) & 1), &never);
        never = 0;
        if (c > 0) role_wait(smem_u32(&mma_bar[st]), static_cast<uint32_t>((c - 1) & 1), &never);
      }
    }
    __syncthreads();
  }
  // stacked: lanes 64 + i hold basis column i's odd digits; fold them onto lane i
  long long* fold = reinterpret_cast<long long*>(smem);  // the stages are idle now
  if (stack && warp >= 10) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) fold[((32 * (warp - 10) + lane) * 8 + j) * 4 + c] = acc[j][c];
  }
  __syncthreads();
  if (stack && warp >= 8 && warp < 10) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[j][c] += fold[((32 * (warp - 8) + lane) * 8 + j) * 4 + c];
  }
  // read-back warps: A column i = 32 (warp - 8) + lane, every B column, scaled in FP64
  if (warp >= 8 && !(stack && warp >= 10)) {
    const int i = 32 * (warp - 8) + lane;
    if (i < M) {
      const int nout = M * 8;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int fj = fexp[j];
        if (fj < -5000) fj = 0;
        double gsum = 0.0;
#pragma unroll
        for (int c = 3; c >= 0; --c) gsum += ldexp(static_cast<double>(acc[j][c]), fj - 10 - 8 * (3 * c + 2));
        partials[static_cast<int64_t>(blockIdx.x) * nout + i * 8 + j] = Ar<F64>::from_d(gsum);
      }
    }
  }
  if (tid == 0) {
    if (bad_flag) atomicOr(err, 1);
    if (abort_flag) atomicOr(err, 2);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

int sm_count() {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_gram_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    cudaFuncSetAttribute(k_gram_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    return n > 0 ? n : 1;
  }();
  return sms;
}

}  // namespace

int64_t qdigits_group_bytes(int64_t n) { return (n + kTcRows - 1) / kTcRows * kGroupChunk; }

unsigned char* qdigits_block(unsigned char* Qd, int64_t n, int a) {
  return Qd + (a / 16) * qdigits_group_bytes(n) + (a % 16) * kBlockChunk;
}

cudaError_t qcut(const float2* Q, int64_t n, unsigned char* out, bool f64, int* err, cudaStream_t s,
                 const int* colexp_dev) {
  const int64_t nch = (n + kTcRows - 1) / kTcRows;
  if (nch == 0) return cudaSuccess;
  const unsigned g = static_cast<unsigned>((nch * 16 + 255) / 256);
  if (f64)
    k_qcut<true><<<g, 256, 0, s>>>(Q, n, nch, colexp_dev, out, err);
  else
    k_qcut<false><<<g, 256, 0, s>>>(Q, n, nch, colexp_dev, out, err);
  count_launch();
  return cudaGetLastError();
}

cudaError_t colexp(const float2* B, int64_t n, int* fexp, bool f64, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(fexp, 0x80, sizeof(int) * 8, s);  // below any exponent
  if (e != cudaSuccess || n <= 0) return e;
  int64_t g = (n + 31) / 32;
  if (g > 4 * sm_count()) g = 4 * sm_count();
  if (f64)
    k_colexp<true><<<static_cast<unsigned>(g), 256, 0, s>>>(B, n, fexp);
  else
    k_colexp<false><<<static_cast<unsigned>(g), 256, 0, s>>>(B, n, fexp);
  count_launch();
  return cudaGetLastError();
}

// Rows per CTA and CTA count of a launch over `rows` rows: one CTA per SM, at
// least 1024 rows a CTA, a multiple of 16 rows, at most 2^22 rows (the 64-bit
// level words cannot overflow).
void gram_tc_geometry(int64_t rows, int sms, int64_t* per, int64_t* ctas) {
  int64_t c = (rows + 1023) / 1024;
  if (c > sms) c = sms;
  if (c < 1) c = 1;
  int64_t p = (rows + c - 1) / c;
  p = (p + kTcRows - 1) / kTcRows * kTcRows;
  if (p > (int64_t(1) << 22)) p = int64_t(1) << 22;
  *per = p;
  *ctas = (rows + p - 1) / p;
}

cudaError_t gram_tc(const unsigned char* Qd, int nblocks, const float2* B, int64_t n, double* out, float2* partials,
                    int64_t partial_cap, bool f64, int* err, int* fexp, cudaStream_t s) {
  if (nblocks < 0 || nblocks > kMaxBlocks) return cudaErrorInvalidValue;
  if (n <= 0 || nblocks == 0) return cudaMemsetAsync(out, 0, sizeof(double) * nblocks * 64, s);
  const int sms = sm_count();
  cudaError_t e = colexp(B, n, fexp, f64, s);  // B's column exponents
  if (e != cudaSuccess) return e;
  int64_t per = 0, ctas = 0;
  gram_tc_geometry(n, sms, &per, &ctas);
  const int64_t gb = qdigits_group_bytes(n);
  // groups of at most 16 blocks (M <= 128), each a launch and a finishing sum
  for (int a0 = 0; a0 < nblocks; a0 += 16) {
    const int na = nblocks - a0 < 16 ? nblocks - a0 : 16;
    const int nout = na * 64;
    if (ctas * nout > partial_cap) return cudaErrorInvalidValue;
    const unsigned gdim = static_cast<unsigned>(ctas);
    const unsigned char* q = Qd + (a0 / 16) * gb;
    if (f64)
      k_gram_tc<true><<<gdim, kTcThreads, kTcSmem, s>>>(q, na, B, fexp, n, per, partials, err);
    else
      k_gram_tc<false><<<gdim, kTcThreads, kTcSmem, s>>>(q, na, B, fexp, n, per, partials, err);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = gram_finish(partials, ctas, nout, out + a0 * 64, f64, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sppc
