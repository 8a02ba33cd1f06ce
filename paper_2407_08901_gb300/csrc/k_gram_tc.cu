// Gram products Q^T B against the orthonormal basis on the tensor cores
// (tcgen05), with FP64-grade accuracy from exact integer digit products.
//
// The projections of block Gram-Schmidt (Eq. blkGS) and the border of the
// projected matrix (Eq. proj) are Gram products G = A^T B with A = the basis
// blocks [Q_0 ... Q_{na-1}] (n x M, M = 8 na <= 128, entries |a| < 2 because the
// columns are orthonormal) and B one n x 8 block.  Both come as value slots
// (double-float pairs or IEEE doubles).  Scheme (the splitting of Ozaki et al.
// into exact integer products):
//   - a -> sign * X_a, X_a = round(|a| 2^61) < 2^62 (fixed point, one scale for
//     all of A); b in column j -> sign * X_b, X_b = round(|b| 2^(61 - f_j)) with
//     2^f_j > max |b_j| over the CTA's rows;
//   - X = sum_s d_s 256^(7 - s) with bytes d_0 (top) .. d_7, so that
//     a b = sum_{s,t} (+-d_s)(+-c_t) 2^(f_j - 10 - 8 (s + t));
//   - each byte is exact in FP16, each byte product exact in the FP32
//     accumulator, and a sum of 256 of them (< 2^24) exact as well;
//   - levels L = s + t <= 8 are kept: the dropped part of a product is below
//     2^(f_j - 63), against the 2^-53 |a| |b| of one FP64 rounding.
// Per CTA (one per SM, 256 threads, rows [c0, c1)) and per 32-row chunk: the
// threads cut A's and B's values into FP16 digits written to shared memory in
// the canonical K-major no-swizzle layout (8-row x 16-byte core matrices); one
// thread issues, for each byte s of A, D_s (+)= A_s^T [B_0 .. B_{8-s}] (M = 128,
// N = 8 (9 - s) rounded up to 16, two K = 16 steps) into tensor memory and
// commits to the stage's mbarrier.  Two stages alternate, so the digits of one
// chunk are cut while the MMAs of the previous one run.  Every 256 rows the
// accumulators are read back (tcgen05.ld) and added into 64-bit integers, three
// levels to a word (exact); the next MMA overwrites them.  At the end each
// column's words are scaled and added in FP64 and written as the CTA's partial
// result for the fixed-order cross-CTA sum of k_dense.cu.
// Errors: an entry of A with |a| >= 2 (or a non-finite value) sets bit 0 of
// *err, a timed-out wait (about a second) bit 1; after a time-out the kernel
// still waits (bounded) for its committed MMAs and frees its tensor memory.
#include <cstdint>

#include "sppc_internal.h"
#include "val.cuh"

namespace sppc {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcRows = 32;                      // rows (K) per chunk
constexpr int kTcGroupChunks = 8;                // chunks summed in tensor memory before a read-back
constexpr int kATile = 128 * kTcRows * 2;        // one digit plane of A: 128 (M) x 32 (K) FP16
constexpr int kBTile = 64 * kTcRows * 2;         // B: 64 (8 digits x 8 columns) x 32 FP16
constexpr int kStage = 8 * kATile + kBTile;      // 69,632 bytes
constexpr int kTcSmem = 2 * kStage;              // 139,264 bytes: one CTA per SM
constexpr int kTmemCols = 512;
constexpr int kMaxLevel = 8;
constexpr int kAShift = 61;                      // X_a = round(|a| 2^61)
constexpr long long kWaitClocks = 1ll << 31;     // about a second

// N of the MMA for A's digit s (B columns t * 8 + j with s + t <= 8, rounded up
// to a multiple of 16) and its first tensor-memory column.
__host__ __device__ constexpr int tc_n(int s) {
  return (8 * (9 - s < 8 ? 9 - s : 8) + 15) / 16 * 16;
}
__host__ __device__ constexpr int tc_col(int s) { return s == 0 ? 0 : tc_col(s - 1) + tc_n(s - 1); }
static_assert(tc_col(8) <= kTmemCols, "tensor-memory columns");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, k) in a K-major tile of 32 K columns: core
// matrices of 8 rows x 8 elements (16 bytes a row, 128 bytes a core), cores
// adjacent in K 128 bytes apart, 8-row groups 512 bytes apart.
__host__ __device__ constexpr uint32_t kmajor_off(int row, int k) {
  return static_cast<uint32_t>(((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading byte offset
// (cores adjacent in K) 128, stride byte offset (8-row groups) 512, descriptor
// version 1, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>(128 >> 4) << 16) |
         (static_cast<uint64_t>(512 >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), FP16 A
// and B (bits 7-9, 10-12 = 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int n) {
  return (1u << 4) | (static_cast<uint32_t>(n >> 3) << 17) | (static_cast<uint32_t>(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
      "}"
      :
      : "r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ bool mbar_done(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t"
      "}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the completion of the mbarrier phase of the given parity; false
// after about a second.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_done(bar, parity)) {
    if (clock64() - t0 > kWaitClocks) return false;
  }
  return true;
}

// round(|w| 2^shift) for one FP32 word, as a signed 64-bit integer; false if
// |w| 2^shift >= 2^62 or w is not finite.
__device__ __forceinline__ bool f32_fixed(float w, int shift, long long& x) {
  const uint32_t bits = __float_as_uint(w);
  const int ex = static_cast<int>((bits >> 23) & 0xFF);
  if (ex == 0xFF) return false;
  if (ex == 0) {  // zero or subnormal: below any resolution used here
    x = 0;
    return true;
  }
  const uint64_t m = (bits & 0x7FFFFFu) | 0x800000u;
  const int sh = ex - 150 + shift;  // |w| 2^shift = m 2^sh
  uint64_t u;
  if (sh >= 39) return false;
  if (sh >= 0) {
    u = m << sh;
  } else if (sh > -32) {
    u = (m >> -sh) + ((m >> (-sh - 1)) & 1ull);
  } else {
    u = 0;
  }
  x = (bits >> 31) ? -static_cast<long long>(u) : static_cast<long long>(u);
  return true;
}

// A slot value as sign and magnitude round(|v| 2^shift) < 2^62; false if it does
// not fit or is not finite.
template <bool F64>
__device__ __forceinline__ bool to_fixed(float2 v, int shift, uint64_t& x, bool& neg) {
  if constexpr (F64) {
    const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(slot_d(v)));
    neg = (bits >> 63) != 0;
    const int ex = static_cast<int>((bits >> 52) & 0x7FF);
    if (ex == 0x7FF) return false;
    if (ex == 0) {
      x = 0;
      return true;
    }
    const uint64_t m = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = ex - 1075 + shift;  // |v| 2^shift = m 2^sh
    if (sh >= 10) return false;
    if (sh >= 0) {
      x = m << sh;
    } else if (sh > -64) {
      x = (m >> -sh) + ((m >> (-sh - 1)) & 1ull);
    } else {
      x = 0;
    }
    return true;
  } else {
    // hi + lo with |lo| <= ulp(hi) / 2: the signed sum of the two words' integers
    long long xh, xl;
    if (!f32_fixed(v.x, shift, xh) || !f32_fixed(v.y, shift, xl)) return false;
    const long long s = xh + xl;
    neg = s < 0;
    x = static_cast<uint64_t>(neg ? -s : s);
    return x < (1ull << 62);
  }
}

// e with |v| < 2^e (a very negative value for zero)
template <bool F64>
__device__ __forceinline__ int exp_bound(float2 v) {
  if constexpr (F64) {
    const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(slot_d(v)));
    const int ex = static_cast<int>((bits >> 52) & 0x7FF);
    if (ex == 0) return (bits << 1) == 0 ? -100000 : -1022;
    return ex - 1022;
  } else {
    // |hi + lo| < 2^e whenever |hi| < 2^e (|lo| <= ulp(hi) / 2)
    const uint32_t bits = __float_as_uint(v.x);
    const int ex = static_cast<int>((bits >> 23) & 0xFF);
    if (ex == 0) return (bits << 1) == 0 ? -100000 : -126;
    return ex - 126;
  }
}

// The eight FP16 digits of X (bytes d_0 .. d_7) as four words whose halves hold
// 1024 + d: E_hi = (d_3, d_1), O_hi = (d_2, d_0), E_lo = (d_7, d_5), O_lo = (d_6, d_4)
// (low half first).  fma(v, +-1, -+1024) then gives +-d exactly.
struct Digits {
  uint32_t w[4];  // E_hi, O_hi, E_lo, O_lo
};
__device__ __forceinline__ Digits spread(uint64_t x) {
  const uint32_t hi = static_cast<uint32_t>(x >> 32), lo = static_cast<uint32_t>(x);
  Digits d;
  d.w[0] = (hi & 0x00FF00FFu) | 0x64006400u;
  d.w[1] = ((hi >> 8) & 0x00FF00FFu) | 0x64006400u;
  d.w[2] = (lo & 0x00FF00FFu) | 0x64006400u;
  d.w[3] = ((lo >> 8) & 0x00FF00FFu) | 0x64006400u;
  return d;
}

// word and half (1 = high) holding digit s
__host__ __device__ constexpr int digit_word(int s) { return (s < 4 ? 0 : 2) + ((s & 1) ? 0 : 1); }
__host__ __device__ constexpr int digit_high(int s) { return (s & 3) < 2 ? 1 : 0; }

__device__ __forceinline__ uint32_t hfma2(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

// sign factors of a pair of rows: S = (+-1, +-1), T = (-+1024, -+1024) in FP16
__device__ __forceinline__ uint32_t sign_s(bool n0, bool n1) {
  return (n0 ? 0xBC00u : 0x3C00u) | ((n1 ? 0xBC00u : 0x3C00u) << 16);
}
__device__ __forceinline__ uint32_t sign_t(bool n0, bool n1) {
  return (n0 ? 0x6400u : 0xE400u) | ((n1 ? 0x6400u : 0xE400u) << 16);
}

// Waits for this thread's tensor-memory loads; the four registers pass through
// the wait so that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_wait4(uint32_t (&v)[4]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3])::"memory");
}

// Reads back the accumulators of A's digit S for the 32 tensor-memory lanes and
// the four B columns j0 .. j0 + 3 at taddr (= lane base + tc_col(S) + j0) and
// adds them, level L = S + t, into acc[j - j0][L / 3] with weight 256^(2 - L % 3).
template <int S>
__device__ __forceinline__ void read_digit(uint32_t taddr, long long (&acc)[4][3]) {
  constexpr int NT = 9 - S < 8 ? 9 - S : 8;  // B digits t with S + t <= 8
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    uint32_t v[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(taddr + static_cast<uint32_t>(t * 8))
                 : "memory");
    tmem_wait4(v);
    const int L = S + t;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const long long q = static_cast<long long>(__float2int_rn(__uint_as_float(v[e])));
      acc[e][L / 3] += q * (1ll << (8 * (2 - L % 3)));
    }
  }
}

template <bool F64>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_gram_tc(BlockList A, const float2* __restrict__ B, int64_t r0, int64_t r1, int64_t rows_per_cta,
              float2* __restrict__ partials, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int fexp[8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int na = A.n;
  const int M = na * 8;
  const int64_t c0 = r0 + static_cast<int64_t>(blockIdx.x) * rows_per_cta;
  const int64_t c1 = min(c0 + rows_per_cta, r1);
  const uint32_t bar0 = smem_u32(&mbar[0]), bar1 = smem_u32(&mbar[1]);

  // both stages zeroed once: tile rows >= M stay zero
  for (int i = tid; i < 2 * kStage / 16; i += kTcThreads) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  if (tid < 8) fexp[tid] = -100000;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
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
  // B's column exponents over this CTA's rows
  {
    int emax = -100000;
    const int j = tid & 7;
    int64_t r = c0 + (tid >> 3);
    for (; r + 96 < c1; r += 128) {
      const float2 v0 = B[r * 8 + j], v1 = B[(r + 32) * 8 + j], v2 = B[(r + 64) * 8 + j], v3 = B[(r + 96) * 8 + j];
      emax = max(max(emax, max(exp_bound<F64>(v0), exp_bound<F64>(v1))), max(exp_bound<F64>(v2), exp_bound<F64>(v3)));
    }
    for (; r < c1; r += 32) emax = max(emax, exp_bound<F64>(B[r * 8 + j]));
    atomicMax(&fexp[j], emax);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  const uint32_t tmem = tmem_base;
  const int jb = tid & 7;  // this thread's B column
  const int fb_mine = fexp[jb] > -100000 ? fexp[jb] : 0;

  // read-back split: warp w takes tensor-memory lanes 32 (w % 4) .. (A columns)
  // and B columns 4 (w / 4) .. 4 (w / 4) + 3, all digits
  long long acc[4][3];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[e][c] = 0;

  // this thread's A units: blocks a = warp and warp + 8, column ic, rows 8 g .. 8 g + 7
  const int ic = lane & 7, g = lane >> 3;
  const bool u0 = warp < na, u1 = warp + 8 < na;
  const float2* __restrict__ A0 = u0 ? A.p[warp] : nullptr;
  const float2* __restrict__ A1 = u1 ? A.p[warp + 8] : nullptr;
  // values of the chunk being cut; a unit's next-chunk values are loaded as soon
  // as its current ones are converted, so the loads overlap the digit stores
  float2 pa[2][8], pb;
  auto load_unit = [&](int u, int64_t base) {
    const float2* __restrict__ Au = u ? A1 : A0;
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
      const int64_t r = base + g * 8 + rr;
      pa[u][rr] = r < c1 ? Au[r * 8 + ic] : make_float2(0.f, 0.f);
    }
  };
  auto load_b = [&](int64_t base) {
    const int64_t rb = base + (tid >> 3);
    pb = rb < c1 ? B[rb * 8 + jb] : make_float2(0.f, 0.f);
  };

  // bit st of pend: stage st has committed MMAs not yet waited for; bit st of
  // ph: parity of the stage barrier's next phase
  uint32_t pend = 0u, ph = 0u;
  auto wait_stage = [&](int st) -> bool {
    if (!((pend >> st) & 1u)) return true;
    pend &= ~(1u << st);
    const bool okw = mbar_wait_bounded(st ? bar1 : bar0, (ph >> st) & 1u);
    ph ^= 1u << st;
    return okw;
  };

  bool bad = false, timed_out = false;
  int in_group = 0, chunk = 0;
  if (c0 < c1) {
    if (u0) load_unit(0, c0);
    if (u1) load_unit(1, c0);
    load_b(c0);
  }
  for (int64_t base = c0; base < c1; base += kTcRows, ++chunk) {
    const int st = chunk & 1;
    const bool more = base + kTcRows < c1;
    const bool late = !wait_stage(st);
    unsigned char* sA = smem + st * kStage;
    // ---- A: one 16-byte store per digit plane and unit
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 0 ? !u0 : !u1) continue;
      uint64_t x[8];
      bool ng[8];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        if (!to_fixed<F64>(pa[u][rr], kAShift, x[rr], ng[rr])) {
          bad = true;
          x[rr] = 0;
        }
      }
      if (more) load_unit(u, base + kTcRows);
      Digits dg[8];
      uint32_t S2[4], T2[4];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) dg[rr] = spread(x[rr]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        S2[q] = sign_s(ng[2 * q], ng[2 * q + 1]);
        T2[q] = sign_t(ng[2 * q], ng[2 * q + 1]);
      }
      const int a = warp + 8 * u;
      unsigned char* dst = sA + ((a * 4 + g) * 128 + ic * 16);
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int w = digit_word(s);
        const uint32_t sel = digit_high(s) ? 0x7632u : 0x5410u;
        uint4 o;
        o.x = hfma2(__byte_perm(dg[0].w[w], dg[1].w[w], sel), S2[0], T2[0]);
        o.y = hfma2(__byte_perm(dg[2].w[w], dg[3].w[w], sel), S2[1], T2[1]);
        o.z = hfma2(__byte_perm(dg[4].w[w], dg[5].w[w], sel), S2[2], T2[2]);
        o.w = hfma2(__byte_perm(dg[6].w[w], dg[7].w[w], sel), S2[3], T2[3]);
        *reinterpret_cast<uint4*>(dst + s * kATile) = o;
      }
    }
    // ---- B: one value per thread (row tid / 8, column tid % 8), eight 2-byte stores
    {
      uint64_t x;
      bool ng;
      if (!to_fixed<F64>(pb, kAShift - fb_mine, x, ng)) {
        bad = true;
        x = 0;
      }
      if (more) load_b(base + kTcRows);
      const Digits dg = spread(x);
      const uint32_t S1 = sign_s(ng, ng), T1 = sign_t(ng, ng);
      uint32_t h[4];
#pragma unroll
      for (int w = 0; w < 4; ++w) h[w] = hfma2(dg.w[w], S1, T1);
      unsigned char* dst = sA + 8 * kATile + kmajor_off(jb, tid >> 3);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const uint32_t word = h[digit_word(t)];
        *reinterpret_cast<uint16_t*>(dst + t * 512) =
            static_cast<uint16_t>(digit_high(t) ? (word >> 16) : (word & 0xFFFFu));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(late)) {
      timed_out = true;
      break;
    }
    // ---- MMAs of this chunk, committed to the stage's barrier
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sA + 8 * kATile);
#pragma unroll
      for (int s = 0; s < 8; ++s) {
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          mma_f16(tmem + static_cast<uint32_t>(tc_col(s)), smem_desc(a0 + s * kATile + kk * 256),
                  smem_desc(b0 + kk * 256), instr_desc(tc_n(s)), (in_group > 0 || kk > 0) ? 1u : 0u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       st ? bar1 : bar0)
                   : "memory");
    }
    pend |= 1u << st;
    ++in_group;
    if (in_group == kTcGroupChunks || base + kTcRows >= c1) {
      bool late2 = !wait_stage(0);
      late2 |= !wait_stage(1);
      if (__syncthreads_or(late2)) {
        timed_out = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int q = warp & 3;
      if (32 * q < M) {
        const uint32_t tl = tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(4 * (warp >> 2));
        read_digit<0>(tl + tc_col(0), acc);
        read_digit<1>(tl + tc_col(1), acc);
        read_digit<2>(tl + tc_col(2), acc);
        read_digit<3>(tl + tc_col(3), acc);
        read_digit<4>(tl + tc_col(4), acc);
        read_digit<5>(tl + tc_col(5), acc);
        read_digit<6>(tl + tc_col(6), acc);
        read_digit<7>(tl + tc_col(7), acc);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      in_group = 0;
    }
  }
  if (timed_out) {
    // let committed MMAs finish (bounded) before the tensor memory is freed
    wait_stage(0);
    wait_stage(1);
  }
  // A column i = 32 (warp % 4) + lane, B columns 4 (warp / 4) + e: scaled in FP64
  const int i = 32 * (warp & 3) + lane;
  if (i < M) {
    const int nout = M * 8;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = 4 * (warp >> 2) + e;
      const int fj = fexp[j] > -100000 ? fexp[j] : 0;
      double gsum = 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) gsum += ldexp(static_cast<double>(acc[e][c]), fj - 10 - 8 * (3 * c + 2));
      partials[static_cast<int64_t>(blockIdx.x) * nout + i * 8 + j] = Ar<F64>::from_d(gsum);
    }
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(err, 1);
  if (timed_out && tid == 0) atomicOr(err, 2);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace

// Rows per CTA and CTA count of a launch over `rows` rows: one CTA per SM, at
// least 1024 rows a CTA, a multiple of 32 rows, at most 2^22 rows (the 64-bit
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

cudaError_t gram_tc(const BlockList& A, const float2* B, int64_t r0, int64_t r1, double* out, float2* partials,
                    int64_t partial_cap, bool f64, int* err, cudaStream_t s) {
  if (A.n < 0 || A.n > kMaxBlocks) return cudaErrorInvalidValue;
  if (r1 <= r0 || A.n == 0) return cudaMemsetAsync(out, 0, sizeof(double) * A.n * 64, s);
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_gram_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    cudaFuncSetAttribute(k_gram_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    return n > 0 ? n : 1;
  }();
  int64_t per = 0, ctas = 0;
  gram_tc_geometry(r1 - r0, sms, &per, &ctas);
  // groups of at most 16 blocks (M <= 128), each a launch and a finishing sum
  for (int a0 = 0; a0 < A.n; a0 += 16) {
    BlockList G;
    G.n = A.n - a0 < 16 ? A.n - a0 : 16;
    for (int a = 0; a < G.n; ++a) G.p[a] = A.p[a0 + a];
    const int nout = G.n * 64;
    if (ctas * nout > partial_cap) return cudaErrorInvalidValue;
    const unsigned gdim = static_cast<unsigned>(ctas);
    if (f64)
      k_gram_tc<true><<<gdim, kTcThreads, kTcSmem, s>>>(G, B, r0, r1, per, partials, err);
    else
      k_gram_tc<false><<<gdim, kTcThreads, kTcSmem, s>>>(G, B, r0, r1, per, partials, err);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = gram_finish(partials, ctas, nout, out + a0 * 64, f64, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sppc
