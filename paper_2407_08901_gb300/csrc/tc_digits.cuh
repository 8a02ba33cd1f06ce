// Shared pieces of the tensor-core kernels (k_gram_tc.cu, k_update_tc.cu):
// the fixed-point digit split of value slots into balanced FP16 digits, the
// 32-byte-swizzled core-matrix atom the basis digits are stored in, tcgen05
// descriptors and instructions, mbarrier waits with a time limit, and the
// read-back of a digit-level accumulator from tensor memory.
//
// Digit scheme (the splitting of Ozaki et al. into exact integer products): a
// value v with |v| < 2^(62 - shift) becomes sign * X, X = round(|v| 2^shift) <
// 2^62, X = sum_s d_s 256^(7 - s) with balanced digits d_s in [-128, 127] (the
// bytes of X + 0x80...80, each minus 128).  Each digit is exact in FP16 and each
// digit product (|.| <= 2^14) exact in an FP32 accumulator.
#pragma once
#include <cstdint>

#include "sppc_internal.h"
#include "val.cuh"

namespace sppc {
namespace tc {

constexpr int kTcRows = 16;                      // basis rows per digit chunk
constexpr int kAtom = 256;                       // one 8 x 16 FP16 tile (a 32-byte-swizzled atom)
constexpr int kBlockChunk = 8 * kAtom;           // one block's digits of one chunk: 8 planes
constexpr int kGroupChunk = 16 * kBlockChunk;    // a 16-block group's digits of one chunk: 32 KB
constexpr int kLevels = 10;                      // digit levels L = s + t kept (0 .. 9)
constexpr int kDCols = 8 * kLevels;              // accumulator columns (L, j): the MMA's N
constexpr int kQShift = 61;                      // basis digits: X_q = round(|q| 2^61)
constexpr long long kWaitClocks = 1ll << 31;     // about a second
static_assert(kDCols % 16 == 0 && kDCols <= 128, "accumulator columns");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row i, k) in a 32-byte-swizzled 8 x 16 FP16 atom:
// rows 32 bytes apart, 16-byte halves k / 8 swapped for rows 4-7 (address bit 4
// XOR bit 7, the 32-byte swizzle pattern; atoms are 256-byte aligned).
__host__ __device__ constexpr uint32_t atom_off(int i, int k) {
  return static_cast<uint32_t>(i * 32 + (((k >> 3) ^ (i >> 2)) & 1) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor (tcgen05) of a K-major operand made of
// 32-byte-swizzled atoms `sbo` bytes apart along M/N: start address, leading
// byte offset 16 (unused by swizzled K-major layouts), stride byte offset,
// descriptor version 1, base offset 0, swizzle mode 6 (32 bytes).
__device__ __forceinline__ uint64_t smem_desc_sw32(uint32_t addr, uint32_t sbo) {
  return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (1ull << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (6ull << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), FP16 A
// and B (bits 7-9, 10-12 = 0), B K-major, A K-major or (a_mn) MN-major (bit 15),
// N >> 3 at bit 17, M = 128 (M >> 4 at bit 24).
__host__ __device__ constexpr uint32_t instr_desc(int n, bool a_mn = false) {
  return (1u << 4) | (a_mn ? (1u << 15) : 0u) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(128 >> 4) << 24);
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
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t"
      "}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
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
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_done(bar, parity)) {
    if (clock64() - t0 > kWaitClocks) return false;
  }
  return true;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// round(|w| 2^shift) for one FP32 word, signed; false if |w| 2^shift >= 2^62 or
// w is not finite.
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
    const uint64_t bits = (static_cast<uint64_t>(__float_as_uint(v.y)) << 32) | __float_as_uint(v.x);
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
    const uint32_t hi = __float_as_uint(v.y);
    const int ex = static_cast<int>((hi >> 20) & 0x7FF);
    if (ex == 0) return ((hi << 1) | __float_as_uint(v.x)) == 0 ? -100000 : -1022;
    return ex - 1022;
  } else {
    // |hi + lo| < 2^e whenever |hi| < 2^e (|lo| <= ulp(hi) / 2)
    const uint32_t bits = __float_as_uint(v.x);
    const int ex = static_cast<int>((bits >> 23) & 0xFF);
    if (ex == 0) return (bits << 1) == 0 ? -100000 : -126;
    return ex - 126;
  }
}

// The eight balanced digits of X as FP16 material: the bytes b_s of
// X + 0x8080808080808080 (d_s = b_s - 128) in four words whose halves hold
// 1024 + b: E_hi = (b_3, b_1), O_hi = (b_2, b_0), E_lo = (b_7, b_5),
// O_lo = (b_6, b_4) (low half first).  fma(v, +-1, -+1152) then gives +-d exactly.
struct Digits {
  uint32_t w[4];  // E_hi, O_hi, E_lo, O_lo
};
__device__ __forceinline__ Digits spread_balanced(uint64_t x) {
  const uint64_t y = x + 0x8080808080808080ull;  // X < 2^62: no carry out of the top byte
  const uint32_t hi = static_cast<uint32_t>(y >> 32), lo = static_cast<uint32_t>(y);
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

// sign factors of a pair of values: S = (+-1, +-1), T = (-+1152, -+1152) in FP16
__device__ __forceinline__ uint32_t sign_s(bool n0, bool n1) {
  return (n0 ? 0xBC00u : 0x3C00u) | ((n1 ? 0xBC00u : 0x3C00u) << 16);
}
__device__ __forceinline__ uint32_t sign_t(bool n0, bool n1) {
  return (n0 ? 0x6480u : 0xE480u) | ((n1 ? 0x6480u : 0xE480u) << 16);
}


// Waits for this thread's tensor-memory loads; the eight registers pass through
// the wait so that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_wait8(uint32_t (&v)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7])::"memory");
}

// Reads back D (one region) for the warp's 32 tensor-memory lanes at taddr, all
// eight B columns and every level L, adding level L + UP into acc[j][(L + UP) / 3]
// with weight 256^(2 - (L + UP) % 3) (UP = 1: lanes whose digits sit one level
// higher than the columns' index says).
template <int UP>
__device__ __forceinline__ void read_levels(uint32_t taddr, long long (&acc)[8][4]) {
#pragma unroll
  for (int L = 0; L < kLevels; ++L) {
    uint32_t v[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr + static_cast<uint32_t>(8 * L))
                 : "memory");
    tmem_wait8(v);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long q = static_cast<long long>(__float2int_rn(__uint_as_float(v[j])));
      acc[j][(L + UP) / 3] += q * (1ll << (8 * (2 - (L + UP) % 3)));
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// A role's wait for the mbarrier phase of the given parity: false when another
// role has given up (*abort set) or after about a second (then sets *abort).
__device__ __forceinline__ bool role_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_done(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > kWaitClocks) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ bool elect_one() {
  uint32_t leader;
  asm volatile("{\n\t.reg .pred P;\n\telect.sync _|P, 0xffffffff;\n\tselp.u32 %0, 1, 0, P;\n\t}" : "=r"(leader));
  return leader != 0;
}

// The level words' exact sum W = w0 2^72 + w1 2^48 + w2 2^24 + w3 (|w_c| <
// 2^41) as its sign and magnitude left-aligned in 128 bits: V = |W| 2^lz with
// bit 127 set (lz = leading zeros of |W|), in two 64-bit halves.  Integer
// operations with selects instead of branches, so that the eight outputs of a
// thread interleave.  Returns false for W = 0.
__device__ __forceinline__ bool words_aligned(const long long (&w)[4], uint64_t& vh, uint64_t& vl, int& msb,
                                              bool& neg) {
  // two's-complement 128-bit sum of the shifted words
  uint64_t lo = static_cast<uint64_t>(w[3]), hi = static_cast<uint64_t>(w[3] >> 63);
  auto add = [&](uint64_t l2, uint64_t h2) {
    const uint64_t nl = lo + l2;
    hi = hi + h2 + (nl < lo ? 1ull : 0ull);
    lo = nl;
  };
  add(static_cast<uint64_t>(w[2]) << 24, static_cast<uint64_t>(w[2] >> 40));
  add(static_cast<uint64_t>(w[1]) << 48, static_cast<uint64_t>(w[1] >> 16));
  hi += static_cast<uint64_t>(w[0]) << 8;
  neg = static_cast<long long>(hi) < 0;
  const uint64_t nlo = ~lo + 1ull, nhi = ~hi + (nlo == 0 ? 1ull : 0ull);
  const uint64_t ul = neg ? nlo : lo, uh = neg ? nhi : hi;
  if ((ul | uh) == 0) return false;
  const int lz = uh ? __clzll(static_cast<long long>(uh)) : 64 + __clzll(static_cast<long long>(ul));
  const int sa = lz & 63;                       // shift within the word
  const uint64_t a_hi = sa ? (uh << sa) | (ul >> (64 - sa)) : uh, a_lo = ul << sa;
  vh = lz >= 64 ? (ul << sa) : a_hi;
  vl = lz >= 64 ? 0ull : a_lo;
  msb = 127 - lz;
  return true;
}

// The nearest double (ties to even) of W 2^e2, W the level words' sum; results
// below the normal range are flushed to zero (they lie far under the values
// the kernels meet).
__device__ __forceinline__ double words_to_double(const long long (&w)[4], int e2) {
  uint64_t vh, vl;
  int msb;
  bool neg;
  if (!words_aligned(w, vh, vl, msb, neg)) return 0.0;
  uint64_t mant = vh >> 11;                     // 53 bits, leading one at bit 52
  const uint64_t rnd = (vh >> 10) & 1ull;
  const uint64_t sticky = ((vh & 0x3FFull) | vl) != 0 ? 1ull : 0ull;
  mant += rnd & (sticky | (mant & 1ull));
  const bool carry = (mant >> 53) != 0;
  mant = carry ? mant >> 1 : mant;
  const int ex = msb + (carry ? 1 : 0) + e2;   // value = 1.mant * 2^ex
  if (ex < -1022) return 0.0;
  const uint64_t bits = (neg ? (1ull << 63) : 0ull) | (static_cast<uint64_t>(ex + 1023) << 52) |
                        (mant & ((1ull << 52) - 1));
  return __longlong_as_double(static_cast<long long>(bits));
}

// The double-float pair of W 2^e2: the top 24 bits and the next 24, both
// truncated, as FP32 bit patterns, then renormalised by an exact fast two-sum.
__device__ __forceinline__ float2 words_to_df(const long long (&w)[4], int e2) {
  uint64_t vh, vl;
  int msb;
  bool neg;
  if (!words_aligned(w, vh, vl, msb, neg)) return make_float2(0.f, 0.f);
  const uint32_t sgn = neg ? 0x80000000u : 0u;
  auto word = [&](uint32_t m, int top) -> float {  // 24-bit chunk m whose bit 23 sits at bit `top`
    if (m == 0) return 0.f;
    const int lead = 31 - __clz(static_cast<int>(m));
    const int ex = top - (23 - lead) + e2;
    if (ex < -126) return 0.f;
    if (ex > 127) return __uint_as_float(sgn | 0x7F800000u);
    return __uint_as_float(sgn | (static_cast<uint32_t>(ex + 127) << 23) | ((m << (23 - lead)) & 0x7FFFFFu));
  };
  const float hi = word(static_cast<uint32_t>(vh >> 40), msb);
  const float lo = word(static_cast<uint32_t>(vh >> 16) & 0xFFFFFFu, msb - 24);
  const float sum = __fadd_rn(hi, lo);
  return make_float2(sum, __fsub_rn(lo, __fsub_rn(sum, hi)));
}

// The FP64 value of D's level words for one output: acc[c] holds levels 3c ..
// 3c + 2 with weight 256^(2 - L % 3), so the exact sum is W = sum_c acc[c]
// 2^(24 (3 - c)) times 2^(scale - 98), scale = the column's exponent g.
template <bool F64>
__device__ __forceinline__ float2 levels_to_slot(const long long (&w)[4], int scale) {
  if constexpr (F64)
    return d_slot(words_to_double(w, scale - 98));
  else
    return words_to_df(w, scale - 98);
}

}  // namespace tc
}  // namespace sppc
