// SpMM Y = H X in FP32 for the mixed-precision path: values rounded to FP32,
// X rounded to FP32 (the high word of its double-float), products accumulated in
// FP32.  Same SELL-16 layout and column array as the double-float kernel; an
// entry moves 32 bytes of X instead of 64 and 8 bytes of matrix instead of 12.
// (A lane pair per row with 16-byte gathers ran 20% slower on c2: the gather
// request count, not the bytes, sets the pace.)
// The result is written into a double-float block (low word zero) so that the
// double-float kernels downstream read it unchanged.
// BF16 variant: off-diagonal values stored as BF16 (2 bytes per entry, the
// diagonal entries stored as 0), the diagonal kept in FP32 and applied once per
// row in the epilogue of the row's first column tile.
#include "spmm_core.cuh"

namespace sppc {

namespace {

__device__ __forceinline__ float ld_stream_f(const float* p) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

// BF16 bits -> FP32 (exact: BF16 is the upper half of an FP32 word)
__device__ __forceinline__ float ld_stream_bf16(const uint16_t* p) {
  unsigned short v;
  asm volatile("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(v) : "l"(p));
  return __uint_as_float(static_cast<uint32_t>(v) << 16);
}

// One lane per row: the NC (8 or 4) FP32 columns of an X row are one 32- or
// 16-byte gather, and a warp covers two 16-row slices (one per half-warp).  Depth-2 pipeline per lane
// (entries t+1, t+2 in flight while t is accumulated), unrolled by three so the
// buffers rotate without copies.
// MODE 0: FP32 values; 1: BF16 values + FP32 diagonal; 2 and 3: the same with
// the absolute values of the matrix (|H| X, the neighbourhood aggregate of the
// learned proposal).
template <int MODE, int NC>
__global__ void __launch_bounds__(128) k_spmm_sell_f32r(SellDev A, const float* __restrict__ val32,
                                                        const uint16_t* __restrict__ val16,
                                                        const float* __restrict__ diag32, int64_t s0, int64_t s1,
                                                        int q, const float* __restrict__ X,
                                                        float2* __restrict__ Y) {
  constexpr int H = kSliceH;
  const int lane = threadIdx.x & 31;
  const int rl = lane & 15, hw = lane >> 4;
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const uint64_t pol = policy_keep();
  for (int64_t s = s0 + 2 * gw + hw; s < s1 + 1; s += 2 * nw) {
    if (s >= s1) continue;
    const int64_t end = A.slice_ptr[s + 1];
    int64_t e = A.slice_ptr[s] + rl;
    float acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.f;
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), b0 = a0, a1 = a0, b1 = a0, a2 = a0, b2 = a0;
    float v0 = 0.f, v1 = 0.f, v2 = 0.f;
    auto fetch = [&](int64_t ee, float4& a, float4& b, float& v) {
      if (ee < end) {
        const int c = ld_stream(A.col + ee);
        v = (MODE & 1) ? ld_stream_bf16(val16 + ee) : ld_stream_f(val32 + ee);
        if (MODE >= 2) v = fabsf(v);
        const float* p = X + static_cast<int64_t>(c) * NC;
        if constexpr (NC == 8)
          asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
                       : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                       : "l"(p), "l"(pol));
        else
          asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                       : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w)
                       : "l"(p), "l"(pol));
      }
    };
    auto mac = [&](const float4& a, const float4& b, float v) {
      acc[0] = __fmaf_rn(v, a.x, acc[0]); acc[1] = __fmaf_rn(v, a.y, acc[1]);
      acc[2] = __fmaf_rn(v, a.z, acc[2]); acc[3] = __fmaf_rn(v, a.w, acc[3]);
      if constexpr (NC == 8) {
        acc[NC - 4] = __fmaf_rn(v, b.x, acc[NC - 4]); acc[NC - 3] = __fmaf_rn(v, b.y, acc[NC - 3]);
        acc[NC - 2] = __fmaf_rn(v, b.z, acc[NC - 2]); acc[NC - 1] = __fmaf_rn(v, b.w, acc[NC - 1]);
      }
    };
    fetch(e, a0, b0, v0);
    fetch(e + H, a1, b1, v1);
    for (; e < end; e += 3 * H) {
      fetch(e + 2 * H, a2, b2, v2);
      mac(a0, b0, v0);
      if (e + H >= end) break;
      fetch(e + 3 * H, a0, b0, v0);
      mac(a1, b1, v1);
      if (e + 2 * H >= end) break;
      fetch(e + 4 * H, a1, b1, v1);
      mac(a2, b2, v2);
    }
    const int row = A.slice_rows[s * H + rl];
    if (row < 0) continue;
    float2* y = Y + static_cast<int64_t>(row) * NC;
    const bool first = (A.nchunks == 1) || (A.row_first[row] == q);
    if ((MODE & 1) && first) {
      const float d = MODE >= 2 ? fabsf(diag32[row]) : diag32[row];
      const float4 xa = *reinterpret_cast<const float4*>(X + static_cast<int64_t>(row) * NC);
      const float4 xb = NC == 8 ? *reinterpret_cast<const float4*>(X + static_cast<int64_t>(row) * NC + 4) : xa;
      mac(xa, xb, d);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) y[c] = make_float2(first ? acc[c] : __fadd_rn(acc[c], y[c].x), 0.f);
  }
}

// X (double-float, n x 8) -> FP32 (its high words, the correctly rounded FP32 values).
__global__ void k_df_hi(const float2* __restrict__ X, float* __restrict__ X32, int64_t count) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < count) X32[i] = X[i].x;
}

// BF16 copy of the SELL values: entry e of slice s belongs to slice row
// (e - slice_ptr[s]) mod 16; diagonal entries become 0 (applied from diag32).
// The values must already be BF16-exact (their double-float high words).
__global__ void k_make_val16(SellDev A, uint16_t* __restrict__ val16) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t s = t >> 4;
  const int l = static_cast<int>(t & 15);
  if (s >= A.nslices) return;
  const int row = A.slice_rows[s * kSliceH + l];
  for (int64_t e = A.slice_ptr[s] + l; e < A.slice_ptr[s + 1]; e += kSliceH) {
    const bool dg = row >= 0 && A.col[e] == row;
    val16[e] = dg ? 0 : static_cast<uint16_t>(__float_as_uint(A.val[e].x) >> 16);
  }
}

}  // namespace

cudaError_t make_val16(const SellDev& A, uint16_t* val16, cudaStream_t s) {
  if (A.nslices == 0) return cudaSuccess;
  const int64_t threads = A.nslices * kSliceH;
  k_make_val16<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, s>>>(A, val16);
  count_launch();
  return cudaGetLastError();
}

cudaError_t df_hi_parts(const float2* in, float* out, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_df_hi<<<static_cast<unsigned>((count + 255) / 256), 256, 0, s>>>(in, out, count);
  count_launch();
  return cudaGetLastError();
}

namespace {

template <int MODE, int NC>
cudaError_t launch_f32(const SellDev& A, const float* val32, const uint16_t* val16, const float* diag32,
                       const float* X32, float2* Y, cudaStream_t s) {
  static const int gmax = [] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_spmm_sell_f32r<MODE, NC>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm_sell_f32r<MODE, NC>, 128, 0);
    return sms * (per_sm < 1 ? 1 : per_sm);
  }();
  for (int q = 0; q < A.nchunks; ++q) {
    const int64_t c0 = A.nchunks == 1 ? 0 : A.chunk_slice[q];
    const int64_t c1 = A.nchunks == 1 ? A.nslices : A.chunk_slice[q + 1];
    if (c1 <= c0) continue;
    int64_t grid = (c1 - c0 + 7) / 8;  // 4 warps x 2 slices per CTA
    if (grid > gmax) grid = gmax;
    k_spmm_sell_f32r<MODE, NC><<<static_cast<unsigned>(grid), 128, 0, s>>>(A, val32, val16, diag32, c0, c1, q, X32,
                                                                           Y);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t spmm_f32(const SellDev& A, const float* val32, const uint16_t* val16, const float* diag32,
                     const float2* X, float* X32, float2* Y, int kp, cudaStream_t s) {
  if (A.nslices == 0) return cudaSuccess;
  const bool bf = val16 != nullptr;
  if (bf && !diag32) return cudaErrorInvalidValue;
  if (!bf && !val32) return cudaErrorInvalidValue;
  if (kp != 4 && kp != 8) return cudaErrorInvalidValue;
  const int64_t count = A.nrows * kp;
  k_df_hi<<<static_cast<unsigned>((count + 255) / 256), 256, 0, s>>>(X, X32, count);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (kp == 4)
    return bf ? launch_f32<1, 4>(A, val32, val16, diag32, X32, Y, s)
              : launch_f32<0, 4>(A, val32, val16, diag32, X32, Y, s);
  return bf ? launch_f32<1, 8>(A, val32, val16, diag32, X32, Y, s) : launch_f32<0, 8>(A, val32, val16, diag32, X32, Y, s);
}

cudaError_t spmm_abs_f32(const SellDev& A, const float* val32, const uint16_t* val16, const float* diag32,
                         const float* X32, float2* Y, cudaStream_t s) {
  if (A.nslices == 0) return cudaSuccess;
  const bool bf = val16 != nullptr;
  if (bf && !diag32) return cudaErrorInvalidValue;
  if (!bf && !val32) return cudaErrorInvalidValue;
  return bf ? launch_f32<3, 8>(A, val32, val16, diag32, X32, Y, s)
            : launch_f32<2, 8>(A, val32, val16, diag32, X32, Y, s);
}

}  // namespace sppc
