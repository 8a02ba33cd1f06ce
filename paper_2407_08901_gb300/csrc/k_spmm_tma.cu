// SpMM Y = H X over the SELL-16 layout with the X rows gathered by the tensor
// memory accelerator (kp = 8, double-float arithmetic).
//
// The register-gather kernel (k_spmm.cu) keeps one gather per lane pair in
// flight and is bound by gather latency.  Here every warp owns a ring of
// kTmaDepth shared-memory stages.  A stage holds one step of the warp's slice
// (the t-th entry of its 16 rows): the 16 gathered X rows (four
// cp.async.bulk.tensor tile::gather4 copies of four 64-byte rows each), the 16
// values (one 128-byte bulk copy) and the 16 column indices of the step that
// will next refill the stage (one 64-byte bulk copy), all signalled on the
// stage's mbarrier.  The warp consumes stage t, then refills it with step
// t + kTmaDepth using the column indices that arrived with it, so kTmaDepth
// steps (about 10 KB per warp) are in flight without registers to hold them.
// Steps run over the warp's slices as one stream (slice s, s + nw, ...), so the
// pipeline does not drain between slices.
//
// Every lane pair accumulates its row exactly as the register-gather kernel does
// (same entry order, same renormalisation cadence), so the two give identical
// bits.  mbarrier waits are bounded (about a second of clock, or A.spin_limit - 1
// non-blocking polls when that is set); on time-out the kernel raises the
// handle's flag, waits (bounded by the clock) for its own copies in flight and
// returns.  The decision to give up is taken by the whole warp at once.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "spmm_core.cuh"

namespace sppc {

namespace {

constexpr int kTmaWarps = 8;
constexpr int kTmaDepth = 8;
constexpr int kStageBytes = 1280;  // 1024 B of X rows + 128 B values + 64 B columns, padded to 128 B
constexpr int kValOff = 1024;
constexpr int kColOff = 1152;
constexpr int kStageTx = 1024 + 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete; false after ~2^31 clocks.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > (1ll << 31)) return false;
  }
  return true;
}

// The pipeline's wait: with cap > 0 at most cap - 1 non-blocking tests (cap = 1
// gives up at the first wait, which makes the time-out path testable), else
// mbar_wait; the warp gives up together if any lane did.
__device__ __forceinline__ bool mbar_wait_capped(uint32_t bar, uint32_t parity, unsigned cap) {
  bool done;
  if (cap > 0) {
    done = false;
    for (unsigned i = 1; i < cap && !done; ++i) done = mbar_test(bar, parity);
  } else {
    done = mbar_wait(bar, parity);
  }
  return __all_sync(0xffffffffu, done) != 0;
}

// Four rows (rows.x .. rows.w) of the 2-D tensor map, columns from x, into dst.
__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap* tm, int x, int4 rows, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(rows.x), "r"(rows.y), "r"(rows.z), "r"(rows.w), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Position in a warp's stream of steps: slice s (s0 + gw + i*nw), entry offset e
// of the step (a multiple of 16), end of the slice.  Empty slices hold no steps.
struct StepCursor {
  int64_t s = 0, e = 0, end = 0;
  __device__ __forceinline__ bool valid(int64_t s1) const { return s < s1; }
  __device__ __forceinline__ void settle(const int64_t* sp, int64_t s1, int64_t nw) {
    while (s < s1 && e >= end) {
      s += nw;
      if (s < s1) {
        e = sp[s];
        end = sp[s + 1];
      }
    }
  }
  __device__ __forceinline__ void begin(const int64_t* sp, int64_t first, int64_t s1, int64_t nw) {
    s = first;
    if (s < s1) {
      e = sp[s];
      end = sp[s + 1];
    }
    settle(sp, s1, nw);
  }
  __device__ __forceinline__ void next(const int64_t* sp, int64_t s1, int64_t nw) {
    e += kSliceH;
    settle(sp, s1, nw);
  }
};

__global__ void __launch_bounds__(kTmaWarps * 32) k_spmm_tma8(SellDev A, const __grid_constant__ CUtensorMap tmX,
                                                              int64_t s0, int64_t s1, int q,
                                                              const float2* __restrict__ X, float2* __restrict__ Y,
                                                              Epi epi) {
  constexpr int CPL = 4, D = kTmaDepth, H = kSliceH;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[kTmaWarps][D];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rl = lane >> 1, half = lane & 1;
  const int64_t gw = static_cast<int64_t>(blockIdx.x) * kTmaWarps + warp;
  const int64_t nw = static_cast<int64_t>(gridDim.x) * kTmaWarps;
  if (s0 + gw >= s1) return;
  unsigned char* ring = smem + static_cast<size_t>(warp) * D * kStageBytes;
  const uint32_t ring_s = smem_u32(ring);
  const uint32_t bar_s = smem_u32(&bars[warp][0]);
  if (lane < D) mbar_init(bar_s + 8 * lane, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();
  const int64_t* sp = A.slice_ptr;

  // ci: next step to issue; cn: the step kTmaDepth after it, whose column
  // indices travel with ci's stage.
  StepCursor ci, cn;
  ci.begin(sp, s0 + gw, s1, nw);
  cn = ci;
  for (int i = 0; i < D; ++i)
    if (cn.valid(s1)) cn.next(sp, s1, nw);

  auto issue = [&](int j, int4 cols) {
    const uint32_t st = ring_s + j * kStageBytes;
    const uint32_t bar = bar_s + 8 * j;
    const bool more = cn.valid(s1);
    if (lane == 0) mbar_arrive_expect(bar, kStageTx + (more ? 64 : 0));
    __syncwarp();
    if (lane < 4) {
      tma_gather4(st + 256 * lane, &tmX, 0, cols, bar);
    } else if (lane == 4) {
      bulk_g2s(st + kValOff, A.val + ci.e, 128, bar);
    } else if (lane == 5 && more) {
      bulk_g2s(st + kColOff, A.col + cn.e, 64, bar);
    }
    ci.next(sp, s1, nw);
    if (more) cn.next(sp, s1, nw);
  };

  uint32_t issued = 0, used = 0;
  for (int j = 0; j < D && ci.valid(s1); ++j) {
    int4 cols = make_int4(0, 0, 0, 0);
    if (lane < 4) cols = __ldg(reinterpret_cast<const int4*>(A.col + ci.e) + lane);
    issue(j, cols);
    ++issued;
  }

  bool ok = true;
  for (int64_t s = s0 + gw; s < s1 && ok; s += nw) {
    const int64_t end = sp[s + 1];
    float ah[CPL], al[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) ah[c] = al[c] = 0.f;
    int cnt = 0;
    for (int64_t e = sp[s]; e < end; e += H) {
      const int j = static_cast<int>(used % D);
      if (!mbar_wait_capped(bar_s + 8 * j, (used / D) & 1u, A.spin_limit)) {
        ok = false;
        break;
      }
      const unsigned char* stp = ring + j * kStageBytes;
      const float2 v = *reinterpret_cast<const float2*>(stp + kValOff + rl * 8);
      const float4 xa = *reinterpret_cast<const float4*>(stp + rl * 64 + half * 32);
      const float4 xb = *reinterpret_cast<const float4*>(stp + rl * 64 + half * 32 + 16);
      acc_mac(ah[0], al[0], v, make_float2(xa.x, xa.y));
      acc_mac(ah[1], al[1], v, make_float2(xa.z, xa.w));
      acc_mac(ah[2], al[2], v, make_float2(xb.x, xb.y));
      acc_mac(ah[3], al[3], v, make_float2(xb.z, xb.w));
      if (((++cnt) & 15) == 0) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc_norm(ah[c], al[c]);
      }
      // refill the stage with the step kTmaDepth ahead (its columns came with this stage)
      const bool refill = ci.valid(s1);
      int4 cols = make_int4(0, 0, 0, 0);
      if (refill && lane < 4) cols = *reinterpret_cast<const int4*>(stp + kColOff + 16 * lane);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (refill) {
        issue(j, cols);
        ++issued;
      }
      ++used;
    }
    if (!ok) break;
    const int row = A.slice_rows[s * H + rl];
    if (row < 0) continue;
    const int off = half * CPL;
    const int64_t base = static_cast<int64_t>(row) * 8 + off;
    const bool first = (A.nchunks == 1) || (A.row_first[row] == q);
    const bool last = (A.nchunks == 1) || (A.row_last[row] == q);
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      float2 r = acc_get(ah[c], al[c]);
      if (!first) r = df_add(r, Y[base + c]);
      if (!last) {
        Y[base + c] = r;
        continue;
      }
      if (epi.alpha) r = df_mul(epi.alpha[off + c], r);
      if (epi.beta) r = df_add(r, df_mul(epi.beta[off + c], X[base + c]));
      if (epi.gamma) r = df_add(r, df_mul(epi.gamma[off + c], epi.Z[base + c]));
      Y[base + c] = r;
    }
  }
  if (!ok) {
    if (lane == 0 && A.tma_flag) atomicExch(A.tma_flag, 1);
    // copies still in flight target this warp's ring: wait for them (bounded)
    for (uint32_t u = used; u < issued; ++u) mbar_wait(bar_s + 8 * (u % D), (u / D) & 1u);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;
}  // namespace

bool spmm_tma_available() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode != nullptr;
}

cudaError_t spmm_tma_read_timeout(const SellDev& A, int* flag, cudaStream_t s) {
  *flag = 0;
  if (!A.tma_flag) return cudaSuccess;
  return cudaMemcpyAsync(flag, A.tma_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
}

cudaError_t spmm_tma8(const SellDev& A, const float2* X, float2* Y, const Epi& epi, cudaStream_t s) {
  if (A.nslices == 0) return cudaSuccess;
  if (!spmm_tma_available()) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) return cudaErrorMisalignedAddress;
  const size_t smem = static_cast<size_t>(kTmaWarps) * kTmaDepth * kStageBytes;
  // grid limit computed once (thread-safe static initialisation); 0 = setup failed
  static const int g_tma_grid = [smem] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaFuncSetAttribute(k_spmm_tma8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm_tma8, kTmaWarps * 32, smem) != cudaSuccess)
      return 0;
    return per_sm < 1 ? 0 : sms * per_sm;
  }();
  if (g_tma_grid == 0) return cudaErrorInvalidConfiguration;
  // X (nrows x 8 double-float) as a 2-D fp32 tensor of 16 columns; one box is
  // one 64-byte row, four boxes per gather4.
  CUtensorMap tm;
  const cuuint64_t dims[2] = {16, static_cast<cuuint64_t>(A.nrows)};
  const cuuint64_t strides[1] = {64};
  const cuuint32_t box[2] = {16, 1};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = g_encode(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(X), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  for (int q = 0; q < A.nchunks; ++q) {
    const int64_t c0 = A.nchunks == 1 ? 0 : A.chunk_slice[q];
    const int64_t c1 = A.nchunks == 1 ? A.nslices : A.chunk_slice[q + 1];
    if (c1 <= c0) continue;
    int64_t grid = (c1 - c0 + kTmaWarps - 1) / kTmaWarps;
    if (grid > g_tma_grid) grid = g_tma_grid;
    k_spmm_tma8<<<static_cast<unsigned>(grid), kTmaWarps * 32, smem, s>>>(A, tm, c0, c1, q, X, Y, epi);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sppc
