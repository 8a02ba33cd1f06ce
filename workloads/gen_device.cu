// Device form of the seeded synthetic Hamiltonian generator (input module; holds
// none of the eigensolver's arithmetic).
//
// It builds, in GPU memory, the same matrix as gen.cpp, bit for bit: the same
// law (H_ii = 10 N(i) + U(-2, 2); each row draws d columns uniformly with
// replacement over the rows within two levels, j != i, each draw mirrored,
// values Normal(0, sigma^2)), the same counter-based SplitMix64 numbers, the
// same Box-Muller normals from the same series for log and cos, evaluated with
// explicitly rounded IEEE operations (no contraction) in the host's order, and
// the same canonical order for summing repeated (i, j) pairs (by column, then
// by drawing row and draw index).  A matrix of 5e9 entries, whose host CSR would
// be 60 GB, is produced in a few seconds without touching the host.
//
// Steps: (1) every draw's column and value (one thread per draw); (2) counts of
// mirrored draws per target row and their offsets (scan); (3) the list of
// mirrored draws per row; (4) per row (one warp): the row's own draws, its
// diagonal and its mirrored draws in shared memory, bitonic-sorted by
// (column << 34 | draw index), repeated columns summed left to right: first
// counted (row pointers), then written.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <vector>

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;
constexpr uint64_t kDiagKey = (1ULL << 34) - 1;
constexpr int kMaxLevels = 32;

struct Levels {
  int64_t off[kMaxLevels + 1];
  int n_levels;
};

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t sm64_at(uint64_t seed, uint64_t n) { return mix64(seed + (n + 1) * kGolden); }
__device__ __forceinline__ uint64_t ctr(uint64_t stream, uint64_t idx) { return (stream << 60) | idx; }
__device__ __forceinline__ double u01_closed_open(uint64_t r) { return __dmul_rn((double)(r >> 11), 0x1.0p-53); }
__device__ __forceinline__ double u01_open_closed(uint64_t r) { return __dmul_rn((double)((r >> 11) + 1), 0x1.0p-53); }

// ln(x), x > 0: the atanh series of gen.cpp, operation for operation.
__device__ double portable_log(double x) {
  int e = 0;
  double m = frexp(x, &e);
  if (m < 0.70710678118654752440) {
    m = __dmul_rn(m, 2.0);
    e -= 1;
  }
  const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double s2 = __dmul_rn(s, s);
  double term = s, sum = 0.0;
  for (int k = 1; k <= 41; k += 2) {
    sum = __dadd_rn(sum, __ddiv_rn(term, (double)k));
    term = __dmul_rn(term, s2);
  }
  const double ln2 = 0.69314718055994530942;
  return __dadd_rn(__dmul_rn(2.0, sum), __dmul_rn((double)e, ln2));
}

__device__ void sincos_half_quadrant(double g, double* s_out, double* c_out) {
  const double half_pi = 1.57079632679489661923;
  const double a = __dmul_rn(g, half_pi);
  const double a2 = __dmul_rn(a, a);
  const double na2 = -a2;
  double ts = a, tc = 1.0, s = 0.0, c = 0.0;
  for (int k = 0; k < 14; ++k) {
    s = __dadd_rn(s, ts);
    c = __dadd_rn(c, tc);
    ts = __ddiv_rn(__dmul_rn(ts, na2), (double)((2 * k + 2) * (2 * k + 3)));
    tc = __ddiv_rn(__dmul_rn(tc, na2), (double)((2 * k + 1) * (2 * k + 2)));
  }
  *s_out = s;
  *c_out = c;
}

__device__ double portable_cos_2pi(double u) {
  const double t = __dmul_rn(4.0, u);
  int q = __double2int_rz(t);
  if (q > 3) q = 3;
  const double f = __dsub_rn(t, (double)q);
  double s, c;
  if (f <= 0.5) {
    sincos_half_quadrant(f, &s, &c);
  } else {
    double s2, c2;
    sincos_half_quadrant(__dsub_rn(1.0, f), &s2, &c2);
    s = c2;
    c = s2;
  }
  switch (q) {
    case 0: return c;
    case 1: return -s;
    case 2: return -c;
    default: return s;
  }
}

__device__ __forceinline__ int level_of(const Levels& L, int64_t i) {
  int a = 0;
  while (a + 1 < L.n_levels && L.off[a + 1] <= i) ++a;
  return a;
}

// (1) column and value of every draw; counts of mirrored draws per target row
__global__ void k_draws(Levels L, int64_t n, int64_t d, double sigma, uint64_t seed, int32_t* __restrict__ dcol,
                        double* __restrict__ dval, unsigned* __restrict__ cnt) {
  const int64_t total = n * d;
  for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = idx / d;
    const int a = level_of(L, i);
    const int64_t lo = L.off[max(a - 2, 0)];
    const int64_t hi = L.off[min(a + 2, L.n_levels - 1) + 1];
    const uint64_t w = static_cast<uint64_t>(hi - lo - 1);
    int64_t j = i;
    if (w > 0) {
      const uint64_t r = sm64_at(seed, ctr(0, static_cast<uint64_t>(idx)));
      const uint64_t pick = __umul64hi(r, w);
      j = lo + static_cast<int64_t>(pick);
      if (j >= i) ++j;
    }
    const double u1 = u01_open_closed(sm64_at(seed, ctr(1, static_cast<uint64_t>(idx))));
    const double u2 = u01_closed_open(sm64_at(seed, ctr(2, static_cast<uint64_t>(idx))));
    const double g = __dmul_rn(__dsqrt_rn(__dmul_rn(-2.0, portable_log(u1))), portable_cos_2pi(u2));
    dcol[idx] = static_cast<int32_t>(j);
    dval[idx] = (w > 0) ? __dmul_rn(sigma, g) : 0.0;
    atomicAdd(cnt + j, 1u);
  }
}

// Exclusive scan of n unsigned counts into int64 offsets (out has n + 1 entries):
// per-block sums, a scan of the block sums on one block, then the fix-up.
constexpr int kScanThreads = 1024;
__global__ void k_block_sums(const unsigned* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
  __shared__ int64_t red[kScanThreads / 32];
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kScanThreads + threadIdx.x;
  int64_t v = i < n ? in[i] : 0;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t s = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) s += red[w];
    sums[blockIdx.x] = s;
  }
}
__global__ void k_scan_sums(int64_t* sums, int64_t nb) {
  if (threadIdx.x == 0) {
    int64_t s = 0;
    for (int64_t b = 0; b < nb; ++b) {
      const int64_t v = sums[b];
      sums[b] = s;
      s += v;
    }
    sums[nb] = s;
  }
}
__global__ void k_block_scan(const unsigned* __restrict__ in, int64_t n, const int64_t* __restrict__ sums,
                             int64_t* __restrict__ out) {
  __shared__ int64_t wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kScanThreads + threadIdx.x;
  const int64_t v = i < n ? in[i] : 0;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < kScanThreads / 32 ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) wsum[lane] = w;
  }
  __syncthreads();
  const int64_t before = (warp > 0 ? wsum[warp - 1] : 0) + sums[blockIdx.x];
  if (i < n) out[i] = before + x - v;
  if (i == n - 1) out[n] = before + x;
}

// (3) the mirrored draws of every row (arrival order is irrelevant: rows are sorted)
__global__ void k_mirror(int64_t total, const int32_t* __restrict__ dcol, const int64_t* __restrict__ inptr,
                         unsigned* __restrict__ fill, uint32_t* __restrict__ inlist) {
  for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t j = dcol[idx];
    const unsigned pos = atomicAdd(fill + j, 1u);
    inlist[inptr[j] + pos] = static_cast<uint32_t>(idx);
  }
}

__global__ void k_max_len(const int64_t* __restrict__ inptr, int64_t n, unsigned* out) {
  unsigned m = 0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    m = max(m, static_cast<unsigned>(inptr[i + 1] - inptr[i]));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// (4) one warp per row: gather, sort, merge.  write = false: uniq[i] = distinct
// columns of row i; write = true: the row's CSR entries at rp[i].
__global__ void k_rows(Levels L, int64_t n, int64_t d, uint64_t seed, const int32_t* __restrict__ dcol,
                       const double* __restrict__ dval, const int64_t* __restrict__ inptr,
                       const uint32_t* __restrict__ inlist, int lp, bool write, unsigned* __restrict__ uniq,
                       const int64_t* __restrict__ rp, int32_t* __restrict__ col, double* __restrict__ val) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  uint64_t* key = reinterpret_cast<uint64_t*>(smem) + static_cast<size_t>(warp) * lp;
  double* vv = reinterpret_cast<double*>(smem + static_cast<size_t>(nwarp) * lp * sizeof(uint64_t)) +
               static_cast<size_t>(warp) * lp;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * nwarp + warp; i < n;
       i += static_cast<int64_t>(gridDim.x) * nwarp) {
    const int64_t in0 = inptr[i], nin = inptr[i + 1] - in0;
    const int64_t len = 1 + d + nin;
    for (int64_t e = lane; e < lp; e += 32) {
      uint64_t kk = ~0ull;
      double x = 0.0;
      if (e < d) {
        const uint64_t idx = static_cast<uint64_t>(i * d + e);
        kk = (static_cast<uint64_t>(dcol[idx]) << 34) | idx;
        x = dval[idx];
      } else if (e == d) {
        const int a = level_of(L, i);
        const double u = u01_closed_open(sm64_at(seed, ctr(3, static_cast<uint64_t>(i))));
        kk = (static_cast<uint64_t>(i) << 34) | kDiagKey;
        x = __dadd_rn(__dmul_rn(10.0, (double)a), __dsub_rn(__dmul_rn(4.0, u), 2.0));
      } else if (e < len) {
        const uint64_t idx = inlist[in0 + (e - d - 1)];
        kk = (static_cast<uint64_t>(idx / static_cast<uint64_t>(d)) << 34) | idx;
        x = dval[idx];
      }
      key[e] = kk;
      vv[e] = x;
    }
    __syncwarp();
    // bitonic sort of lp (a power of two) keys, padding keys last
    for (int k = 2; k <= lp; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int e = lane; e < lp; e += 32) {
          const int ix = e ^ j;
          if (ix > e) {
            const bool up = (e & k) == 0;
            const uint64_t ke = key[e], kx = key[ix];
            if ((ke > kx) == up) {
              key[e] = kx;
              key[ix] = ke;
              const double t = vv[e];
              vv[e] = vv[ix];
              vv[ix] = t;
            }
          }
        }
        __syncwarp();
      }
    }
    // merge repeated columns: each head sums its run left to right
    int64_t base = write ? rp[i] : 0;
    unsigned count = 0;
    for (int64_t e0 = 0; e0 < len; e0 += 32) {
      const int64_t e = e0 + lane;
      bool head = false;
      uint64_t c = 0;
      double acc = 0.0;
      if (e < len) {
        c = key[e] >> 34;
        head = (e == 0) || ((key[e - 1] >> 34) != c);
        if (head) {
          acc = vv[e];
          for (int64_t f = e + 1; f < len && (key[f] >> 34) == c; ++f) acc = __dadd_rn(acc, vv[f]);
        }
      }
      const unsigned ball = __ballot_sync(0xffffffffu, head);
      if (write && head) {
        const int64_t pos = base + count + __popc(ball & ((1u << lane) - 1u));
        col[pos] = static_cast<int32_t>(c);
        val[pos] = acc;
      }
      count += __popc(ball);
    }
    if (!write && lane == 0) uniq[i] = count;
    __syncwarp();
  }
}

struct Gen {
  Levels L{};
  int64_t n = 0, d = 0, nnz = 0;
  double sigma = 0.5;
  uint64_t seed = 0;
  int lp = 0;
  int32_t* dcol = nullptr;
  double* dval = nullptr;
  int64_t* inptr = nullptr;
  uint32_t* inlist = nullptr;
  int64_t* rp = nullptr;
  unsigned* uniq = nullptr;
};

void release(Gen* g) {
  if (!g) return;
  cudaFree(g->dcol);
  cudaFree(g->dval);
  cudaFree(g->inptr);
  cudaFree(g->inlist);
  cudaFree(g->rp);
  cudaFree(g->uniq);
  delete g;
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

cudaError_t scan(const unsigned* in, int64_t n, int64_t* out, cudaStream_t s) {
  const int64_t nb = (n + kScanThreads - 1) / kScanThreads;
  int64_t* sums = nullptr;
  cudaError_t e = cudaMallocAsync(&sums, sizeof(int64_t) * (nb + 1), s);
  if (e != cudaSuccess) return e;
  k_block_sums<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(in, n, sums);
  k_scan_sums<<<1, 32, 0, s>>>(sums, nb);
  k_block_scan<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(in, n, sums, out);
  e = cudaGetLastError();
  cudaFreeAsync(sums, s);
  return e;
}

int warps_per_cta(int lp) {
  int w = 4;
  while (w > 1 && static_cast<size_t>(w) * lp * 16 > 96 * 1024) w >>= 1;
  return w;
}

cudaError_t rows_pass(Gen* g, bool write, int32_t* col, double* val, cudaStream_t s) {
  const int w = warps_per_cta(g->lp);
  const size_t smem = static_cast<size_t>(w) * g->lp * 16;
  cudaError_t e = cudaFuncSetAttribute(k_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::min<int64_t>((g->n + w - 1) / w, static_cast<int64_t>(sm_count()) * 64);
  k_rows<<<static_cast<unsigned>(blocks), 32 * w, smem, s>>>(g->L, g->n, g->d, g->seed, g->dcol, g->dval, g->inptr,
                                                             g->inlist, g->lp, write, g->uniq, g->rp, col, val);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

// Builds the matrix of gen.cpp's sppcgen_build on the current device, up to the
// row pointers: level_sizes[n_levels] rows per level, d draws per row, value
// spread sigma, SplitMix64 seed.  Returns an opaque handle (nullptr on bad
// arguments, a CUDA error or a row longer than the per-warp sort allows);
// sppcgen_dev_nnz gives the entry count, sppcgen_dev_fill writes the CSR.
// Requires n * d < 2^32.  Synchronises `stream`.
void* sppcgen_dev_build(const int64_t* level_sizes, int32_t n_levels, int32_t draws_per_row, double sigma,
                        uint64_t seed, void* stream) {
  if (!level_sizes || n_levels <= 0 || n_levels > kMaxLevels || draws_per_row < 0) return nullptr;
  Gen* g = new (std::nothrow) Gen();
  if (!g) return nullptr;
  g->L.n_levels = n_levels;
  g->L.off[0] = 0;
  for (int a = 0; a < n_levels; ++a) {
    if (level_sizes[a] <= 0) {
      delete g;
      return nullptr;
    }
    g->L.off[a + 1] = g->L.off[a] + level_sizes[a];
  }
  g->n = g->L.off[n_levels];
  g->d = draws_per_row;
  g->sigma = sigma;
  g->seed = seed;
  const int64_t n = g->n, d = g->d, total = n * d;
  if (n >= (1LL << 30) || total >= (1LL << 32)) {
    delete g;
    return nullptr;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* cnt = nullptr;
  unsigned* dmax = nullptr;
  cudaError_t e = cudaMalloc(&g->dcol, sizeof(int32_t) * std::max<int64_t>(total, 1));
  if (e == cudaSuccess) e = cudaMalloc(&g->dval, sizeof(double) * std::max<int64_t>(total, 1));
  if (e == cudaSuccess) e = cudaMalloc(&g->inptr, sizeof(int64_t) * (n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&g->inlist, sizeof(uint32_t) * std::max<int64_t>(total, 1));
  if (e == cudaSuccess) e = cudaMalloc(&g->rp, sizeof(int64_t) * (n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&g->uniq, sizeof(unsigned) * n);
  if (e == cudaSuccess) e = cudaMallocAsync(&cnt, sizeof(unsigned) * n, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&dmax, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dmax, 0, sizeof(unsigned), s);
  const unsigned grid = static_cast<unsigned>(sm_count() * 16);
  if (e == cudaSuccess) {
    k_draws<<<grid, 256, 0, s>>>(g->L, n, d, sigma, seed, g->dcol, g->dval, cnt);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = scan(cnt, n, g->inptr, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * n, s);
  if (e == cudaSuccess) {
    k_mirror<<<grid, 256, 0, s>>>(total, g->dcol, g->inptr, cnt, g->inlist);
    k_max_len<<<grid, 256, 0, s>>>(g->inptr, n, dmax);
    e = cudaGetLastError();
  }
  unsigned maxin = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&maxin, dmax, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (cnt) cudaFreeAsync(cnt, s);
  if (dmax) cudaFreeAsync(dmax, s);
  if (e != cudaSuccess) {
    release(g);
    return nullptr;
  }
  const int64_t maxlen = 1 + d + maxin;
  int lp = 32;
  while (lp < maxlen) lp <<= 1;
  if (lp > 8192) {  // beyond the per-warp shared-memory sort
    release(g);
    return nullptr;
  }
  g->lp = lp;
  e = rows_pass(g, false, nullptr, nullptr, s);
  if (e == cudaSuccess) e = scan(g->uniq, n, g->rp, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&g->nnz, g->rp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    release(g);
    return nullptr;
  }
  return g;
}

int64_t sppcgen_dev_n(void* h) { return h ? static_cast<Gen*>(h)->n : -1; }
int64_t sppcgen_dev_nnz(void* h) { return h ? static_cast<Gen*>(h)->nnz : -1; }

// Writes the CSR into caller-owned device buffers of n + 1, nnz and nnz
// entries.  Returns 0, or -1 on a CUDA error.  Synchronises `stream`.
int32_t sppcgen_dev_fill(void* h, int64_t* row_ptr, int32_t* col, double* val, void* stream) {
  if (!h || !row_ptr || (static_cast<Gen*>(h)->nnz > 0 && (!col || !val))) return -1;
  Gen* g = static_cast<Gen*>(h);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(row_ptr, g->rp, sizeof(int64_t) * (g->n + 1), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = rows_pass(g, true, col, val, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? 0 : -1;
}

void sppcgen_dev_free(void* h) { release(static_cast<Gen*>(h)); }

}  // extern "C"
