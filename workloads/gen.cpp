// Seeded synthetic hierarchical Hamiltonian generator (input module; holds none of
// the eigensolver's arithmetic).
//
// Stands in for the NCSM Hamiltonians of the paper's Table I, which are not
// available: a symmetric matrix whose basis is ordered by excitation level N,
// with the leading block (level 0) playing the small configuration space of
// Sec. 2 / Eq. (split2).  Law (one reading, applied to every workload):
//   * H_ii = 10*N(i) + U(-2, 2)
//   * every row i draws d off-diagonal columns j != i, uniformly with
//     replacement over the rows whose level differs from N(i) by at most 2;
//     each draw carries v ~ Normal(0, sigma^2) and emits both (i,j,v), (j,i,v);
//   * repeated (i,j) pairs are summed in a canonical order (by drawing row,
//     then draw index), so H == H^T holds bit for bit.
// Random numbers: one SplitMix64 sequence used in counter form (the n-th output
// is mix(seed + (n+1)*golden)), with disjoint counter ranges per stream.
// Normals: Box-Muller with a log and a cosine written here from their series
// (atanh series for log, Taylor series after quadrant reduction for cos) in
// plain IEEE +,-,*,/,sqrt, compiled without FMA contraction, so x86-64 and
// aarch64 hosts produce identical bytes.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
// n-th output of the SplitMix64 sequence whose state starts at `seed`.
inline uint64_t sm64_at(uint64_t seed, uint64_t n) { return mix64(seed + (n + 1) * kGolden); }
inline uint64_t ctr(uint64_t stream, uint64_t idx) { return (stream << 60) | idx; }
inline double u01_closed_open(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }       // [0,1)
inline double u01_open_closed(uint64_t r) { return (double)((r >> 11) + 1) * 0x1.0p-53; }  // (0,1]

// ln(x) for x > 0: x = m * 2^e with m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s),
// s = (m-1)/(m+1), |s| <= 0.1716, series summed to s^41.
double portable_log(double x) {
  int e = 0;
  double m = std::frexp(x, &e);  // exact: m in [0.5, 1)
  if (m < 0.70710678118654752440) {
    m = m * 2.0;
    e -= 1;
  }
  const double s = (m - 1.0) / (m + 1.0);
  const double s2 = s * s;
  double term = s, sum = 0.0;
  for (int k = 1; k <= 41; k += 2) {
    sum = sum + term / (double)k;
    term = term * s2;
  }
  const double ln2 = 0.69314718055994530942;
  return 2.0 * sum + (double)e * ln2;
}

// sin and cos of g*pi/2 for g in [0, 1/2] (argument <= pi/4), Taylor series.
void sincos_half_quadrant(double g, double* s_out, double* c_out) {
  const double half_pi = 1.57079632679489661923;
  const double a = g * half_pi;
  const double a2 = a * a;
  double ts = a, tc = 1.0, s = 0.0, c = 0.0;
  for (int k = 0; k < 14; ++k) {
    s = s + ts;
    c = c + tc;
    ts = ts * (-a2) / (double)((2 * k + 2) * (2 * k + 3));
    tc = tc * (-a2) / (double)((2 * k + 1) * (2 * k + 2));
  }
  *s_out = s;
  *c_out = c;
}

// cos(2*pi*u) for u in [0, 1).
double portable_cos_2pi(double u) {
  const double t = 4.0 * u;  // exact
  int q = (int)t;
  if (q > 3) q = 3;
  const double f = t - (double)q;  // exact, in [0, 1)
  double s, c;
  if (f <= 0.5) {
    sincos_half_quadrant(f, &s, &c);
  } else {
    double s2, c2;
    sincos_half_quadrant(1.0 - f, &s2, &c2);  // 1-f exact
    s = c2;
    c = s2;
  }
  // cos(q*pi/2 + a) for a = f*pi/2
  switch (q) {
    case 0: return c;
    case 1: return -s;
    case 2: return -c;
    default: return s;
  }
}

struct Entry {
  uint64_t key;  // (col << 34) | canonical contribution index
  double val;
};

struct Matrix {
  int64_t n = 0, nnz = 0;
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
};

constexpr uint64_t kDiagKey = (1ULL << 34) - 1;

}  // namespace

extern "C" {

// Builds the matrix described at the top of this file.
//   level_sizes[n_levels]: rows per level N = 0..n_levels-1 (contiguous blocks)
//   draws_per_row: d (about half the target nonzeros per row)
//   sigma: standard deviation of the off-diagonal values
//   seed: SplitMix64 start state
// Returns an opaque handle (nullptr on bad arguments or allocation failure).
void* sppcgen_build(const int64_t* level_sizes, int32_t n_levels, int32_t draws_per_row, double sigma,
                    uint64_t seed, int32_t n_threads) {
  if (!level_sizes || n_levels <= 0 || draws_per_row < 0) return nullptr;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
  std::vector<int64_t> off(n_levels + 1, 0);
  for (int a = 0; a < n_levels; ++a) {
    if (level_sizes[a] <= 0) return nullptr;
    off[a + 1] = off[a] + level_sizes[a];
  }
  const int64_t n = off[n_levels];
  if (n >= (1LL << 30)) return nullptr;
  const int64_t d = draws_per_row;
  if ((uint64_t)(n * d) >= (1ULL << 34) - 1) return nullptr;

  Matrix* M = new (std::nothrow) Matrix();
  if (!M) return nullptr;
  try {
    std::vector<int32_t> level_of(n);
    for (int a = 0; a < n_levels; ++a)
      for (int64_t i = off[a]; i < off[a + 1]; ++i) level_of[i] = a;

    // 1. draws
    std::vector<int32_t> dcol((size_t)(n * d));
    std::vector<double> dval((size_t)(n * d));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      const int a = level_of[i];
      const int64_t lo = off[std::max(a - 2, 0)];
      const int64_t hi = off[std::min(a + 2, n_levels - 1) + 1];
      const uint64_t w = (uint64_t)(hi - lo - 1);  // allowed columns excluding i
      for (int64_t t = 0; t < d; ++t) {
        const uint64_t idx = (uint64_t)(i * d + t);
        int64_t j = i;
        if (w > 0) {
          const uint64_t r = sm64_at(seed, ctr(0, idx));
          const uint64_t pick = (uint64_t)(((unsigned __int128)r * (unsigned __int128)w) >> 64);
          j = lo + (int64_t)pick;
          if (j >= i) ++j;
        }
        const double u1 = u01_open_closed(sm64_at(seed, ctr(1, idx)));
        const double u2 = u01_closed_open(sm64_at(seed, ctr(2, idx)));
        const double g = std::sqrt(-2.0 * portable_log(u1)) * portable_cos_2pi(u2);
        dcol[idx] = (int32_t)j;
        dval[idx] = (w > 0) ? sigma * g : 0.0;
      }
    }
    // 2. bucket sizes: diagonal + own draws + mirrored draws
    std::vector<int64_t> incoming(n, 0);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n * d; ++e) {
#pragma omp atomic
      incoming[dcol[e]] += 1;
    }
    std::vector<int64_t> bptr(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) bptr[i + 1] = bptr[i] + 1 + d + incoming[i];
    std::vector<Entry> bucket((size_t)bptr[n]);
    std::vector<int64_t> fill(n, 0);
    // own draws and diagonal
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      Entry* b = &bucket[bptr[i]];
      for (int64_t t = 0; t < d; ++t) {
        const uint64_t idx = (uint64_t)(i * d + t);
        b[t].key = ((uint64_t)dcol[idx] << 34) | idx;
        b[t].val = dval[idx];
      }
      const int a = level_of[i];
      const double u = u01_closed_open(sm64_at(seed, ctr(3, (uint64_t)i)));
      b[d].key = ((uint64_t)i << 34) | kDiagKey;
      b[d].val = 10.0 * (double)a + (4.0 * u - 2.0);
    }
    // mirrored draws (arrival order is irrelevant: rows are sorted below)
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
      for (int64_t t = 0; t < d; ++t) {
        const uint64_t idx = (uint64_t)(r * d + t);
        const int64_t j = dcol[idx];
        int64_t pos;
#pragma omp atomic capture
        pos = fill[j]++;
        Entry& e = bucket[bptr[j] + 1 + d + pos];
        e.key = ((uint64_t)r << 34) | idx;
        e.val = dval[idx];
      }
    }
    std::vector<int32_t>().swap(dcol);
    std::vector<double>().swap(dval);
    // 3. sort each row by (col, contribution index) and merge duplicates
    std::vector<int64_t> uniq(n, 0);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
      Entry* b = &bucket[bptr[i]];
      const int64_t len = bptr[i + 1] - bptr[i];
      std::sort(b, b + len, [](const Entry& x, const Entry& y) { return x.key < y.key; });
      int64_t u = 0;
      for (int64_t s = 0; s < len;) {
        const uint64_t c = b[s].key >> 34;
        double acc = b[s].val;
        int64_t e = s + 1;
        while (e < len && (b[e].key >> 34) == c) {
          acc = acc + b[e].val;
          ++e;
        }
        b[u].key = c;
        b[u].val = acc;
        ++u;
        s = e;
      }
      uniq[i] = u;
    }
    M->n = n;
    M->row_ptr.assign(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) M->row_ptr[i + 1] = M->row_ptr[i] + uniq[i];
    M->nnz = M->row_ptr[n];
    M->col.resize((size_t)M->nnz);
    M->val.resize((size_t)M->nnz);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      const Entry* b = &bucket[bptr[i]];
      int64_t o = M->row_ptr[i];
      for (int64_t s = 0; s < uniq[i]; ++s) {
        M->col[o + s] = (int32_t)b[s].key;
        M->val[o + s] = b[s].val;
      }
    }
  } catch (...) {
    delete M;
    return nullptr;
  }
  return M;
}

int64_t sppcgen_n(void* h) { return h ? static_cast<Matrix*>(h)->n : -1; }
int64_t sppcgen_nnz(void* h) { return h ? static_cast<Matrix*>(h)->nnz : -1; }

// Copies the CSR arrays into caller-owned buffers of sizes n+1, nnz, nnz.
int32_t sppcgen_copy(void* h, int64_t* row_ptr, int32_t* col, double* val) {
  if (!h) return -1;
  const Matrix* M = static_cast<Matrix*>(h);
  std::memcpy(row_ptr, M->row_ptr.data(), sizeof(int64_t) * (size_t)(M->n + 1));
  std::memcpy(col, M->col.data(), sizeof(int32_t) * (size_t)M->nnz);
  std::memcpy(val, M->val.data(), sizeof(double) * (size_t)M->nnz);
  return 0;
}

void sppcgen_free(void* h) { delete static_cast<Matrix*>(h); }

// Exposed for the generator's own tests: the portable log / cos / normal.
double sppcgen_log(double x) { return portable_log(x); }
double sppcgen_cos2pi(double u) { return portable_cos_2pi(u); }
uint64_t sppcgen_sm64(uint64_t seed, uint64_t n) { return sm64_at(seed, n); }

}  // extern "C"
