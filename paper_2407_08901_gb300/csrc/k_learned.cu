// Learned correction proposal (not in the paper): a per-row network
// 6 -> 64 -> 64 -> 1 with GELU (tanh form, Hendrycks and Gimpel 2016) predicts,
// for row i and Ritz pair j, a relative correction m_ij to the diagonally
// preconditioned residual; the proposal g_ij = (r_ij / den_ij)(1 + m_ij),
// den_ij = H_ii - theta_j clamped to |den| >= clamp (Davidson's shifted diagonal).
// Features: H_ii, level(i), ||H_i,:||_2, rhat_ij = r_ij sqrt(n) / ||r_j||, theta_j,
// (|H| |rhat_j|)_i, standardised by the training set's mean and spread.
//
// Parameters (one flat FP32 vector, 4,673 values): W1 (64 x 6, row-major),
// b1 (64), W2 (64 x 64, W2[o][i] at o*64 + i), b2 (64), w3 (64), b3.
//
// Inference (the solve): BF16 weights and activations (inputs, h1, h2 rounded
// to BF16 before each product), FP32 sums and biases, tanh.approx in GELU.
// Training: FP32 throughout (tanhf), one CTA per 128 samples computes the
// forward pass, the backward pass and its partial weight gradient in shared
// memory; a second kernel sums the partials in a fixed order (deterministic);
// Adam (Kingma and Ba 2015) updates the parameters.
#include <cuda_bf16.h>

#include "df.cuh"
#include "sppc_internal.h"

namespace sppc {

namespace {

constexpr int NF = kNetFeatures, NH = kNetHidden;
constexpr int OFF_W1 = 0, OFF_B1 = NH * NF, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == kNetParams, "parameter layout");
static_assert(OFF_W2 % 4 == 0, "W2 rows must be 16-byte aligned in shared memory");
constexpr int NSW = (NPARAM + 2 * NF + 3) / 4 * 4;  // weights + mu + sd, padded
constexpr float kC = 0.7978845608028654f;           // sqrt(2 / pi)
constexpr float kA = 0.044715f;
constexpr int TB = 128;   // training samples per CTA
constexpr int LD = 65;    // padded row stride of the per-sample activations
constexpr double kMinOverlap = 0.5;  // training pairs need |z_j^T psi_j| >= this

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float gelu_fast(float a) { return 0.5f * a * (1.f + tanh_fast(kC * (a + kA * a * a * a))); }
__device__ __forceinline__ float gelu_acc(float a) { return 0.5f * a * (1.f + tanhf(kC * (a + kA * a * a * a))); }
__device__ __forceinline__ float gelu_grad(float a) {
  const float th = tanhf(kC * (a + kA * a * a * a));
  return 0.5f * (1.f + th) + 0.5f * a * (1.f - th * th) * kC * (1.f + 3.f * kA * a * a);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ bool is_bias(int q) {
  return (q >= OFF_B1 && q < OFF_W2) || (q >= OFF_B2 && q < OFF_W3) || q == OFF_B3;
}

// Stage the parameters (and mu, sd when given) into shared memory; with BF the
// weights (not the biases) are rounded to BF16.
template <bool BF>
__device__ __forceinline__ void load_net(float* sw, const float* __restrict__ params, const float* __restrict__ musd) {
  for (int q = threadIdx.x; q < NSW; q += blockDim.x) {
    float v = 0.f;
    if (q < NPARAM) {
      v = params[q];
      if (BF && !is_bias(q)) v = bf16r(v);
    } else if (q < NPARAM + 2 * NF && musd) {
      v = musd[q - NPARAM];
    }
    sw[q] = v;
  }
}

// m = w3 . gelu(W2 gelu(W1 x + b1) + b2) + b3 for one sample (x standardised).
template <bool BF>
__device__ __forceinline__ float mlp_eval(const float* __restrict__ sw, const float (&xin)[NF]) {
  float x[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) x[f] = BF ? bf16r(xin[f]) : xin[f];
  float h1[NH];
#pragma unroll
  for (int o = 0; o < NH; ++o) {
    float a = sw[OFF_B1 + o];
#pragma unroll
    for (int f = 0; f < NF; ++f) a = fmaf(sw[OFF_W1 + o * NF + f], x[f], a);
    h1[o] = BF ? bf16r(gelu_fast(a)) : gelu_acc(a);
  }
  float m = sw[OFF_B3];
#pragma unroll 1
  for (int o = 0; o < NH; ++o) {
    float a = sw[OFF_B2 + o];
    const float4* w = reinterpret_cast<const float4*>(sw + OFF_W2 + o * NH);
#pragma unroll
    for (int i = 0; i < NH / 4; ++i) {
      const float4 q = w[i];
      a = fmaf(q.x, h1[4 * i], a);
      a = fmaf(q.y, h1[4 * i + 1], a);
      a = fmaf(q.z, h1[4 * i + 2], a);
      a = fmaf(q.w, h1[4 * i + 3], a);
    }
    const float h2 = BF ? bf16r(gelu_fast(a)) : gelu_acc(a);
    m = fmaf(sw[OFF_W3 + o], h2, m);
  }
  return m;
}

// Network output for `count` standardised samples X (count x 6).
template <bool BF>
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ params, const float* __restrict__ X,
                                                     int64_t count, float* __restrict__ out) {
  __shared__ __align__(16) float sw[NSW];
  load_net<BF>(sw, params, nullptr);
  __syncthreads();
#pragma unroll 1
  for (int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < count;
       s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    asm volatile("" ::: "memory");  // keep the staged weights in shared memory, not hoisted into registers
    float x[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) x[f] = X[s * NF + f];
    out[s] = mlp_eval<BF>(sw, x);
  }
}

// One CTA = up to 128 samples of a minibatch: forward, backward, and the CTA's
// partial sums of dL/dparams (L = inv_b * sum (rhat (1 + m) - y)^2) and of the
// squared errors, written to part[blockIdx.x * (NPARAM + 1) + q].
__global__ void __launch_bounds__(TB) k_mlp_grad(const float* __restrict__ params, const float* __restrict__ X,
                                                 const float* __restrict__ rhat, const float* __restrict__ y,
                                                 const int64_t* __restrict__ perm, int64_t base, int64_t count,
                                                 float inv_b, float* __restrict__ part) {
  extern __shared__ __align__(16) float smem[];
  float* sw = smem;                    // NSW
  float* sX = sw + NSW;                // TB * NF
  float* sDm = sX + TB * NF;           // TB
  float* sL = sDm + TB;                // TB
  float* sA1 = sL + TB;                // TB * LD: a1, later h1
  float* sA2 = sA1 + TB * LD;          // TB * LD: a2, later delta2
  float* sD1 = sA2 + TB * LD;          // TB * LD: dm * h2, later delta1
  load_net<false>(sw, params, nullptr);
  const int t = threadIdx.x;
  const int64_t local = static_cast<int64_t>(blockIdx.x) * TB + t;
  const bool valid = local < count;
  float x[NF], r = 0.f, yy = 0.f;
  if (valid) {
    const int64_t idx = perm ? perm[base + local] : base + local;
#pragma unroll
    for (int f = 0; f < NF; ++f) x[f] = X[idx * NF + f];
    r = rhat[idx];
    yy = y[idx];
  } else {
#pragma unroll
    for (int f = 0; f < NF; ++f) x[f] = 0.f;
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) sX[t * NF + f] = x[f];
  __syncthreads();
  // forward
  float h1[NH];
#pragma unroll
  for (int o = 0; o < NH; ++o) {
    float a = sw[OFF_B1 + o];
#pragma unroll
    for (int f = 0; f < NF; ++f) a = fmaf(sw[OFF_W1 + o * NF + f], x[f], a);
    sA1[t * LD + o] = a;
    h1[o] = gelu_acc(a);
  }
  float m = sw[OFF_B3];
#pragma unroll 1
  for (int o = 0; o < NH; ++o) {
    float a = sw[OFF_B2 + o];
    const float4* w = reinterpret_cast<const float4*>(sw + OFF_W2 + o * NH);
#pragma unroll
    for (int i = 0; i < NH / 4; ++i) {
      const float4 q = w[i];
      a = fmaf(q.x, h1[4 * i], a);
      a = fmaf(q.y, h1[4 * i + 1], a);
      a = fmaf(q.z, h1[4 * i + 2], a);
      a = fmaf(q.w, h1[4 * i + 3], a);
    }
    sA2[t * LD + o] = a;
    m = fmaf(sw[OFF_W3 + o], gelu_acc(a), m);
  }
  const float e = r * (1.f + m) - yy;
  const float dm = valid ? 2.f * e * r * inv_b : 0.f;
  sDm[t] = dm;
  sL[t] = valid ? e * e : 0.f;
  // output layer: dm * h2 (for dw3) and delta2 = dm w3 gelu'(a2)
#pragma unroll 4
  for (int o = 0; o < NH; ++o) {
    const float a = sA2[t * LD + o];
    sD1[t * LD + o] = dm * gelu_acc(a);
    sA2[t * LD + o] = dm * sw[OFF_W3 + o] * gelu_grad(a);
  }
  __syncthreads();
  float* pg = part + static_cast<int64_t>(blockIdx.x) * (NPARAM + 1);
  if (t < NH) {
    float g = 0.f;
    for (int s = 0; s < TB; ++s) g += sD1[s * LD + t];
    pg[OFF_W3 + t] = g;
  } else if (t == NH) {
    float g = 0.f;
    for (int s = 0; s < TB; ++s) g += sDm[s];
    pg[OFF_B3] = g;
  } else if (t == NH + 1) {
    float g = 0.f;
    for (int s = 0; s < TB; ++s) g += sL[s];
    pg[NPARAM] = g;
  }
  __syncthreads();
  // delta1 = gelu'(a1) (W2^T delta2), then h1 in place of a1
  {
    float d2[NH];
#pragma unroll
    for (int o = 0; o < NH; ++o) d2[o] = sA2[t * LD + o];
#pragma unroll 1
    for (int i = 0; i < NH; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int o = 0; o < NH; ++o) acc = fmaf(sw[OFF_W2 + o * NH + i], d2[o], acc);
      const float a = sA1[t * LD + i];
      sD1[t * LD + i] = acc * gelu_grad(a);
      sA1[t * LD + i] = gelu_acc(a);
    }
  }
  __syncthreads();
  // weight gradients: sums over the CTA's samples in sample order
  for (int q = t; q < NH * NH; q += TB) {
    const int o = q / NH, i = q % NH;
    float g = 0.f;
    for (int s = 0; s < TB; ++s) g = fmaf(sA2[s * LD + o], sA1[s * LD + i], g);
    pg[OFF_W2 + q] = g;
  }
  for (int q = t; q < NH * NF; q += TB) {
    const int o = q / NF, f = q % NF;
    float g = 0.f;
    for (int s = 0; s < TB; ++s) g = fmaf(sD1[s * LD + o], sX[s * NF + f], g);
    pg[OFF_W1 + q] = g;
  }
  if (t < NH) {
    float g1 = 0.f, g2 = 0.f;
    for (int s = 0; s < TB; ++s) {
      g1 += sD1[s * LD + t];
      g2 += sA2[s * LD + t];
    }
    pg[OFF_B1 + t] = g1;
    pg[OFF_B2 + t] = g2;
  }
}

// grad[q] = sum over CTAs of part[b][q] (fixed order); grad[NPARAM] = loss.
__global__ void k_grad_reduce(const float* __restrict__ part, int nb, float inv_b, float* __restrict__ grad,
                              float* __restrict__ loss_slot) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q > NPARAM) return;
  float g = 0.f;
  for (int b = 0; b < nb; ++b) g += part[static_cast<int64_t>(b) * (NPARAM + 1) + q];
  if (q < NPARAM)
    grad[q] = g;
  else if (loss_slot)
    *loss_slot = g * inv_b;
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ mo, float* __restrict__ ve,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= NPARAM) return;
  const float gq = g[q];
  const float m = b1 * mo[q] + (1.f - b1) * gq;
  const float v = b2 * ve[q] + (1.f - b2) * gq * gq;
  mo[q] = m;
  ve[q] = v;
  p[q] -= lr * (m * c1) / (sqrtf(v * c2) + eps);
}

// Per-row constants of the features: (level(i), ||H_i,:||_2) from the CSR.
__global__ void k_row_consts(int64_t n, const int64_t* __restrict__ rp, const double* __restrict__ va,
                             const int64_t* __restrict__ lev, int nlev, float2* __restrict__ out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t t = rp[i]; t < rp[i + 1]; ++t) s = fma(va[t], va[t], s);
  int lv = 0;
  while (lv + 1 < nlev && i >= lev[lv + 1]) ++lv;
  out[i] = make_float2(static_cast<float>(lv), static_cast<float>(sqrt(s)));
}

// rhat_ij = r_ij sqrt(n) / ||r_j|| (FP32; 0 for padding columns or r_j = 0) and
// its absolute value, the input of the |H| product; both n x 8.
__global__ void k_prop_prep(const float2* __restrict__ R, int kp, int k, const double* __restrict__ rn2, int64_t n,
                            float* __restrict__ rhat, float* __restrict__ absr) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n * 8) return;
  const int64_t i = t >> 3;
  const int j = static_cast<int>(t & 7);
  float v = 0.f;
  if (j < k && rn2[j] > 0.0) {
    const double sc = sqrt(static_cast<double>(n) / rn2[j]);
    const float2 r = R[i * kp + j];
    v = static_cast<float>(((double)r.x + (double)r.y) * sc);
  }
  rhat[t] = v;
  absr[t] = fabsf(v);
}

__device__ __forceinline__ float2 shifted_den(float2 d, float2 th, float clamp) {
  float2 den = df_sub(d, th);
  if (fabsf(den.x) < clamp) den = make_float2(den.x < 0.f ? -clamp : clamp, 0.f);
  return den;
}

__device__ __forceinline__ void sample_features(float (&f)[NF], float2 dg, float2 rc, float rh, float2 th, float ag) {
  f[0] = dg.x;
  f[1] = rc.x;
  f[2] = rc.y;
  f[3] = rh;
  f[4] = th.x;
  f[5] = ag;
}

// The proposal block for rows [n0, n): Tprop = (R / den)(1 + m), Tplain = R / den;
// padding columns 0.  Persistent grid; the network staged once per CTA.
__global__ void __launch_bounds__(128) k_prop_mlp(const float* __restrict__ net, const float2* __restrict__ R,
                                                  const float2* __restrict__ diag, const float2* __restrict__ rowc,
                                                  const float* __restrict__ rhat, const float2* __restrict__ agg,
                                                  const float2* __restrict__ theta, float clamp, int k, int kp,
                                                  int64_t n0, int64_t n, float2* __restrict__ Tprop,
                                                  float2* __restrict__ Tplain) {
  __shared__ __align__(16) float sw[NSW];
  load_net<true>(sw, net, net + NPARAM);
  __syncthreads();
  const float* mu = sw + NPARAM;
  const float* sd = sw + NPARAM + NF;
  const int64_t count = (n - n0) * kp;
#pragma unroll 1
  for (int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < count;
       s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    asm volatile("" ::: "memory");  // keep the staged weights in shared memory, not hoisted into registers
    const int64_t i = n0 + s / kp;
    const int j = static_cast<int>(s % kp);
    const int64_t o = i * kp + j;
    if (j >= k) {
      Tprop[o] = make_float2(0.f, 0.f);
      Tplain[o] = make_float2(0.f, 0.f);
      continue;
    }
    const float2 dg = diag[i], th = theta[j];
    float f[NF];
    sample_features(f, dg, rowc[i], rhat[i * 8 + j], th, agg[i * 8 + j].x);
    float x[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) x[q] = (f[q] - mu[q]) / sd[q];
    const float m = mlp_eval<true>(sw, x);
    const float2 t = df_div(R[o], shifted_den(dg, th, clamp));
    Tplain[o] = t;
    Tprop[o] = df_mul(t, make_float2(1.f + m, 0.f));
  }
}

// Training samples from the current Ritz state and exact eigenvectors psi:
// rows [n0, n), pairs j < k, sample (i - n0) * k + j: raw features, rhat and the
// target y = -den (psi_j / c_j - z_j)_i sqrt(n) / ||r_j||, c_j = z_j^T psi_j
// (rhat = y = 0 for pairs with |c_j| < 1/2).
__global__ void k_prop_samples(const float2* __restrict__ R, const double* __restrict__ Z, int64_t ldz,
                               const double* __restrict__ psi, int64_t ldpsi, const double* __restrict__ c,
                               const double* __restrict__ rn2, const float2* __restrict__ diag,
                               const float2* __restrict__ rowc, const float* __restrict__ rhat,
                               const float2* __restrict__ agg, const float2* __restrict__ theta, float clamp, int k,
                               int kp, int64_t n0, int64_t n, float* __restrict__ F, float* __restrict__ rh_out,
                               float* __restrict__ y) {
  const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= (n - n0) * k) return;
  const int64_t i = n0 + s / k;
  const int j = static_cast<int>(s % k);
  const float2 dg = diag[i], th = theta[j];
  float f[NF];
  sample_features(f, dg, rowc[i], rhat[i * 8 + j], th, agg[i * 8 + j].x);
#pragma unroll
  for (int q = 0; q < NF; ++q) F[s * NF + q] = f[q];
  // a Ritz vector far from its eigenvector (|c_j| < 1/2) gives no usable target:
  // rhat = y = 0 (zero loss and gradient)
  if (fabs(c[j]) < kMinOverlap) {
    rh_out[s] = 0.f;
    y[s] = 0.f;
    return;
  }
  rh_out[s] = f[3];
  const float2 den = shifted_den(dg, th, clamp);
  const double t = psi[i * ldpsi + j] / c[j] - Z[i * ldz + j];
  const double sc = rn2[j] > 0.0 ? sqrt(static_cast<double>(n) / rn2[j]) : 0.0;
  y[s] = static_cast<float>(-((double)den.x + (double)den.y) * t * sc);
  (void)R;
  (void)kp;
}

// c[j] = sum_i Z[i, j] psi[i, j] (FP64; partial sums per CTA, then one thread per
// column in CTA order).
__global__ void k_dot_cols(const double* __restrict__ Z, int64_t ldz, const double* __restrict__ psi, int64_t ldpsi,
                           int k, int64_t n, double* __restrict__ part) {
  __shared__ double red[8][256];
  for (int j = 0; j < k; ++j) {
    double s = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
      s = fma(Z[i * ldz + j], psi[i * ldpsi + j], s);
    red[j][threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int t = 0; t < blockDim.x; ++t) s += red[threadIdx.x][t];
    part[blockIdx.x * 8 + threadIdx.x] = s;
  }
}

__global__ void k_dot_finish(const double* __restrict__ part, int nb, int k, double* __restrict__ c) {
  const int j = threadIdx.x;
  if (j >= k) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[b * 8 + j];
  c[j] = s;
}

// Per-feature sums of f and f^2 over `count` samples (FP64; partial sums per CTA
// in a fixed order, finished by one thread per feature).
__global__ void k_moments(const float* __restrict__ F, int64_t count, double* __restrict__ part) {
  __shared__ double red[2 * NF][256];
  double s[2 * NF];
#pragma unroll
  for (int q = 0; q < 2 * NF; ++q) s[q] = 0.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const double v = F[i * NF + f];
      s[f] += v;
      s[NF + f] = fma(v, v, s[NF + f]);
    }
  }
#pragma unroll
  for (int q = 0; q < 2 * NF; ++q) red[q][threadIdx.x] = s[q];
  __syncthreads();
  if (threadIdx.x < 2 * NF) {
    double a = 0.0;
    for (int t = 0; t < blockDim.x; ++t) a += red[threadIdx.x][t];
    part[blockIdx.x * 2 * NF + threadIdx.x] = a;
  }
}

__global__ void k_moments_finish(const double* __restrict__ part, int nb, int64_t count, double* __restrict__ out) {
  const int f = threadIdx.x;
  if (f >= NF) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nb; ++i) {
    a += part[i * 2 * NF + f];
    b += part[i * 2 * NF + NF + f];
  }
  const double mean = a / static_cast<double>(count);
  const double var = b / static_cast<double>(count) - mean * mean;
  out[f] = mean;
  out[NF + f] = sqrt(var > 0.0 ? var : 0.0);
}

__global__ void k_standardize(const float* __restrict__ F, int64_t count, float4 m0, float2 m1, float4 r0, float2 r1,
                              float* __restrict__ X) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= count * NF) return;
  const int f = static_cast<int>(t % NF);
  const float mu[NF] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y};
  const float sd[NF] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y};
  X[t] = (F[t] - mu[f]) / sd[f];
}

int persistent_grid(const void* fn, int threads) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0);
  return sms * (per < 1 ? 1 : per);
}

size_t grad_smem() { return sizeof(float) * (NSW + TB * NF + 2 * TB + 3 * TB * LD); }

}  // namespace

cudaError_t mlp_forward(const float* params, const float* X, int64_t count, bool bf16, float* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const void* fn = bf16 ? reinterpret_cast<const void*>(k_mlp_forward<true>)
                        : reinterpret_cast<const void*>(k_mlp_forward<false>);
  int64_t grid = (count + 127) / 128;
  const int gmax = persistent_grid(fn, 128);
  if (grid > gmax) grid = gmax;
  if (bf16)
    k_mlp_forward<true><<<static_cast<unsigned>(grid), 128, 0, s>>>(params, X, count, out);
  else
    k_mlp_forward<false><<<static_cast<unsigned>(grid), 128, 0, s>>>(params, X, count, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mlp_grad(const float* params, const float* X, const float* rhat, const float* y, const int64_t* perm,
                     int64_t base, int64_t count, float inv_b, float* part, float* grad, float* loss_slot,
                     cudaStream_t s) {
  if (count <= 0) return cudaErrorInvalidValue;
  const size_t sm = grad_smem();
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(grad_smem()));
  if (attr != cudaSuccess) return attr;
  const int nb = static_cast<int>((count + TB - 1) / TB);
  k_mlp_grad<<<nb, TB, sm, s>>>(params, X, rhat, y, perm, base, count, inv_b, part);
  count_launch();
  k_grad_reduce<<<(NPARAM + 1 + 255) / 256, 256, 0, s>>>(part, nb, inv_b, grad, loss_slot);
  count_launch();
  return cudaGetLastError();
}

int64_t mlp_grad_part_floats(int64_t batch) { return ((batch + TB - 1) / TB) * (NPARAM + 1); }

cudaError_t mlp_adam(float* params, float* mom, float* vel, const float* grad, float lr, float b1, float b2,
                     float eps, float c1, float c2, cudaStream_t s) {
  k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(params, mom, vel, grad, lr, b1, b2, eps, c1, c2);
  count_launch();
  return cudaGetLastError();
}

cudaError_t row_consts(int64_t n, const int64_t* rp, const double* va, const int64_t* lev, int nlev, float2* out,
                       cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_row_consts<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(n, rp, va, lev, nlev, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t prop_prep(const float2* R, int kp, int k, const double* rn2, int64_t n, float* rhat, float* absr,
                      cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_prop_prep<<<static_cast<unsigned>((n * 8 + 255) / 256), 256, 0, s>>>(R, kp, k, rn2, n, rhat, absr);
  count_launch();
  return cudaGetLastError();
}

cudaError_t prop_mlp(const float* net, const float2* R, const float2* diag, const float2* rowc, const float* rhat,
                     const float2* agg, const float2* theta, float clamp, int k, int kp, int64_t n0, int64_t n,
                     float2* Tprop, float2* Tplain, cudaStream_t s) {
  if (n <= n0) return cudaSuccess;
  static const int gmax = persistent_grid(reinterpret_cast<const void*>(k_prop_mlp), 128);
  int64_t grid = ((n - n0) * kp + 127) / 128;
  if (grid > gmax) grid = gmax;
  k_prop_mlp<<<static_cast<unsigned>(grid), 128, 0, s>>>(net, R, diag, rowc, rhat, agg, theta, clamp, k, kp, n0, n,
                                                         Tprop, Tplain);
  count_launch();
  return cudaGetLastError();
}

cudaError_t prop_samples(const float2* R, const double* Z, int64_t ldz, const double* psi, int64_t ldpsi,
                         const double* rn2, const float2* diag, const float2* rowc, const float* rhat,
                         const float2* agg, const float2* theta, float clamp, int k, int kp, int64_t n0, int64_t n,
                         double* scratch, float* F, float* rh_out, float* y, cudaStream_t s) {
  if (n <= n0) return cudaSuccess;
  constexpr int NB = 256;
  k_dot_cols<<<NB, 256, 0, s>>>(Z, ldz, psi, ldpsi, k, n, scratch);
  count_launch();
  k_dot_finish<<<1, 32, 0, s>>>(scratch, NB, k, scratch + NB * 8);
  count_launch();
  const int64_t cnt = (n - n0) * k;
  k_prop_samples<<<static_cast<unsigned>((cnt + 255) / 256), 256, 0, s>>>(
      R, Z, ldz, psi, ldpsi, scratch + NB * 8, rn2, diag, rowc, rhat, agg, theta, clamp, k, kp, n0, n, F, rh_out, y);
  count_launch();
  return cudaGetLastError();
}

int64_t prop_samples_scratch_doubles() { return 256 * 8 + 8; }

cudaError_t feature_moments(const float* F, int64_t count, double* scratch, cudaStream_t s) {
  constexpr int NB = 256;
  if (count <= 0) return cudaErrorInvalidValue;
  k_moments<<<NB, 256, 0, s>>>(F, count, scratch);
  count_launch();
  k_moments_finish<<<1, 32, 0, s>>>(scratch, NB, count, scratch + NB * 2 * NF);
  count_launch();
  return cudaGetLastError();
}

int64_t feature_moments_scratch_doubles() { return 256 * 2 * NF + 2 * NF; }

cudaError_t standardize(const float* F, int64_t count, const float* mu, const float* sd, float* X, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_standardize<<<static_cast<unsigned>((count * NF + 255) / 256), 256, 0, s>>>(
      F, count, make_float4(mu[0], mu[1], mu[2], mu[3]), make_float2(mu[4], mu[5]),
      make_float4(sd[0], sd[1], sd[2], sd[3]), make_float2(sd[4], sd[5]), X);
  count_launch();
  return cudaGetLastError();
}

}  // namespace sppc
