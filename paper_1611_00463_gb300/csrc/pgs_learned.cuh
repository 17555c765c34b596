// Learned-CDF splitters: a monotone 1 -> 32 -> 32 -> 1 ReLU model of the key
// CDF, trained in FP32 on the method's own sorted sample (K10), gives every
// key a bucket; as the model is monotone and the runs sorted, the cut of run r
// at bucket b is found by bisection of the run (K11).  The sampled splitters
// with the investigator stay the
// judge: if the learned buckets are more unbalanced than 1 + eps, or a given
// model is not monotone, the sampled cuts are kept.
//
// Model layout (PGS_MLP_WORDS 4-byte words): w1[32], b1[32], W2[32][32]
// (row k, column j; only entries with k and j in the same half are used),
// b2[32], w3[32], b3, then kmin (low, high 32-bit words), scale (float) and a
// validity flag.  Units 0..15 take +x and enter the output with weight >= 0;
// units 16..31 take -x (w1 <= 0) and enter with weight <= 0; W2 >= 0.  With
// these signs every fp32 operation of the evaluation below is monotone, so
// the bucket id is non-decreasing in the key.
#pragma once

#include <cstdint>

#include "pgs_kernels.cuh"

namespace pgs {

constexpr int kMlpH = 32;
constexpr int kMlpHalf = 16;
constexpr int kMlpW = 1153;                 // weights
constexpr int kMlpWords = kMlpW + 4;        // + kmin lo, kmin hi, scale, flag
constexpr int kMlpOffW1 = 0, kMlpOffB1 = 32, kMlpOffW2 = 64, kMlpOffB2 = 1088, kMlpOffW3 = 1120, kMlpOffB3 = 1152;
constexpr int kMlpSteps = 300;
constexpr float kMlpLr = 0.01f;
constexpr float kMlpOffDiag = -6.0f;
constexpr int kMlpBatch = 128;              // training samples per CTA (3 CTAs of 72 KB per SM)
// Largest P the model is trained for.  Its output is piecewise linear with at
// most 32 layer-1 knots and 32 layer-2 clipping points, about 64 pieces, so it
// cannot place P - 1 > 64 bucket boundaries within eps of their quantiles for
// a general CDF (measured: no model passed the judge at P >= 64 on the
// exponential, normal + lognormal or Zipf keys).  Above it no model is
// trained, the sampled cuts stand (fallback) and the model's own imbalance is
// reported as NaN (not evaluated).  A caller-given model is still judged.
constexpr uint32_t kLearnedMaxP = 64;

__device__ __forceinline__ bool same_half(int k, int j) { return (k < kMlpHalf) == (j < kMlpHalf); }

// Key -> model input: x = f32(f64(max(k, kmin) - kmin)) * scale.
template <typename K>
__device__ __forceinline__ float mlp_input(K key, uint64_t kmin, float scale) {
  const uint64_t k = (uint64_t)key;
  const uint64_t d = k > kmin ? k - kmin : 0;
  return __fmul_rn(__double2float_rn(__ull2double_rn(d)), scale);
}

// Bucket id min(P-1, floor(P clamp(y, 0, 1))), y evaluated in fp32 in a fixed
// order with every product and sum rounded separately (no fused multiply-add):
// h1_j = max(w1_j x + b1_j, 0); acc = b2_k; acc += W2_kj h1_j for j of k's half
// in increasing order; h2_k = max(acc, 0); y = b3; y += w3_k h2_k, k = 0..31.
// W: a pointer to the weights (a volatile one keeps a loop that evaluates the
// model many times from holding every weight in registers).
template <typename W = const float*>
__device__ __forceinline__ uint32_t mlp_bucket(W w, float x, uint32_t P) {
  float h1[kMlpH];
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) {
    const float z = __fadd_rn(__fmul_rn(w[kMlpOffW1 + j], x), w[kMlpOffB1 + j]);
    h1[j] = z > 0.0f ? z : 0.0f;
  }
  float y = w[kMlpOffB3];
#pragma unroll
  for (int k = 0; k < kMlpH; ++k) {
    float acc = w[kMlpOffB2 + k];
    const int lo = k < kMlpHalf ? 0 : kMlpHalf;
#pragma unroll
    for (int j = 0; j < kMlpHalf; ++j) acc = __fadd_rn(acc, __fmul_rn(w[kMlpOffW2 + k * kMlpH + lo + j], h1[lo + j]));
    const float h2 = acc > 0.0f ? acc : 0.0f;
    y = __fadd_rn(y, __fmul_rn(w[kMlpOffW3 + k], h2));
  }
  const float c = fminf(fmaxf(y, 0.0f), 1.0f);
  const float t = floorf(__fmul_rn((float)P, c));
  const uint32_t b = (uint32_t)t;
  return b < P ? b : P - 1;
}

// ---------------------------------------------------------------------------
// K10: training.  Raw parameters (v1, b1, V2, b2, v3, b3) map to the weights
// w1 = +-exp(v1), W2 = exp(V2) inside a half, w3 = +-exp(v3); full-batch Adam
// on the mean squared error against the empirical CDF (i + 1/2) / S.
// ---------------------------------------------------------------------------

struct MlpState {
  float raw[kMlpW];
  float m[kMlpW];
  float v[kMlpW];
  uint64_t kmin;
  float scale;
  float loss;
};

__device__ __forceinline__ float mlp_sign(int j) { return j < kMlpHalf ? 1.0f : -1.0f; }

// One CTA: normalisation from the sorted sample, knots of layer 1 at the
// samples of sorted index floor((2j + 1) S / 32), layer 2 close to the identity.
template <typename K>
__global__ void k_mlp_init(const K* __restrict__ sorted, uint64_t S, MlpState* st) {
  pdl_enter();
  const uint64_t kmin = (uint64_t)sorted[0];
  const uint64_t span = (uint64_t)sorted[S - 1] - kmin;
  const float scale = span == 0 ? 0.0f : __fdiv_rn(1.0f, __double2float_rn(__ull2double_rn(span)));
  for (int p = threadIdx.x; p < kMlpW; p += blockDim.x) {
    float r = 0.0f;
    if (p >= kMlpOffB1 && p < kMlpOffW2) {
      const int j = p - kMlpOffB1;
      const int jj = j % kMlpHalf;
      const float q = mlp_input<K>(sorted[((2ull * jj + 1) * S) / (2 * kMlpHalf)], kmin, scale);
      r = j < kMlpHalf ? -q : q;
    } else if (p >= kMlpOffW2 && p < kMlpOffB2) {
      const int k = (p - kMlpOffW2) / kMlpH, j = (p - kMlpOffW2) % kMlpH;
      r = same_half(k, j) ? (k == j ? 0.0f : kMlpOffDiag) : 0.0f;
    } else if (p >= kMlpOffW3 && p < kMlpOffB3) {
      r = -3.4657359f;                                    // log(1/32)
    } else if (p == kMlpOffB3) {
      r = 0.5f;
    }
    st->raw[p] = r;
    st->m[p] = 0.0f;
    st->v[p] = 0.0f;
  }
  if (threadIdx.x == 0) {
    st->kmin = kmin;
    st->scale = scale;
    st->loss = 0.0f;
  }
}

// Per-sample activations are stored unit-major with a padded row (kMlpBatch + 1
// floats): a thread's stores of its own sample and the per-parameter sums over
// samples (consecutive units across a warp) are both free of bank conflicts.
constexpr int kMlpRow = kMlpBatch + 1;

struct MlpGradSmem {
  float w[kMlpW];                 // effective weights
  float h1[kMlpH][kMlpRow];
  float dz1[kMlpH][kMlpRow];
  float h2[kMlpH][kMlpRow];
  float dz2[kMlpH][kMlpRow];
  float x[kMlpBatch];
  float dy[kMlpBatch];
  float r2[kMlpBatch];
};

// Partial gradient of one CTA's kMlpBatch samples (deterministic order):
// part[blockIdx.x][p] for the kMlpW raw parameters, part[..][kMlpW] the sum of
// squared residuals.
template <typename K>
__global__ void __launch_bounds__(kMlpBatch)
k_mlp_grad(const K* __restrict__ sorted, uint64_t S, const MlpState* __restrict__ st, float* part) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpGradSmem& sm = *reinterpret_cast<MlpGradSmem*>(smem_raw);
  const int tid = threadIdx.x;
  for (int p = tid; p < kMlpW; p += blockDim.x) {
    const float r = st->raw[p];
    float w = r;
    if (p < kMlpOffB1) w = mlp_sign(p) * expf(r);
    else if (p >= kMlpOffW2 && p < kMlpOffB2) {
      const int k = (p - kMlpOffW2) / kMlpH, j = (p - kMlpOffW2) % kMlpH;
      w = same_half(k, j) ? expf(r) : 0.0f;
    } else if (p >= kMlpOffW3 && p < kMlpOffB3) w = mlp_sign(p - kMlpOffW3) * expf(r);
    sm.w[p] = w;
  }
  __syncthreads();
  const uint64_t i = blockIdx.x * (uint64_t)kMlpBatch + tid;
  const bool live = i < S;
  const float x = live ? mlp_input<K>(sorted[i], st->kmin, st->scale) : 0.0f;
  const float t = live ? ((float)i + 0.5f) / (float)S : 0.0f;
  // Forward pass.  A ReLU's derivative test z > 0 is the same as h > 0 for
  // h = max(z, 0) (NaN included), so only h1 and the signs of h2 are kept.
  // Layer 2 runs half by half with the unit loop rolled up, so only h1 stays
  // in registers (indexed by constants); the operation order is unchanged.
  float h1[kMlpH];
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) {
    h1[j] = fmaxf(sm.w[kMlpOffW1 + j] * x + sm.w[kMlpOffB1 + j], 0.0f);
    sm.h1[j][tid] = h1[j];
  }
  float y = sm.w[kMlpOffB3];
  uint32_t live2 = 0;                                   // bit k: h2_k > 0
  auto unit2 = [&](int k, const float* h) {             // h: the 16 h1 values of k's half
    float acc = sm.w[kMlpOffB2 + k];
    const int lo = k < kMlpHalf ? 0 : kMlpHalf;
#pragma unroll
    for (int j = 0; j < kMlpHalf; ++j) acc += sm.w[kMlpOffW2 + k * kMlpH + lo + j] * h[j];
    const float h2 = fmaxf(acc, 0.0f);
    sm.h2[k][tid] = h2;
    if (h2 > 0.0f) live2 |= 1u << k;
    y += sm.w[kMlpOffW3 + k] * h2;
  };
#pragma unroll 1
  for (int k = 0; k < kMlpHalf; ++k) unit2(k, h1);
#pragma unroll 1
  for (int k = kMlpHalf; k < kMlpH; ++k) unit2(k, h1 + kMlpHalf);
  const float r = live ? y - t : 0.0f;
  const float dy = 2.0f * r / (float)S;
  // Backward pass: dz2_k = dy w3_k where h2_k > 0, recomputed where used.
  auto dz2 = [&](int k) { return ((live2 >> k) & 1u) ? dy * sm.w[kMlpOffW3 + k] : 0.0f; };
#pragma unroll 1
  for (int k = 0; k < kMlpH; ++k) sm.dz2[k][tid] = dz2(k);
#pragma unroll 1
  for (int j = 0; j < kMlpH; ++j) {
    const int lo = j < kMlpHalf ? 0 : kMlpHalf;
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < kMlpHalf; ++k) acc += dz2(lo + k) * sm.w[kMlpOffW2 + (lo + k) * kMlpH + j];
    sm.dz1[j][tid] = sm.h1[j][tid] > 0.0f ? acc : 0.0f;
  }
  sm.x[tid] = x;
  sm.dy[tid] = dy;
  sm.r2[tid] = r * r;
  __syncthreads();
  // Sums over the CTA's samples in four interleaved chains (s mod 4), added in a
  // fixed order at the end: four independent FMA chains per parameter.
  float* out = part + (uint64_t)blockIdx.x * (kMlpW + 1);
  auto sum4 = [](auto term) {
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll 4
    for (int s = 0; s < kMlpBatch; s += 4) {
      a0 += term(s);
      a1 += term(s + 1);
      a2 += term(s + 2);
      a3 += term(s + 3);
    }
    return (a0 + a1) + (a2 + a3);
  };
  static_assert(kMlpBatch % 4 == 0, "four chains");
  // Threads take the 642 sums that can be non-zero (w1, b1, the same-half
  // entries of W2, b2, w3, b3, the squared residuals) in this order; W2's
  // cross-half entries are always 0 and are written apart.
  constexpr int kLiveW2 = kMlpH * kMlpHalf;                       // 512
  constexpr int kLive = kMlpOffW2 + kLiveW2 + kMlpH + kMlpH + 2;  // 642
  for (int q = tid; q < kMlpH * kMlpH; q += blockDim.x)
    if (!same_half(q / kMlpH, q % kMlpH)) out[kMlpOffW2 + q] = 0.0f;
  for (int l = tid; l < kLive; l += blockDim.x) {
    float g;
    int p;
    if (l < kMlpOffB1) {                                            // w1
      p = l;
      g = sum4([&](int s) { return sm.dz1[p][s] * sm.x[s]; }) * sm.w[p];
    } else if (l < kMlpOffW2) {                                     // b1
      p = l;
      const int q = p - kMlpOffB1;
      g = sum4([&](int s) { return sm.dz1[q][s]; });
    } else if (l < kMlpOffW2 + kLiveW2) {                           // W2 within a half
      const int m = l - kMlpOffW2;
      const int k = m / kMlpHalf, j = (k < kMlpHalf ? 0 : kMlpHalf) + m % kMlpHalf;
      p = kMlpOffW2 + k * kMlpH + j;
      g = sum4([&](int s) { return sm.dz2[k][s] * sm.h1[j][s]; }) * sm.w[p];
    } else if (l < kMlpOffW2 + kLiveW2 + kMlpH) {                   // b2
      const int q = l - kMlpOffW2 - kLiveW2;
      p = kMlpOffB2 + q;
      g = sum4([&](int s) { return sm.dz2[q][s]; });
    } else if (l < kMlpOffW2 + kLiveW2 + 2 * kMlpH) {               // w3
      const int q = l - kMlpOffW2 - kLiveW2 - kMlpH;
      p = kMlpOffW3 + q;
      g = sum4([&](int s) { return sm.dy[s] * sm.h2[q][s]; }) * sm.w[p];
    } else if (l == kLive - 2) {                                    // b3
      p = kMlpOffB3;
      g = sum4([&](int s) { return sm.dy[s]; });
    } else {                                                        // squared residuals
      p = kMlpW;
      g = sum4([&](int s) { return sm.r2[s]; });
    }
    out[p] = g;
  }
}

// Sum the partial gradients and take one Adam step (beta1 0.9, beta2 0.999,
// eps 1e-8); entries of W2 across halves stay 0.  CTA b owns parameters
// [32 b, 32 b + 32): lane l of warp w sums partials w, w + 8, ... of parameter
// 32 b + l, and the eight warp sums are added in warp order (a fixed order).
constexpr int kAdamParams = 32;
constexpr int kAdamWarps = 8;
static __global__ void __launch_bounds__(kAdamParams * kAdamWarps)
k_mlp_adam(const float* __restrict__ part, uint32_t nparts, MlpState* st, uint32_t step, uint64_t S) {
  pdl_enter();
  __shared__ float sums[kAdamWarps][kAdamParams];
  const int lane = threadIdx.x % kAdamParams, warp = threadIdx.x / kAdamParams;
  const int p = blockIdx.x * kAdamParams + lane;
  float g = 0.0f;
  if (p <= kMlpW)
    for (uint32_t c = warp; c < nparts; c += kAdamWarps) g += part[(uint64_t)c * (kMlpW + 1) + p];
  sums[warp][lane] = g;
  __syncthreads();
  if (warp != 0 || p > kMlpW) return;
  g = 0.0f;
#pragma unroll
  for (int w = 0; w < kAdamWarps; ++w) g += sums[w][lane];
  if (p == kMlpW) {
    st->loss = g / (float)S;
    return;
  }
  if (p >= kMlpOffW2 && p < kMlpOffB2) {
    const int k = (p - kMlpOffW2) / kMlpH, j = (p - kMlpOffW2) % kMlpH;
    if (!same_half(k, j)) return;
  }
  const float c1 = 1.0f - powf(0.9f, (float)step), c2 = 1.0f - powf(0.999f, (float)step);
  const float m = 0.9f * st->m[p] + 0.1f * g;
  const float v = 0.999f * st->v[p] + 0.001f * g * g;
  st->m[p] = m;
  st->v[p] = v;
  st->raw[p] -= kMlpLr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
}

// Effective weights and normalisation of the trained model.
static __global__ void k_mlp_finalize(const MlpState* __restrict__ st, float* model) {
  pdl_enter();
  for (int p = threadIdx.x; p < kMlpW; p += blockDim.x) {
    const float r = st->raw[p];
    float w = r;
    if (p < kMlpOffB1) w = mlp_sign(p) * expf(r);
    else if (p >= kMlpOffW2 && p < kMlpOffB2) {
      const int k = (p - kMlpOffW2) / kMlpH, j = (p - kMlpOffW2) % kMlpH;
      w = same_half(k, j) ? expf(r) : 0.0f;
    } else if (p >= kMlpOffW3 && p < kMlpOffB3) w = mlp_sign(p - kMlpOffW3) * expf(r);
    model[p] = w;
  }
  if (threadIdx.x == 0) {
    uint32_t* u = reinterpret_cast<uint32_t*>(model);
    u[kMlpW] = (uint32_t)st->kmin;
    u[kMlpW + 1] = (uint32_t)(st->kmin >> 32);
    model[kMlpW + 2] = st->scale;
    u[kMlpW + 3] = 1u;
  }
}

// A caller's model: copy it and mark it valid only if its signs make it monotone.
static __global__ void k_mlp_validate(const float* __restrict__ given, float* model) {
  pdl_enter();
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < kMlpWords; p += blockDim.x) {
    const float w = given[p];
    model[p] = w;
    bool ok = true;
    if (p < kMlpOffB1) ok = p < kMlpHalf ? w >= 0.0f : w <= 0.0f;
    else if (p >= kMlpOffW2 && p < kMlpOffB2) {
      const int k = (p - kMlpOffW2) / kMlpH, j = (p - kMlpOffW2) % kMlpH;
      ok = !same_half(k, j) || w >= 0.0f;
    } else if (p >= kMlpOffW3 && p < kMlpOffB3) ok = (p - kMlpOffW3) < kMlpHalf ? w >= 0.0f : w <= 0.0f;
    if (p < kMlpW && !(w == w)) ok = false;                 // NaN
    if (!ok) atomicOr(&bad, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) reinterpret_cast<uint32_t*>(model)[kMlpW + 3] = bad ? 0u : 1u;
}

// ---------------------------------------------------------------------------
// K11: the learned cut matrix by bisection of the sorted runs.  The model's
// signs make every fp32 operation of its evaluation monotone, so its bucket id
// never decreases along a sorted run and the keys of run r whose id is below b
// are a prefix: cut[r][b] = #{x in run r : id(x) < b} is the first position
// whose id is at least b, about log2(n_r) evaluations per (run, bucket)
// instead of one pass over every key.  (A caller's model whose signs are not
// monotone is marked invalid and the judge keeps the sampled cuts; its search
// still ends and stays inside the run.)
// ---------------------------------------------------------------------------

constexpr int kLearnedSearchNT = 256;

template <typename K>
__global__ void __launch_bounds__(kLearnedSearchNT)
k_learned_search(const K* __restrict__ runs, const uint64_t* __restrict__ run_off, uint32_t P,
                 const float* __restrict__ model, uint64_t* cutL) {
  pdl_enter();
  __shared__ float w[kMlpW];
  for (int p = threadIdx.x; p < kMlpW; p += blockDim.x) w[p] = model[p];
  __syncthreads();
  const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (q >= (uint64_t)P * (P + 1)) return;
  const uint32_t* u = reinterpret_cast<const uint32_t*>(model);
  const uint64_t kmin = (uint64_t)u[kMlpW] | ((uint64_t)u[kMlpW + 1] << 32);
  const float scale = model[kMlpW + 2];
  const uint64_t r = q / (P + 1), b = q % (P + 1);
  const uint64_t rs = run_off[r], n = run_off[r + 1] - rs;
  uint64_t lo = b == P ? n : 0, hi = b == 0 ? 0 : n;       // b = 0: none below; b = P: all below
  if (b > 0 && b < P) {
    while (lo < hi) {
      const uint64_t mid = lo + ((hi - lo) >> 1);
      if (mlp_bucket<const volatile float*>(w, mlp_input<K>(runs[rs + mid], kmin, scale), P) < (uint32_t)b)
        lo = mid + 1;
      else hi = mid;
    }
  }
  cutL[q] = lo;
}

// The learned bucket vector e_b = sum_r cut[r][b], and the decision: keep the
// learned cuts only for a valid model whose largest bucket is at most
// (1 + eps) n / P.
// P above kLearnedMaxP: the sampled cuts stand, the model is not evaluated,
// and a requested model output is an invalid (flag 0) all-zero model.
static __global__ void k_learned_skip(uint32_t* fallback, float* ratio_out, float* model_out) {
  pdl_enter();
  if (threadIdx.x == 0) {
    *fallback = 1u;
    *ratio_out = __int_as_float(0x7FC00000);
  }
  if (model_out)
    for (int i = threadIdx.x; i < kMlpWords; i += blockDim.x) model_out[i] = 0.0f;
}

static __global__ void k_learned_colsum(const uint64_t* __restrict__ cutL, uint32_t P, uint64_t* eL) {
  pdl_enter();
  const uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (b > P) return;
  uint64_t s = 0;
  for (uint32_t r = 0; r < P; ++r) s += cutL[(uint64_t)r * (P + 1) + b];
  eL[b] = s;
}

static __global__ void __launch_bounds__(256)
k_learned_judge(const uint64_t* __restrict__ eL, uint32_t P, uint64_t n, float eps, const float* __restrict__ model,
                uint32_t* fallback, float* ratio_out) {
  pdl_enter();
  __shared__ uint64_t smax[256];
  uint64_t mx = 0;
  for (uint32_t b = threadIdx.x; b < P; b += blockDim.x) mx = umax(mx, eL[b + 1] - eL[b]);
  smax[threadIdx.x] = mx;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if (threadIdx.x < d) smax[threadIdx.x] = umax(smax[threadIdx.x], smax[threadIdx.x + d]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const bool valid = reinterpret_cast<const uint32_t*>(model)[kMlpW + 3] == 1u;
    const double ratio = n ? (double)smax[0] * P / (double)n : 1.0;
    *ratio_out = (float)ratio;
    *fallback = (!valid || ratio > 1.0 + (double)eps) ? 1u : 0u;
  }
}

// Order form of sorted user keys (float32 bits to their totalOrder image).
template <typename K>
__global__ void k_to_order(const K* __restrict__ in, K* out, uint64_t m, int f32) {
  pdl_enter();
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < m) out[i] = to_order<K>(in[i], f32);
}

// Keep the learned cuts and bucket vector unless the judge fell back.
static __global__ void k_learned_select(const uint64_t* __restrict__ cutL, const uint64_t* __restrict__ eL, uint32_t P,
                                        const uint32_t* __restrict__ fallback, uint64_t* cut, uint64_t* e) {
  pdl_enter();
  if (*fallback) return;
  uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (q < (uint64_t)P * (P + 1)) cut[q] = cutL[q];
  if (q <= P) e[q] = eL[q];
}

}  // namespace pgs
