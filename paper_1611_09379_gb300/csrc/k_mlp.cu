// Learned density compensation for the least-squares INUFFT (M > N).
//
// Per point j, a small network maps 8 scale-free neighbour spacings to a
// weight w_j for the weighted normal equations A^H W A c = A^H W g, so that
// A^H W A is close to the identity and CG needs few iterations.
//
// Features: in periodic position order, the 8 gaps around the point,
// gap_{r+i} = Y_(r+i+1) - Y_(r+i), i = -4..3 (grid units), as log(gap M / N)
// (the mean gap is N/M grid units, so the features do not depend on N, M).
//
// Network: 8 -> 64 -> 64 -> 1, GELU (erf form) on the hidden layers,
// softplus on the output: w = log(1 + e^z).  Parameters (4801 floats):
//   W1[64][8] b1[64] W2[64][64] b2[64] W3[64] b3
// Training keeps FP32 master weights and minimises the mean of
// (log w - log w*)^2 with Adam; inference uses the weights rounded to BF16
// with FP32 accumulation.  All per-point work is one thread per point; the
// weight gradients are reduced per CTA in shared memory and then across CTAs
// in a fixed order.
#include <cmath>
#include <cstdint>
#include <cuda_bf16.h>
#include <new>

#include "common.cuh"

using namespace nufft;

namespace {

constexpr int kIn = 8, kH = 64;
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kH, kNParam = oB3 + 1;  // 4801
constexpr int kTrainPts = 64;                    // points per CTA in training

__device__ inline float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ inline float gelu_d(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * 0.39894228040143268f * expf(-0.5f * x * x);
}
__device__ inline float softplus(float z) { return z > 20.f ? z : log1pf(expf(z)); }
__device__ inline float sigmoid(float z) { return 1.0f / (1.0f + expf(-z)); }

// ---------------------------------------------------------------- features

// Per leaf: order the leaf's points by position (bitonic sort of
// (local position, sorted index) in shared memory); writes rank order
// `pos_perm` (sorted-by-position index -> plan's sorted index).
__global__ void k_position_sort(const int32_t* __restrict__ start, const int32_t* __restrict__ k0s,
                                const double* __restrict__ dels, int N, int s,
                                int32_t* __restrict__ pos_perm, int* __restrict__ status) {
  constexpr int kMax = 2048;
  __shared__ double key[kMax];
  __shared__ int32_t val[kMax];
  int b = blockIdx.x;
  int a = start[b], e = start[b + 1], n = e - a;
  if (n <= 0) return;
  if (n > kMax) {
    if (threadIdx.x == 0) atomicOr(status, kDevSegTooLarge);
    return;
  }
  int P = 1;
  while (P < n) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    if (i < n) {
      // position relative to the leaf origin: (k0 - b s mod N) + delta
      int off = (k0s[a + i] - b * s) & (N - 1);
      key[i] = (double)off + dels[a + i];
      val[i] = a + i;
    } else {
      key[i] = 1e300;
      val[i] = INT32_MAX;
    }
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          bool up = ((i & k) == 0);
          bool gt = key[i] > key[ixj] || (key[i] == key[ixj] && val[i] > val[ixj]);
          if (gt == up) {
            double tk = key[i]; key[i] = key[ixj]; key[ixj] = tk;
            int32_t tv = val[i]; val[i] = val[ixj]; val[ixj] = tv;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) pos_perm[a + i] = val[i];
}

// feat[orig j][8] from the position order (periodic)
__global__ void k_features(const int32_t* __restrict__ pos_perm, const int32_t* __restrict__ perm,
                           const int32_t* __restrict__ k0s, const double* __restrict__ dels,
                           int64_t M, int64_t N, float* __restrict__ feat) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= M) return;
  auto pos = [&](int64_t rr, double wrap) {
    int32_t i = pos_perm[rr];
    int64_t kk = (k0s[i] == 0 && dels[i] < 0.0) ? N : (int64_t)k0s[i];
    return (double)kk + dels[i] + wrap;
  };
  const double scale = (double)M / (double)N;
  float f[kIn];
  for (int t = 0; t < kIn; ++t) {
    int64_t lo = r + t - 4;  // gap between ranks lo and lo + 1
    double wl = 0.0, wh = 0.0;
    int64_t a = lo, b = lo + 1;
    if (a < 0) { a += M; wl = -(double)N; }
    if (a >= M) { a -= M; wl = (double)N; }
    if (b < 0) { b += M; wh = -(double)N; }
    if (b >= M) { b -= M; wh = (double)N; }
    double gap = pos(b, wh) - pos(a, wl);
    if (!(gap > 1e-12)) gap = 1e-12;
    f[t] = (float)log(gap * scale);
  }
  int32_t j = perm[pos_perm[r]];
  for (int t = 0; t < kIn; ++t) feat[(int64_t)j * kIn + t] = f[t];
}

// ---------------------------------------------------------------- inference

// w[i] = softplus(MLP(feat[i])) with BF16 weights, FP32 accumulation.
__global__ void __launch_bounds__(256) k_mlp_infer(const __nv_bfloat16* __restrict__ wb,
                                                   const float* __restrict__ feat, int64_t n,
                                                   float* __restrict__ out) {
  __shared__ float W[kNParam];
  for (int i = threadIdx.x; i < kNParam; i += blockDim.x) W[i] = __bfloat162float(wb[i]);
  __syncthreads();
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  float x[kIn];
  for (int t = 0; t < kIn; ++t) x[t] = feat[p * kIn + t];
  float h1[kH];
#pragma unroll
  for (int i = 0; i < kH; ++i) {
    float a = W[oB1 + i];
#pragma unroll
    for (int t = 0; t < kIn; ++t) a = fmaf(W[oW1 + i * kIn + t], x[t], a);
    h1[i] = gelu(a);
  }
  float z = W[oB3];
  for (int i = 0; i < kH; ++i) {
    float a = W[oB2 + i];
#pragma unroll
    for (int k = 0; k < kH; ++k) a = fmaf(W[oW2 + i * kH + k], h1[k], a);
    z = fmaf(W[oW3 + i], gelu(a), z);
  }
  out[p] = softplus(z);
}

// ---------------------------------------------------------------- training

// One CTA: kTrainPts points.  Phase 1 (one thread per point): forward in FP32
// and backprop of l = (log softplus(z) - t)^2 / n.  Phase 2 (all threads): the
// CTA's weight gradients as sums over its points, written to part[cta][4801].
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ Wg,
                                                  const float* __restrict__ feat,
                                                  const float* __restrict__ target, int64_t n,
                                                  float* __restrict__ part,
                                                  float* __restrict__ loss_part) {
  extern __shared__ float sm[];
  float* W = sm;                                // kNParam
  float* H1 = W + kNParam + 3;                  // [kTrainPts][65]
  float* H2 = H1 + kTrainPts * 65;              // [kTrainPts][65]
  float* D2 = H2 + kTrainPts * 65;              // [kTrainPts][65]
  float* D1 = D2 + kTrainPts * 65;              // [kTrainPts][65]
  float* X = D1 + kTrainPts * 65;               // [kTrainPts][kIn]
  float* DZ = X + kTrainPts * kIn;              // [kTrainPts]
  for (int i = threadIdx.x; i < kNParam; i += blockDim.x) W[i] = Wg[i];
  __syncthreads();
  const int64_t p0 = (int64_t)blockIdx.x * kTrainPts;
  const int t = threadIdx.x;
  if (t < kTrainPts) {
    int64_t p = p0 + t;
    float* h1 = H1 + t * 65;
    float* h2 = H2 + t * 65;
    float* d2 = D2 + t * 65;
    float* d1 = D1 + t * 65;
    float* x = X + t * kIn;
    if (p < n) {
      for (int k = 0; k < kIn; ++k) x[k] = feat[p * kIn + k];
      for (int i = 0; i < kH; ++i) {
        float a = W[oB1 + i];
        for (int k = 0; k < kIn; ++k) a = fmaf(W[oW1 + i * kIn + k], x[k], a);
        d1[i] = a;        // layer-1 pre-activation (kept for the backward pass)
        h1[i] = gelu(a);  // activation
      }
      float z = W[oB3];
      for (int i = 0; i < kH; ++i) {
        float a = W[oB2 + i];
        for (int k = 0; k < kH; ++k) a = fmaf(W[oW2 + i * kH + k], h1[k], a);
        d2[i] = a;  // layer-2 pre-activation
        float g2 = gelu(a);
        h2[i] = g2;
        z = fmaf(W[oW3 + i], g2, z);
      }
      float w = softplus(z);
      float e = logf(w) - target[p];
      DZ[t] = 2.0f * e / (float)n * sigmoid(z) / w;  // dl/dz
      atomicAdd(loss_part + blockIdx.x, e * e / (float)n);
      float dz = DZ[t];
      for (int i = 0; i < kH; ++i) d2[i] = dz * W[oW3 + i] * gelu_d(d2[i]);  // delta2
      for (int k = 0; k < kH; ++k) {
        float a = 0.f;
        for (int i = 0; i < kH; ++i) a = fmaf(W[oW2 + i * kH + k], d2[i], a);
        d1[k] = a * gelu_d(d1[k]);  // delta1
      }
    } else {
      for (int k = 0; k < kIn; ++k) x[k] = 0.f;
      for (int i = 0; i < kH; ++i) { h1[i] = 0.f; h2[i] = 0.f; d2[i] = 0.f; d1[i] = 0.f; }
      DZ[t] = 0.f;
    }
  }
  __syncthreads();
  float* G = part + (int64_t)blockIdx.x * kNParam;
  for (int e = threadIdx.x; e < kNParam; e += blockDim.x) {
    float a = 0.f;
    if (e < oB1) {                       // dW1[i][k] = sum delta1_i x_k
      int i = e / kIn, k = e - i * kIn;
      for (int q = 0; q < kTrainPts; ++q) a = fmaf(D1[q * 65 + i], X[q * kIn + k], a);
    } else if (e < oW2) {                // db1
      int i = e - oB1;
      for (int q = 0; q < kTrainPts; ++q) a += D1[q * 65 + i];
    } else if (e < oB2) {                // dW2[i][k] = sum delta2_i h1_k
      int i = (e - oW2) / kH, k = (e - oW2) - i * kH;
      for (int q = 0; q < kTrainPts; ++q) a = fmaf(D2[q * 65 + i], H1[q * 65 + k], a);
    } else if (e < oW3) {                // db2
      int i = e - oB2;
      for (int q = 0; q < kTrainPts; ++q) a += D2[q * 65 + i];
    } else if (e < oB3) {                // dW3[i] = sum dz h2_i
      int i = e - oW3;
      for (int q = 0; q < kTrainPts; ++q) a = fmaf(DZ[q], H2[q * 65 + i], a);
    } else {                             // db3
      for (int q = 0; q < kTrainPts; ++q) a += DZ[q];
    }
    G[e] = a;
  }
}

// grad[e] = sum over CTAs (fixed order); loss = sum of loss parts
__global__ void k_mlp_reduce(const float* __restrict__ part, int nblocks, float* __restrict__ grad,
                             const float* __restrict__ loss_part, float* __restrict__ loss) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < kNParam) {
    float a = 0.f;
    for (int b = 0; b < nblocks; ++b) a += part[(int64_t)b * kNParam + e];
    grad[e] = a;
  }
  if (e == 0) {
    float l = 0.f;
    for (int b = 0; b < nblocks; ++b) l += loss_part[b];
    *loss = l;
  }
}

// Adam (beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on the FP32 master weights,
// then the BF16 copy used for inference.
__global__ void k_mlp_adam(float* __restrict__ W, float* __restrict__ m1, float* __restrict__ m2,
                           const float* __restrict__ grad, float lr, int step,
                           __nv_bfloat16* __restrict__ wb) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kNParam) return;
  float g = grad[e];
  float a = 0.9f * m1[e] + 0.1f * g, b = 0.999f * m2[e] + 0.001f * g * g;
  m1[e] = a;
  m2[e] = b;
  float ah = a / (1.0f - powf(0.9f, (float)step)), bh = b / (1.0f - powf(0.999f, (float)step));
  float w = W[e] - lr * ah / (sqrtf(bh) + 1e-8f);
  W[e] = w;
  wb[e] = __float2bfloat16_rn(w);
}

__global__ void k_to_bf16(const float* __restrict__ W, __nv_bfloat16* __restrict__ wb) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < kNParam) wb[e] = __float2bfloat16_rn(W[e]);
}

// ---------------------------------------------------------------- training data

// Features of S sorted point sets y[S][M] (radians, ascending): the same
// 8 log gaps as k_features (gap in radians times M / (2 pi)).
__global__ void k_features_sorted(const double* __restrict__ y, int64_t S, int M,
                                  float* __restrict__ feat) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= S * M) return;
  int64_t set = idx / M;
  int r = (int)(idx - set * M);
  const double* ys = y + set * M;
  const double scale = (double)M / kTwoPiHi;
  for (int t = 0; t < kIn; ++t) {
    int a = r + t - 4, b = a + 1;
    double wl = 0.0, wh = 0.0;
    if (a < 0) { a += M; wl = -kTwoPiHi; }
    if (a >= M) { a -= M; wl = kTwoPiHi; }
    if (b < 0) { b += M; wh = -kTwoPiHi; }
    if (b >= M) { b -= M; wh = kTwoPiHi; }
    double gap = (ys[b] + wh) - (ys[a] + wl);
    if (!(gap > 1e-12)) gap = 1e-12;
    feat[idx * kIn + t] = (float)log(gap * scale);
  }
}

// Density-compensation weights of one point set by the multiplicative
// fixed-point iteration w_i <- w_i N / sum_j F(y_i - y_j) w_j, F(t) = |D_N(t)|^2
// = sin^2(N t/2) / sin^2(t/2) (Pipe & Menon's update for the equations
// sum_j F(y_i - y_j) w_j = N that make A^H W A closest to I in Frobenius
// norm; it keeps w > 0).  One CTA per set (M <= 1024), all iterations in
// shared memory; out: log(w / mean w).
__global__ void __launch_bounds__(1024) k_dcf_targets(const double* __restrict__ y, int M, int N,
                                                      int iters, float* __restrict__ logw) {
  __shared__ float ys[1024];
  __shared__ float w[1024];
  __shared__ float red[32];
  const double* yy = y + (int64_t)blockIdx.x * M;
  const int i = threadIdx.x;
  if (i < M) {
    ys[i] = (float)(yy[i] * (1.0 / kTwoPiHi));  // in turns
    w[i] = 1.0f;
  }
  __syncthreads();
  const float Nf = (float)N;
  for (int it = 0; it < iters; ++it) {
    float acc = 0.f;
    if (i < M) {
      float yi = ys[i];
      for (int j = 0; j < M; ++j) {
        float u = yi - ys[j];
        float su = sinpif(u);
        // D_N ratio sin(pi N u) / sin(pi u), whose limit at u -> 0 is N
        float f = (fabsf(su) < 1e-6f) ? Nf : sinpif(Nf * u) / su;
        acc = fmaf(f * f, w[j], acc);
      }
    }
    __syncthreads();
    if (i < M) w[i] = w[i] * Nf / fmaxf(acc, 1e-30f);
    __syncthreads();
  }
  // normalise to mean 1 (scale free) and take logs, floored at 1e-4
  float v = (i < M) ? w[i] : 0.f;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((i & 31) == 0) red[i >> 5] = v;
  __syncthreads();
  if (i < 32) {
    float t = (i < (int)((blockDim.x + 31) / 32)) ? red[i] : 0.f;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (i == 0) red[0] = t;
  }
  __syncthreads();
  float mean = red[0] / (float)M;
  if (i < M) logw[(int64_t)blockIdx.x * M + i] = logf(fmaxf(w[i] / mean, 1e-4f));
}

// sum of w in FP64: per-CTA partials over a fixed stride, then one CTA
// adds them in order (the same sum on every run)
constexpr int kSumBlocks = 256;
__global__ void __launch_bounds__(256) k_sum_partial(const float* __restrict__ w, int64_t n,
                                                     double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)w[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < (unsigned)h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// w_i <- w_i / mean(w), the mean from the partials (every CTA adds them in
// the same order)
__global__ void __launch_bounds__(256) k_scale_to_mean1(float* __restrict__ w, int64_t n,
                                                        const double* __restrict__ part) {
  __shared__ float inv;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < kSumBlocks; ++b) t += part[b];
    inv = t > 0.0 ? (float)((double)n / t) : 1.0f;
  }
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) w[i] *= inv;
}

inline unsigned nblk(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

size_t grad_smem() { return (size_t)(kNParam + 3 + 4 * kTrainPts * 65 + kTrainPts * kIn + kTrainPts) * 4; }

}  // namespace

struct nufft_mlp_s {
  float* W = nullptr;        // FP32 master weights
  float* m1 = nullptr;       // Adam moments
  float* m2 = nullptr;
  float* grad = nullptr;
  __nv_bfloat16* wb = nullptr;  // BF16 inference weights
  float* part = nullptr;     // per-CTA gradient partials
  float* loss = nullptr;     // [1] + loss parts
  int64_t cap = 0;           // points the partial buffers hold
  int step = 0;
};

static void mlp_free(nufft_mlp_s* m) {
  void* ptrs[] = {m->W, m->m1, m->m2, m->grad, m->wb, m->part, m->loss};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete m;
}

static int mlp_reserve(nufft_mlp_s* m, int64_t n) {
  if (n <= m->cap) return NUFFT_OK;
  if (m->part) cudaFree(m->part);
  if (m->loss) cudaFree(m->loss);
  m->part = nullptr;
  m->loss = nullptr;
  int64_t nb = (n + kTrainPts - 1) / kTrainPts;
  if (cudaMalloc((void**)&m->part, (size_t)nb * kNParam * 4) != cudaSuccess ||
      cudaMalloc((void**)&m->loss, (size_t)(nb + 1) * 4) != cudaSuccess) {
    m->cap = 0;
    return NUFFT_ENOMEM;
  }
  m->cap = nb * kTrainPts;
  return NUFFT_OK;
}

extern "C" {

int nufft_mlp_create(nufft_mlp* out) {
  if (!out) return NUFFT_EINVAL;
  *out = nullptr;
  static int configured = 0;
  if (!configured) {
    if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)grad_smem()) != cudaSuccess)
      return NUFFT_ECUDA;
    configured = 1;
  }
  nufft_mlp_s* m = new (std::nothrow) nufft_mlp_s();
  if (!m) return NUFFT_ENOMEM;
  if (cudaMalloc((void**)&m->W, kNParam * 4) != cudaSuccess ||
      cudaMalloc((void**)&m->m1, kNParam * 4) != cudaSuccess ||
      cudaMalloc((void**)&m->m2, kNParam * 4) != cudaSuccess ||
      cudaMalloc((void**)&m->grad, kNParam * 4) != cudaSuccess ||
      cudaMalloc((void**)&m->wb, kNParam * 2) != cudaSuccess) {
    mlp_free(m);
    return NUFFT_ENOMEM;
  }
  if (cudaMemset(m->W, 0, kNParam * 4) != cudaSuccess ||
      cudaMemset(m->m1, 0, kNParam * 4) != cudaSuccess ||
      cudaMemset(m->m2, 0, kNParam * 4) != cudaSuccess ||
      cudaMemset(m->wb, 0, kNParam * 2) != cudaSuccess) {
    mlp_free(m);
    return NUFFT_ECUDA;
  }
  *out = m;
  return NUFFT_OK;
}

int nufft_mlp_destroy(nufft_mlp m) {
  if (!m) return NUFFT_EINVAL;
  cudaDeviceSynchronize();
  mlp_free(m);
  return NUFFT_OK;
}

int nufft_mlp_num_params(void) { return kNParam; }

int nufft_mlp_set_params(nufft_mlp m, const float* host, int reset_optimizer) {
  if (!m || !host) return NUFFT_EINVAL;
  if (cudaMemcpy(m->W, host, kNParam * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return NUFFT_ECUDA;
  k_to_bf16<<<nblk(kNParam, 256), 256>>>(m->W, m->wb);
  if (reset_optimizer) {
    m->step = 0;
    if (cudaMemset(m->m1, 0, kNParam * 4) != cudaSuccess ||
        cudaMemset(m->m2, 0, kNParam * 4) != cudaSuccess)
      return NUFFT_ECUDA;
  }
  return cudaDeviceSynchronize() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

int nufft_mlp_get_params(nufft_mlp m, float* host) {
  if (!m || !host) return NUFFT_EINVAL;
  return cudaMemcpy(host, m->W, kNParam * 4, cudaMemcpyDeviceToHost) == cudaSuccess
             ? NUFFT_OK : NUFFT_ECUDA;
}

int nufft_mlp_infer(nufft_mlp m, const float* feat, int64_t n, float* w, void* stream) {
  if (!m || !feat || !w || n < 0) return NUFFT_EINVAL;
  if (n == 0) return NUFFT_OK;
  k_mlp_infer<<<nblk(n, 256), 256, 0, (cudaStream_t)stream>>>(m->wb, feat, n, w);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

int nufft_mlp_grad(nufft_mlp m, const float* feat, const float* target, int64_t n, float* grad,
                   float* loss, void* stream) {
  if (!m || !feat || !target || n < 1) return NUFFT_EINVAL;
  int rc = mlp_reserve(m, n);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int nb = (int)((n + kTrainPts - 1) / kTrainPts);
  if (cudaMemsetAsync(m->loss, 0, (size_t)(nb + 1) * 4, st) != cudaSuccess) return NUFFT_ECUDA;
  k_mlp_grad<<<nb, 256, grad_smem(), st>>>(m->W, feat, target, n, m->part, m->loss + 1);
  k_mlp_reduce<<<nblk(kNParam, 256), 256, 0, st>>>(m->part, nb, m->grad, m->loss + 1, m->loss);
  if (grad && cudaMemcpyAsync(grad, m->grad, kNParam * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return NUFFT_ECUDA;
  if (loss && cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return NUFFT_ECUDA;
  if ((grad || loss) && cudaStreamSynchronize(st) != cudaSuccess) return NUFFT_ECUDA;
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

int nufft_mlp_train_step(nufft_mlp m, const float* feat, const float* target, int64_t n, float lr,
                         float* loss, void* stream) {
  int rc = nufft_mlp_grad(m, feat, target, n, nullptr, nullptr, stream);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  m->step += 1;
  k_mlp_adam<<<nblk(kNParam, 256), 256, 0, st>>>(m->W, m->m1, m->m2, m->grad, lr, m->step, m->wb);
  if (loss) {
    if (cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return NUFFT_ECUDA;
  }
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

int nufft_dcf_features_sorted(const double* y, int64_t S, int64_t M, float* feat, void* stream) {
  if (!y || !feat || S < 1 || M < 9) return NUFFT_EINVAL;
  k_features_sorted<<<nblk(S * M, 256), 256, 0, (cudaStream_t)stream>>>(y, S, (int)M, feat);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

int nufft_dcf_targets(const double* y, int64_t S, int64_t M, int64_t N, int iters, float* logw,
                      void* stream) {
  if (!y || !logw || S < 1 || M < 1 || M > 1024 || N < 1 || iters < 0) return NUFFT_EINVAL;
  int th = (int)((M + 31) / 32 * 32);
  k_dcf_targets<<<(unsigned)S, th, 0, (cudaStream_t)stream>>>(y, (int)M, (int)N, iters, logw);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

// Features of a plan's points (original order): [M][8] floats.
int nufft_plan_dcf_weights(nufft_plan pl, nufft_mlp m, float* w) {
  if (!pl || !m || !w) return NUFFT_EINVAL;
  cudaStream_t st = pl->stream;
  const int64_t M = pl->M;
  float* feat = nullptr;
  double* part = nullptr;
  if (cudaMallocAsync((void**)&feat, (size_t)M * 8 * 4, st) != cudaSuccess) return NUFFT_ENOMEM;
  if (cudaMallocAsync((void**)&part, kSumBlocks * 8, st) != cudaSuccess) {
    cudaFreeAsync(feat, st);
    return NUFFT_ENOMEM;
  }
  int rc = nufft_plan_dcf_features(pl, feat);
  if (!rc) rc = nufft_mlp_infer(m, feat, M, w, st);
  if (!rc) {
    k_sum_partial<<<kSumBlocks, 256, 0, st>>>(w, M, part);
    k_scale_to_mean1<<<nblk(M, 256), 256, 0, st>>>(w, M, part);
    if (cudaGetLastError() != cudaSuccess) rc = NUFFT_ECUDA;
  }
  cudaFreeAsync(feat, st);
  cudaFreeAsync(part, st);
  return rc;
}

int nufft_plan_dcf_features(nufft_plan pl, float* feat) {
  if (!pl || !feat) return NUFFT_EINVAL;
  cudaStream_t st = pl->stream;
  int32_t* pos_perm = nullptr;
  if (cudaMallocAsync((void**)&pos_perm, pl->M * 4, st) != cudaSuccess) return NUFFT_ENOMEM;
  k_position_sort<<<pl->B, 256, 0, st>>>(pl->leaf_start, pl->k0, pl->delta, (int)pl->N, pl->s,
                                         pos_perm, pl->status);
  k_features<<<nblk(pl->M, 256), 256, 0, st>>>(pos_perm, pl->perm, pl->k0, pl->delta, pl->M, pl->N,
                                               feat);
  cudaFreeAsync(pos_perm, st);
  int hst = 0;
  if (cudaMemcpyAsync(&hst, pl->status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return NUFFT_ECUDA;
  if (hst & kDevSegTooLarge) return NUFFT_ENOTSUP;
  return NUFFT_OK;
}

}  // extern "C"
