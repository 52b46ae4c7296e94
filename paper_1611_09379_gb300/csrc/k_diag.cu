// Diagnostics of the near-field arithmetic.
//
// The near-field pair sums (the singular part 2/t of Eq. p20, over a leaf
// and its two neighbours, Sec. 2.1) cost one reciprocal per pair, which
// bounds the target kernels:
//   nufft_diag_rcp         evaluates the library's pair reciprocal rcp_t
//                          (common.cuh) on caller values, so tests can check
//                          it against IEEE division;
//   nufft_diag_pipe_rates  measures how many FP32 reciprocals
//                          (rcp.approx.ftz.f32, the special-function unit)
//                          and FP32 FMAs one SM completes per clock, the
//                          peaks the pair loop is held against.
#include <algorithm>
#include <vector>

#include "common.cuh"

using namespace nufft;

namespace {

__global__ void k_diag_rcp(const double* __restrict__ t, int64_t n, double* __restrict__ r64,
                           float* __restrict__ r32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = t[i];
  if (r64) r64[i] = rcp_t(v);
  if (r32) r32[i] = rcp_t((float)v);
}

constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 4;  // 1024 threads (32 warps) per SM
constexpr int kChains = 8;          // independent dependency chains per thread

struct ProbeRec {
  long long t0, t1;
  int sm, pad;
};

__device__ inline unsigned smid() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// kind 0: x <- rcp(x) + 1/2 (bounded in [1/2, 5/2]; the added constant
// keeps the compiler from folding rcp(rcp(x)) = x, and its FP32 add runs on
// the FMA pipe, which has 8x the reciprocal's lanes); kind 1: x <- x a + b
// (bounded).  Each CTA records its SM and the SM clock before and after its
// loop; `sink` keeps the results live.
__global__ void __launch_bounds__(kProbeThreads) k_probe(int kind, int iters, ProbeRec* rec,
                                                         float* sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0f + 0.125f * c + 1e-3f * (threadIdx.x & 31);
  __syncthreads();
  long long t0 = clock64();
  if (kind == 0) {
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        float r;
        asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[c]));
        asm volatile("add.rn.f32 %0, %1, 0f3F000000;" : "=f"(x[c]) : "f"(r));
      }
    }
  } else {
    const float a = 0.999f, b = 0.001f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(a), "f"(b));
    }
  }
  __syncthreads();
  long long t1 = clock64();
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678f) sink[threadIdx.x] = s;  // practically never: keeps x live
  if (threadIdx.x == 0) {
    ProbeRec r;
    r.t0 = t0;
    r.t1 = t1;
    r.sm = (int)smid();
    r.pad = 0;
    rec[blockIdx.x] = r;
  }
}

}  // namespace

extern "C" int nufft_diag_rcp(const double* t, int64_t n, double* r64, float* r32, void* stream) {
  if (n < 0 || (n > 0 && !t) || (!r64 && !r32)) return NUFFT_EINVAL;
  if (n == 0) return NUFFT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  k_diag_rcp<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(t, n, r64, r32);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

extern "C" int nufft_diag_pipe_rates(double* rcp_per_clk, double* ffma_per_clk, void* stream) {
  if (!rcp_per_clk && !ffma_per_clk) return NUFFT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    return NUFFT_ECUDA;
  const int nctas = nsm * kProbeCtasPerSm;
  ProbeRec* rec = nullptr;
  float* sink = nullptr;
  if (cudaMalloc(&rec, sizeof(ProbeRec) * nctas) != cudaSuccess) return NUFFT_ENOMEM;
  if (cudaMalloc(&sink, sizeof(float) * kProbeThreads) != cudaSuccess) {
    cudaFree(rec);
    return NUFFT_ENOMEM;
  }
  std::vector<ProbeRec> h(nctas);
  int rc = NUFFT_OK;
  for (int kind = 0; kind < 2 && rc == NUFFT_OK; ++kind) {
    double* out = kind == 0 ? rcp_per_clk : ffma_per_clk;
    if (!out) continue;
    const int iters = kind == 0 ? 2048 : 16384;
    for (int rep = 0; rep < 2 && rc == NUFFT_OK; ++rep) {  // the first run warms up
      k_probe<<<nctas, kProbeThreads, 0, st>>>(kind, iters, rec, sink);
      if (cudaGetLastError() != cudaSuccess ||
          cudaMemcpyAsync(h.data(), rec, sizeof(ProbeRec) * nctas, cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        rc = NUFFT_ECUDA;
    }
    if (rc) break;
    // per SM: operations of all its CTAs over the span from the first start
    // to the last end on its own clock; the median over the SMs
    std::vector<long long> lo(nsm, -1), hi(nsm, -1);
    std::vector<int> cnt(nsm, 0);
    for (const ProbeRec& r : h) {
      if (r.sm < 0 || r.sm >= nsm) continue;
      if (lo[r.sm] < 0 || r.t0 < lo[r.sm]) lo[r.sm] = r.t0;
      if (hi[r.sm] < 0 || r.t1 > hi[r.sm]) hi[r.sm] = r.t1;
      cnt[r.sm]++;
    }
    std::vector<double> rate;
    for (int m = 0; m < nsm; ++m)
      if (cnt[m] > 0 && hi[m] > lo[m])
        rate.push_back((double)cnt[m] * kProbeThreads * kChains * (double)iters /
                       (double)(hi[m] - lo[m]));
    if (rate.empty()) { rc = NUFFT_ECUDA; break; }
    std::sort(rate.begin(), rate.end());
    *out = rate[rate.size() / 2];
  }
  cudaFree(rec);
  cudaFree(sink);
  return rc;
}
