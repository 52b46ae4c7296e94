// Near field of the batched forward transform on the tensor cores (tcgen05,
// three TF32 passes, FP32 accumulation).
//
// For many signals sharing one point set the near-field sum of Eq. p20,
//   h_j[sig] = sum_{k in leaves b_j-1, b_j, b_j+1, k != k0_j} f_k[sig] / t_jk,
//   t_jk = (k0_j - k) + delta_j   (grid units),
// is a dense contraction: a tile of 128 sorted targets and the grid samples
// of its leaf window (leaves bl-1 .. bh+1) give
//   H [128 x 2 NS] = K [128 x W] * F [W x 2 NS],
// K_jc = 1 / t_jc inside target j's three leaves (0 outside and for its
// nearest grid point, whose pair E_j carries), F the window samples of NS = 64
// signals, real and imaginary parts as separate columns (N = 128).  The
// window is processed in chunks of 64 samples: the CTA forms K (reciprocals
// on the special-function unit) and gathers F into shared memory in the
// no-swizzle K-major core-matrix layout, split into TF32 hi / lo; one thread
// issues 3 x 8 tcgen05.mma (M = 128, N = 128, K = 8) into one of four TMEM
// accumulators (chunk c into accumulator c mod 4), whose partial sums are
// added with Kahan compensation at the end.  The sums go to hnear [signal][M] (sorted order); the
// forward target kernel adds the far field, the regular part and F_j, E_j.
// Every wait is bounded (status word, then TMEM is freed).
#include <cstdint>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace nufft {
namespace {

using namespace tc;

constexpr int kNtThreads = 256;  // 8 warps
constexpr int kNtRows = 128;     // targets per tile (MMA M)
constexpr int kNtSig = 64;       // signals per tile
constexpr int kNtCols = 2 * kNtSig;  // MMA N: real, imaginary
constexpr int kNtK = 64;         // window samples per chunk
constexpr int kNtRegions = 4;     // accumulators: chunk c adds into region c mod 4
constexpr int kNtTmemCols = kNtCols * kNtRegions;

struct NtSmem {
  static constexpr size_t a_hi = 0;
  static constexpr size_t a_lo = a_hi + (size_t)kNtRows * kNtK * 4;
  static constexpr size_t b_hi = a_lo + (size_t)kNtRows * kNtK * 4;
  static constexpr size_t b_lo = b_hi + (size_t)kNtCols * kNtK * 4;
  static constexpr size_t info = b_lo + (size_t)kNtCols * kNtK * 4;  // per-target data
  static constexpr size_t bars = info + (size_t)kNtRows * 16;
  static constexpr size_t total = bars + 64;
};

__global__ void __launch_bounds__(kNtThreads, 1)
    k_near_tc(TreeDims d, int M, const int32_t* __restrict__ k0s, const double* __restrict__ dels,
              const float* __restrict__ dels_f, const float2* __restrict__ fgrid,
              float2* __restrict__ hnear, int* __restrict__ status) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(1024) unsigned char smraw[];
  float* Ahi = reinterpret_cast<float*>(smraw + NtSmem::a_hi);
  float* Alo = reinterpret_cast<float*>(smraw + NtSmem::a_lo);
  float* Bhi = reinterpret_cast<float*>(smraw + NtSmem::b_hi);
  float* Blo = reinterpret_cast<float*>(smraw + NtSmem::b_lo);
  int* s_kr = reinterpret_cast<int*>(smraw + NtSmem::info);  // nearest grid point, window coords
  int* s_lo = s_kr + kNtRows;                                // first sample of its 3 leaves
  float* s_dt = reinterpret_cast<float*>(s_lo + kNtRows);   // delta
  int* s_b = reinterpret_cast<int*>(s_dt + kNtRows);         // leaf (-1: no target)
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw + NtSmem::bars);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = (int)d.N, s = d.s;
  const int j0 = blockIdx.x * kNtRows;
  const int sig0 = blockIdx.y * kNtSig;
  const uint32_t bar_mma = smem_u32(&bars[0]);

  if (tid == 0) {
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kNtTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid < kNtRows) {
    const int j = j0 + tid;
    int b = -1, o = 0;
    float dt = 0.f;
    if (j < M) {
      point_local(k0s[j], dels[j], N, s, &b, &o);
      dt = dels_f[j];
    }
    s_b[tid] = b;
    s_dt[tid] = dt;
    s_kr[tid] = o;  // leaf-relative for now
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // tile leaf range (targets sorted by leaf) and window of leaves bl-1..bh+1
  const int nval = M - j0 < kNtRows ? M - j0 : kNtRows;
  const int bl = s_b[0], bh = s_b[nval - 1];
  const int W = (bh - bl + 3) * s;
  const int wb = (bl - 1) * s;  // first sample (grid index, unwrapped)
  __syncthreads();
  if (tid < kNtRows && s_b[tid] >= 0) {
    const int sl = s_b[tid] - bl + 1;  // leaf slot of the target in the window
    s_kr[tid] += sl * s;               // nearest grid point in window coordinates
    s_lo[tid] = (sl - 1) * s;
  }
  __syncthreads();

  const uint32_t idesc = tc_idesc(kNtCols, kNtRows);
  const uint32_t sbo = (uint32_t)kNtK * 32u;
  const int jj = lane & 7, kq = lane >> 3;
  const float2* fsig = fgrid + (int64_t)sig0 * N;
  uint32_t phase = 0;
  int ok = 1;
  const int nchunk = (W + kNtK - 1) / kNtK;
  for (int ch = 0; ok && ch < nchunk; ++ch) {
    const int c0 = ch * kNtK;
    // A = K rows: 8 rows x 4 k-groups per warp item, 16-byte stores
    for (int it = warp; it < (kNtRows / 8) * (kNtK / 16); it += kNtThreads / 32) {
      const int row = (it & 15) * 8 + jj;
      const int kg = (it >> 4) * 4 + kq;  // k group of 4
      const int kr = s_kr[row], lo = s_lo[row];
      const float dt = s_dt[row];
      const bool valid = s_b[row] >= 0;
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = c0 + 4 * kg + e;
        const int D = kr - c;  // k0 - k
        float r = 0.f;
        if (valid && c >= lo && c < lo + 3 * s && D != 0) {
          float t = (float)D + dt;
          asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
        }
        v[e] = r;
      }
      float4 h, l;
      split_tf32(v[0], h.x, l.x); split_tf32(v[1], h.y, l.y);
      split_tf32(v[2], h.z, l.z); split_tf32(v[3], h.w, l.w);
      *reinterpret_cast<float4*>(Ahi + tc_off(row, 4 * kg, kNtK)) = h;
      *reinterpret_cast<float4*>(Alo + tc_off(row, 4 * kg, kNtK)) = l;
    }
    // B = window samples: rows 2 sl (real), 2 sl + 1 (imaginary); lane = 4
    // signals x 8 k-groups
    for (int it = warp; it < (kNtSig / 4) * (kNtK / 32); it += kNtThreads / 32) {
      const int sl = (it & 15) * 4 + (lane & 3);
      const int kg = (it >> 4) * 8 + (lane >> 2);
      const float2* fs = fsig + (int64_t)sl * N;
      float re[4], im[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = c0 + 4 * kg + e;
        float2 x = make_float2(0.f, 0.f);
        if (c < W) x = fs[(wb + c + N) & (N - 1)];
        re[e] = x.x;
        im[e] = x.y;
      }
      float4 h, l;
      split_tf32(re[0], h.x, l.x); split_tf32(re[1], h.y, l.y);
      split_tf32(re[2], h.z, l.z); split_tf32(re[3], h.w, l.w);
      *reinterpret_cast<float4*>(Bhi + tc_off(2 * sl, 4 * kg, kNtK)) = h;
      *reinterpret_cast<float4*>(Blo + tc_off(2 * sl, 4 * kg, kNtK)) = l;
      split_tf32(im[0], h.x, l.x); split_tf32(im[1], h.y, l.y);
      split_tf32(im[2], h.z, l.z); split_tf32(im[3], h.w, l.w);
      *reinterpret_cast<float4*>(Bhi + tc_off(2 * sl + 1, 4 * kg, kNtK)) = h;
      *reinterpret_cast<float4*>(Blo + tc_off(2 * sl + 1, 4 * kg, kNtK)) = l;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    int done = 1;
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(Ahi), a1 = smem_u32(Alo);
      const uint32_t b0 = smem_u32(Bhi), b1 = smem_u32(Blo);
      for (int pass = 0; pass < 3; ++pass) {
        const uint32_t ab = pass == 2 ? a1 : a0, bb = pass == 1 ? b1 : b0;
        for (int kk = 0; kk < kNtK / 8; ++kk)
          tc_mma(tmem + (uint32_t)((ch % kNtRegions) * kNtCols), tc_desc(ab + kk * 256u, sbo),
                 tc_desc(bb + kk * 256u, sbo), idesc,
                 (ch >= kNtRegions || pass || kk) ? 1u : 0u);
      }
      tc_commit(bar_mma);
      done = mbar_wait(bar_mma, phase) ? 1 : 0;
    }
    phase ^= 1u;
    if (!__syncthreads_and(done)) ok = 0;
    tc_fence_after();
  }
  if (ok) {
    // accumulator rows = targets (warp quadrant), columns 2 sl + ri: warps
    // 0-3 take signals 0..31, warps 4-7 signals 32..63
    const int row = 32 * (warp & 3) + lane;
    const int j = j0 + row;
    const int cbase = (warp >> 2) * kNtSig;
    const int nreg = nchunk < kNtRegions ? nchunk : kNtRegions;
    for (int cb = 0; cb < kNtSig; cb += 8) {
      // the regions' partial sums, added with compensation
      float v[8], comp[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) { v[e] = 0.f; comp[e] = 0.f; }
      for (int rg = 0; rg < nreg; ++rg) {
        float w[8];
        tc_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(rg * kNtCols + cbase + cb),
               w);
        tc_wait_ld();
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float yv = w[e] - comp[e];
          const float tv = v[e] + yv;
          comp[e] = (tv - v[e]) - yv;
          v[e] = tv;
        }
      }
      if (j < M) {
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          const int sl = (cbase + cb + e) >> 1;
          hnear[(int64_t)(sig0 + sl) * M + j] = make_float2(v[e], v[e + 1]);
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(status, kDevTimeout);
    mbar_wait(bar_mma, phase ^ 1u);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kNtTmemCols)
                 : "memory");
}

}  // namespace
}  // namespace nufft

using namespace nufft;

int near_tc_configure() {
  return cudaFuncSetAttribute(k_near_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)NtSmem::total) == cudaSuccess
             ? NUFFT_OK : NUFFT_ECUDA;
}

// The batched forward's near-field sums on the tensor cores, for signals in
// groups of 64 (batch % 64 == 0), into hnear [batch][M] (sorted order).
int near_tc_forward(const TreeDims& d, int M, int batch, const int32_t* k0s, const double* dels,
                    const float* dels_f, const float2* fgrid, float2* hnear, int* status,
                    cudaStream_t st) {
  if (batch % kNtSig != 0 || M < 1) return NUFFT_EINVAL;
  dim3 grid((unsigned)((M + kNtRows - 1) / kNtRows), (unsigned)(batch / kNtSig));
  launch_pdl(k_near_tc, grid, kNtThreads, NtSmem::total, st, d, M, k0s, dels, dels_f, fgrid, hnear,
             status);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}
