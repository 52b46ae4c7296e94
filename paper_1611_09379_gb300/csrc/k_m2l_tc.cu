// M2L + L2L of one tree level on the 5th-generation tensor cores (tcgen05),
// FP32 data in three TF32 passes with FP32 accumulation.
//
// The downward pass of the 1/t FMM (Sec. 2.1) forms, for every box i of
// level l, the local expansion
//   L_l[i][n] = sum_{o in list(i)} sum_m T_o[m][n] M_l[i+o][m]
//             + sum_{k>=n} R_{i mod 2}[k][n] L_{l-1}[i/2][k]
// with the interaction list {-2,+2,+3} for even i and {-3,-2,+2} for odd i
// (separation ratio 1/3, Sec. 2.1) and level-independent scaled operators.
// Both children of a parent P draw on the same four boxes 2P-2, 2P-1, 2P+2,
// 2P+3 and on L_{l-1}[P], so one row per (parent, real/imaginary part)
//   A[(ri, P)][s*p + m] = component ri of {M_l[2P-2], M_l[2P-1], M_l[2P+2],
//                         M_l[2P+3], L_{l-1}[P]}[s][m]         (K = 5p)
// times one fixed operator matrix B [2p x 5p] (columns 0..p-1: child 2P,
// p..2p-1: child 2P+1; the two box slots a child does not use are zero)
// gives both children's locals: D = A B^T, a dense GEMM of shape
// (2 x parents) x 2p x 5p.  A tile is 64 parents = 128 rows (the MMA's M).
//
// Precision: x = x_hi + x_lo with x_hi the TF32 truncation of x; D =
// A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated in FP32 in tensor memory,
// which keeps the FP32 accuracy of the SIMT kernels (one TF32 pass alone
// would leave ~1e-4 relative error).
//
// Data path per tile: the CTA gathers A from the level's multipoles into
// shared memory (no-swizzle K-major core-matrix layout), one thread issues
// 3 x Kpad/8 tcgen05.mma (M = 128, N = Npad, K = 8) into a TMEM accumulator
// and commits them to an mbarrier; all warps read the accumulator back with
// tcgen05.ld, stage it in shared memory and store the 128 children's locals
// with coalesced writes.  The operator B (hi and lo) is loaded once per CTA
// with one bulk copy (cp.async.bulk); the grid is persistent (one CTA per SM).
// Every wait is bounded: a barrier that does not complete sets kDevTimeout in
// the status word, and the CTA still frees its tensor memory before leaving.
#include <cstdint>
#include <vector>

#include "common.cuh"

namespace nufft {

namespace {

constexpr int kTcParents = 64;   // parents per tile
constexpr int kTcRows = 128;     // MMA M (parents x {re, im})
constexpr int kTcThreads = 256;  // 8 warps
constexpr int kTcTmemCols = 64;  // accumulator columns allocated (>= Npad)
constexpr int kMaxGrp = 36;      // kpad / 4 for p <= 28
constexpr long long kSpinLimit = 1ll << 26;   // iteration cap besides the time limit
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s

__host__ __device__ inline int tc_kpad(int p) { return (5 * p + 7) & ~7; }
__host__ __device__ inline int tc_npad(int p) { return (2 * p + 15) & ~15; }

// float offset of element (row, k) in a K-major no-swizzle operand with
// kpad columns: 8 x 4 core matrices of 128 contiguous bytes, K-adjacent core
// matrices 128 B apart, 8-row groups kpad * 32 B apart.
__host__ __device__ inline int tc_off(int row, int k, int kpad) {
  return ((row >> 3) * (kpad >> 2) + (k >> 2)) * 32 + (row & 7) * 4 + (k & 3);
}

__device__ inline uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start, leading (K) byte offset 128,
// stride (8-row group) byte offset sbo, fixed version bits 46-48 = 0b001,
// no swizzle
__device__ inline uint64_t tc_desc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ inline uint32_t tc_idesc(int n, int m) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ inline void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ inline bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ inline uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait for the phase with the given parity to complete (gives up
// after about one second)
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (long long i = 0; i < kSpinLimit; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 255) == 255 && global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

__device__ inline void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// one bulk copy global -> shared, completion counted on the mbarrier
__device__ inline void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ inline void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ inline void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ inline void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ inline void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                              uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "setp.ne.b32 P1, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, P1;\n\t}" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ inline void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// 8 consecutive accumulator columns of this thread's lane
__device__ inline void tc_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ inline void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// TF32 split: hi keeps the top 19 bits (what the tensor core reads)
__device__ inline void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

// Shared memory: A_hi, A_lo [128 x kpad], B_hi, B_lo [npad x kpad] (the
// order of the device table), then the mbarriers and the TMEM address.
__host__ __device__ inline size_t tc_smem_floats(int p) {
  return (size_t)2 * kTcRows * tc_kpad(p) + (size_t)2 * tc_npad(p) * tc_kpad(p);
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_m2l_tc(TreeDims d, int l, int nsig, const float* __restrict__ bops,
             const float2* __restrict__ mexp, float2* __restrict__ lexp, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const int p = d.p, pm = d.pm;
  const int kpad = tc_kpad(p), npad = tc_npad(p);
  float* Ahi = reinterpret_cast<float*>(smraw);
  float* Alo = Ahi + kTcRows * kpad;
  float* Bhi = Alo + kTcRows * kpad;
  uint64_t* bars = reinterpret_cast<uint64_t*>(Bhi + 2 * npad * kpad);  // [0] B load, [1] MMA
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar_b = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);

  // A starts at zero (its K padding stays zero); barriers; B by one bulk copy
  for (int i = tid; i < 2 * kTcRows * kpad; i += kTcThreads) Ahi[i] = 0.f;
  const uint32_t bbytes = (uint32_t)(2 * npad * kpad * sizeof(float));
  if (tid == 0) {
    mbar_init(bar_b, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  int ok = 1;
  if (tid == 0) {
    mbar_expect_tx(bar_b, bbytes);
    bulk_g2s(smem_u32(Bhi), bops, bbytes, bar_b);
    ok = mbar_wait(bar_b, 0) ? 1 : 0;
  }
  ok = __syncthreads_and(ok);

  const int nb = 1 << l;
  const int npar = nb >> 1;
  const int tiles_per_sig = (npar + kTcParents - 1) / kTcParents;
  const int ntiles = tiles_per_sig * nsig;
  const uint32_t idesc = tc_idesc(npad, kTcRows);
  const uint32_t sbo = (uint32_t)kpad * 32u;
  // gather mapping: warp w covers parents 8w..8w+7 (lane & 7) and, per item
  // q, the 4 consecutive k = 4q + (lane >> 3) (conflict-free stores of the
  // core-matrix layout)
  const int kq = lane >> 3, j = warp * 8 + (lane & 7);
  const int ngrp = kpad >> 2;
  uint32_t phase = 0;
  // staging of the result (reuses A_lo once the MMAs are done): per parent
  // 4p floats (child 2P then 2P+1, interleaved re/im), row stride 4p + 1
  float* S = Alo;
  const int srow = 4 * p + 1;

  // this thread's A entries of tile t, all loads issued back to back
  float2 v[kMaxGrp];
  auto load_tile = [&](int t) {
    const int sig = t / tiles_per_sig;
    const int P0 = (t - sig * tiles_per_sig) * kTcParents;
    const int nval = npar - P0 < kTcParents ? npar - P0 : kTcParents;
    const float2* ml = mexp + sig * d.mstride + level_off(l) * pm;
    const float2* lp = lexp + sig * d.lstride + (level_off(l - 1) - 4) * (int64_t)p;
    const int P = P0 + j;
    const bool valid = j < nval;
#pragma unroll
    for (int q = 0; q < kMaxGrp; ++q) {
      v[q] = make_float2(0.f, 0.f);
      const int k = 4 * q + kq;
      if (q < ngrp && valid && k < 5 * p) {
        const int s = (k >= p) + (k >= 2 * p) + (k >= 3 * p) + (k >= 4 * p);
        const int m = k - s * p;
        if (s < 4) {
          const int off = s == 0 ? -2 : (s == 1 ? -1 : s);  // 2P-2, 2P-1, 2P+2, 2P+3
          const int box = (2 * P + off + nb) & (nb - 1);
          v[q] = ml[(int64_t)box * pm + m];
        } else {
          v[q] = lp[(int64_t)P * p + m];
        }
      }
    }
  };

  int t = blockIdx.x;
  if (t < ntiles) load_tile(t);
  for (; ok && t < ntiles; t += gridDim.x) {
    const int sig = t / tiles_per_sig;
    const int P0 = (t - sig * tiles_per_sig) * kTcParents;
    const int nval = npar - P0 < kTcParents ? npar - P0 : kTcParents;
    // A (hi and lo) from the registers; rows j (real) and j + 64 (imaginary)
#pragma unroll
    for (int q = 0; q < kMaxGrp; ++q) {
      if (q < ngrp) {
        const int k = 4 * q + kq;
        float h, r;
        split_tf32(v[q].x, h, r);
        Ahi[tc_off(j, k, kpad)] = h;
        Alo[tc_off(j, k, kpad)] = r;
        split_tf32(v[q].y, h, r);
        Ahi[tc_off(j + kTcParents, k, kpad)] = h;
        Alo[tc_off(j + kTcParents, k, kpad)] = r;
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(Ahi), a1 = smem_u32(Alo);
      const uint32_t b0 = smem_u32(Bhi), b1 = smem_u32(Bhi + npad * kpad);
      const int nk = kpad >> 3;
      for (int pass = 0; pass < 3; ++pass) {
        const uint32_t ab = pass == 2 ? a1 : a0, bb = pass == 1 ? b1 : b0;
        for (int kk = 0; kk < nk; ++kk)
          tc_mma(tmem, tc_desc(ab + kk * 256u, sbo), tc_desc(bb + kk * 256u, sbo), idesc,
                 (pass | kk) ? 1u : 0u);
      }
      tc_commit(bar_mma);
    }
    // the next tile's loads are in flight during the MMAs and the epilogue
    if (t + (int)gridDim.x < ntiles) load_tile(t + gridDim.x);
    int done = 1;
    if (tid == 0) done = mbar_wait(bar_mma, phase) ? 1 : 0;
    phase ^= 1u;
    if (!__syncthreads_and(done)) { ok = 0; break; }
    tc_fence_after();
    // accumulator -> staging: warp quadrant (warp & 3) holds rows 32*(warp & 3)
    // ..+31; warps 0-3 read columns [0, npad/2), warps 4-7 [npad/2, npad)
    {
      const int row = 32 * (warp & 3) + lane;
      const int ri = row >> 6, jr = row & 63;
      const int c0 = (warp >> 2) * (npad >> 1);
      for (int cb = 0; cb < (npad >> 1); cb += 8) {
        float acc[8];
        tc_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(c0 + cb), acc);
        tc_wait_ld();
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int c = c0 + cb + e;
          if (c < 2 * p) {
            const int h = c >= p, n = c - h * p;
            S[jr * srow + h * 2 * p + 2 * n + ri] = acc[e];
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    // children 2P0 .. 2P0 + 2 nval - 1 are contiguous: 2 nval p complex,
    // written as float4 (16-byte aligned: the offset is an even box index)
    {
      float4* dst = reinterpret_cast<float4*>(lexp + sig * d.lstride +
                                              (level_off(l) - 4 + 2 * (int64_t)P0) * p);
      const int nf4 = p * nval;  // (4 p nval) / 4
      for (int e = tid; e < nf4; e += kTcThreads) {
        const int f = 4 * e;
        const int jr = f / (4 * p), w = f - jr * 4 * p;
        const float* src = S + jr * srow + w;  // 4p divisible by 4: no row crossing
        dst[e] = make_float4(src[0], src[1], src[2], src[3]);
      }
    }
    __syncthreads();
  }
  if (!ok && tid == 0) atomicOr(status, kDevTimeout);
  // leave only with the tensor memory freed; a timed-out MMA gets one more
  // bounded wait first
  if (tid == 0 && !ok) {
    mbar_wait(bar_b, 0);
    mbar_wait(bar_mma, phase ^ 1u);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTcTmemCols)
                 : "memory");
}

int g_num_sms = 0;

}  // namespace
}  // namespace nufft

using namespace nufft;

bool m2l_tc_supported(int p) {
  return tc_npad(p) <= kTcTmemCols && (tc_kpad(p) >> 2) <= kMaxGrp &&
         tc_smem_floats(p) * 4 + 64 <= 227 * 1024;
}

size_t m2l_tc_table_floats(int p) { return (size_t)2 * tc_npad(p) * tc_kpad(p); }

// Operator B of the level GEMM in the kernel's shared-memory layout, hi then
// lo, from the plan's M2L [4][p][p] ([d][m][n], d = -3,-2,+2,+3) and L2L
// [2][p][p] ([sigma][k][n]) tables.
void m2l_tc_table(int p, const long double* m2l, const long double* l2l, float* out) {
  const int kpad = tc_kpad(p), npad = tc_npad(p);
  const size_t half = (size_t)npad * kpad;
  for (size_t i = 0; i < 2 * half; ++i) out[i] = 0.f;
  // slot of the M2L table used by (child parity, box slot s); -1 = none
  const int slot[2][4] = {{1, -1, 2, 3}, {0, 1, -1, 2}};
  for (int h = 0; h < 2; ++h)
    for (int n = 0; n < p; ++n) {
      const int c = h * p + n;
      for (int k = 0; k < 5 * p; ++k) {
        const int s = k / p, m = k % p;
        long double v = 0;
        if (s < 4) {
          if (slot[h][s] >= 0) v = m2l[(size_t)slot[h][s] * p * p + (size_t)m * p + n];
        } else if (m >= n) {
          v = l2l[(size_t)h * p * p + (size_t)m * p + n];
        }
        const float f = (float)v;
        uint32_t u;
        __builtin_memcpy(&u, &f, 4);
        u &= 0xFFFFE000u;
        float hi;
        __builtin_memcpy(&hi, &u, 4);
        const float lo = (float)(v - (long double)hi);
        out[tc_off(c, k, kpad)] = hi;
        out[half + tc_off(c, k, kpad)] = lo;
      }
    }
}

int m2l_tc_configure() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NUFFT_ECUDA;
  if (cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return NUFFT_ECUDA;
  if (cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
      cudaSuccess)
    return NUFFT_ECUDA;
  return NUFFT_OK;
}

// Launch the level-l M2L + L2L (l >= 4) for all signals of a plan.
int m2l_tc_level(const TreeDims& d, int l, int nsig, const float* bops, const float2* mexp,
                 float2* lexp, int* status, cudaStream_t st) {
  const int npar = 1 << (l - 1);
  const int ntiles = ((npar + kTcParents - 1) / kTcParents) * nsig;
  const int nsm = g_num_sms > 0 ? g_num_sms : 1;
  const int grid = ntiles < nsm ? ntiles : nsm;
  const size_t smem = tc_smem_floats(d.p) * sizeof(float) + 64;
  k_m2l_tc<<<grid, kTcThreads, smem, st>>>(d, l, nsig, bops, mexp, lexp, status);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}
