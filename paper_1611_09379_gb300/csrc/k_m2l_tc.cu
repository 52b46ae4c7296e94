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
#include "tc_ptx.cuh"

namespace nufft {

namespace {

using namespace tc;

constexpr int kTcParents = 64;   // parents per tile
constexpr int kTcRows = 128;     // MMA M (parents x {re, im})
constexpr int kTcThreads = 256;  // 8 warps
constexpr int kTcTmemCols = 64;  // accumulator columns allocated (>= Npad)
__host__ __device__ inline int tc_kpad(int p) { return (5 * p + 7) & ~7; }
__host__ __device__ inline int tc_npad(int p) { return (2 * p + 15) & ~15; }

// Shared-memory plan of the kernel (byte offsets; the MMA operands start on
// 1024-byte boundaries, the rest on 128-byte ones):
// A_hi, A_lo [128 x kpad] f32; B_hi, B_lo [npad x kpad] f32 (the order of
// the device table); raw multipoles [132 boxes][pm] and raw parent locals
// [64][p] (complex, as in global memory); result staging [64][4p + 1] f32;
// three mbarriers and the TMEM address.
struct TcSmem {
  size_t a_hi, a_lo, b, raw_m, raw_l, stage, bars, total;
};
__host__ __device__ inline size_t tc_align(size_t x) { return (x + 1023) & ~size_t(1023); }
__host__ __device__ inline size_t tc_align16(size_t x) { return (x + 127) & ~size_t(127); }
__host__ __device__ inline TcSmem tc_smem(int p, int pm) {
  const size_t kpad = tc_kpad(p), npad = tc_npad(p);
  TcSmem m;
  m.a_hi = 0;
  m.a_lo = tc_align(m.a_hi + (size_t)kTcRows * kpad * 4);
  m.b = tc_align(m.a_lo + (size_t)kTcRows * kpad * 4);
  m.raw_m = tc_align(m.b + (size_t)2 * npad * kpad * 4);
  m.raw_l = tc_align16(m.raw_m + (size_t)(2 * kTcParents + 4) * pm * 8);
  m.stage = tc_align16(m.raw_l + (size_t)kTcParents * p * 8);
  m.bars = tc_align16(m.stage + (size_t)kTcParents * (4 * p + 1) * 4);
  m.total = m.bars + 64;
  return m;
}

// One tile = parents P0 .. P0 + nval - 1 of one signal at level l - 1.
struct TcTile {
  int sig, P0, nval;
};
__device__ inline TcTile tc_tile(int t, int tiles_per_sig, int npar) {
  TcTile r;
  r.sig = t / tiles_per_sig;
  r.P0 = (t - r.sig * tiles_per_sig) * kTcParents;
  r.nval = npar - r.P0 < kTcParents ? npar - r.P0 : kTcParents;
  return r;
}

// Issue the bulk copies of a tile's raw operands (one thread): multipole
// boxes 2 P0 - 2 .. 2 P0 + 2 nval + 1 (periodic: up to three segments, each
// starting at an even box, so every copy is 16-byte aligned and a multiple
// of 16 bytes) and the parents' locals.  Completion on `bar`.
__device__ inline void tc_issue_raw(const TreeDims& d, int l, const TcTile& tl,
                                    const float2* mexp, const float2* lexp, uint32_t raw_m,
                                    uint32_t raw_l, uint32_t bar) {
  const int pm = d.pm, p = d.p;
  const int nb = 1 << l;
  const int nbox = 2 * tl.nval + 4;
  const float2* ml = mexp + tl.sig * d.mstride + level_off(l) * pm;
  const float2* lp = lexp + tl.sig * d.lstride + (level_off(l - 1) - 4 + (int64_t)tl.P0) * p;
  const uint32_t bytes = (uint32_t)((size_t)nbox * pm * 8 + (size_t)tl.nval * p * 8);
  mbar_expect_tx(bar, bytes);
  int b = 0;
  while (b < nbox) {
    const int box = (2 * tl.P0 - 2 + b + nb) & (nb - 1);
    const int len = nbox - b < nb - box ? nbox - b : nb - box;
    bulk_g2s(raw_m + (uint32_t)(b * pm * 8), ml + (int64_t)box * pm, (uint32_t)(len * pm * 8), bar);
    b += len;
  }
  bulk_g2s(raw_l, lp, (uint32_t)(tl.nval * p * 8), bar);
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_m2l_tc(TreeDims d, int l, int nsig, const float* __restrict__ bops,
             const float2* __restrict__ mexp, float2* __restrict__ lexp, int* __restrict__ status) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(1024) unsigned char smraw[];
  const int p = d.p, pm = d.pm;
  const int kpad = tc_kpad(p), npad = tc_npad(p);
  const TcSmem so = tc_smem(p, pm);
  float* Ahi = reinterpret_cast<float*>(smraw + so.a_hi);
  float* Alo = reinterpret_cast<float*>(smraw + so.a_lo);
  float* Bhi = reinterpret_cast<float*>(smraw + so.b);
  const float2* rawM = reinterpret_cast<const float2*>(smraw + so.raw_m);
  const float2* rawL = reinterpret_cast<const float2*>(smraw + so.raw_l);
  float* S = reinterpret_cast<float*>(smraw + so.stage);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw + so.bars);  // B load, MMA, raw
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar_b = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]),
                 bar_raw = smem_u32(&bars[2]);
  const uint32_t raw_m_u = smem_u32(smraw + so.raw_m), raw_l_u = smem_u32(smraw + so.raw_l);

  const int nb = 1 << l;
  const int npar = nb >> 1;
  const int tiles_per_sig = (npar + kTcParents - 1) / kTcParents;
  const int ntiles = tiles_per_sig * nsig;
  const int G = gridDim.x;

  if (tid == 0) {
    mbar_init(bar_b, 1);
    mbar_init(bar_mma, 1);
    mbar_init(bar_raw, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  int ok = 1;
  if (tid == 0) {
    const uint32_t bbytes = (uint32_t)(2 * npad * kpad * sizeof(float));
    mbar_expect_tx(bar_b, bbytes);
    bulk_g2s(smem_u32(Bhi), bops, bbytes, bar_b);
    if ((int)blockIdx.x < ntiles)
      tc_issue_raw(d, l, tc_tile(blockIdx.x, tiles_per_sig, npar), mexp, lexp, raw_m_u, raw_l_u,
                   bar_raw);
    ok = mbar_wait(bar_b, 0) ? 1 : 0;
  }
  ok = __syncthreads_and(ok);

  const uint32_t idesc = tc_idesc(npad, kTcRows);
  const uint32_t sbo = (uint32_t)kpad * 32u;
  const int ngrp = kpad >> 2;             // k groups of 4
  const int nquad = (ngrp + 3) >> 2;      // k-group quads per row group
  const int srow = 4 * p + 1;
  // A-build mapping: lane -> parent row jj = lane & 7 of a group of 8 and
  // k group 4 qq + (lane >> 3): 16-byte stores, 512 contiguous bytes per warp
  const int jj = lane & 7, kg = lane >> 3;
  // accumulator rows / columns of this thread (epilogue)
  const int arow = 32 * (warp & 3) + lane;
  const int ari = arow >> 6, aj = arow & 63;
  const int ac0 = (warp >> 2) * (npad >> 1);
  float acc[32];
  uint32_t ph_raw = 0, ph_mma = 0;
  TcTile prev{0, 0, 0};
  bool have_prev = false;

  // staged result of a finished tile -> the children's locals (contiguous)
  auto store_prev = [&]() {
#pragma unroll
    for (int e = 0; e < 32; ++e) {
      const int c = ac0 + e;
      if (e < (npad >> 1) && c < 2 * p) {
        const int h = c >= p, n = c - h * p;
        S[aj * srow + h * 2 * p + 2 * n + ari] = acc[e];
      }
    }
    __syncthreads();
    float4* dst = reinterpret_cast<float4*>(lexp + prev.sig * d.lstride +
                                            (level_off(l) - 4 + 2 * (int64_t)prev.P0) * p);
    const int nf4 = p * prev.nval;  // 4 p nval floats
    for (int e = tid; e < nf4; e += kTcThreads) {
      const int f = 4 * e;
      const int jr = f / (4 * p), w = f - jr * 4 * p;
      const float* src = S + jr * srow + w;
      dst[e] = make_float4(src[0], src[1], src[2], src[3]);
    }
  };

  for (int t = blockIdx.x; ok && t < ntiles; t += G) {
    const TcTile tl = tc_tile(t, tiles_per_sig, npar);
    int got = 1;
    if (tid == 0) got = mbar_wait(bar_raw, ph_raw) ? 1 : 0;
    ph_raw ^= 1u;
    if (!__syncthreads_and(got)) { ok = 0; break; }
    // A (hi, lo) from the raw operands; rows j (real part), j + 64 (imaginary)
    for (int it = warp; it < 8 * nquad; it += kTcThreads / 32) {
      const int j = (it & 7) * 8 + jj;
      const int gk = (it >> 3) * 4 + kg;  // k group
      if (gk >= ngrp) continue;
      float re[4], im[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = 4 * gk + i;
        float2 v = make_float2(0.f, 0.f);
        if (j < tl.nval && k < 5 * p) {
          const int s = (k >= p) + (k >= 2 * p) + (k >= 3 * p) + (k >= 4 * p);
          const int m = k - s * p;
          if (s < 4) {
            const int bs = s < 2 ? s : s + 2;  // box slots 2j + {0, 1, 4, 5}
            v = rawM[(2 * j + bs) * pm + m];
          } else {
            v = rawL[j * p + m];
          }
        }
        re[i] = v.x;
        im[i] = v.y;
      }
      float4 h, r;
      split_tf32(re[0], h.x, r.x); split_tf32(re[1], h.y, r.y);
      split_tf32(re[2], h.z, r.z); split_tf32(re[3], h.w, r.w);
      *reinterpret_cast<float4*>(Ahi + tc_off(j, 4 * gk, kpad)) = h;
      *reinterpret_cast<float4*>(Alo + tc_off(j, 4 * gk, kpad)) = r;
      split_tf32(im[0], h.x, r.x); split_tf32(im[1], h.y, r.y);
      split_tf32(im[2], h.z, r.z); split_tf32(im[3], h.w, r.w);
      *reinterpret_cast<float4*>(Ahi + tc_off(j + kTcParents, 4 * gk, kpad)) = h;
      *reinterpret_cast<float4*>(Alo + tc_off(j + kTcParents, 4 * gk, kpad)) = r;
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
      // the raw operands are consumed: fetch the next tile's meanwhile
      if (t + G < ntiles)
        tc_issue_raw(d, l, tc_tile(t + G, tiles_per_sig, npar), mexp, lexp, raw_m_u, raw_l_u,
                     bar_raw);
    }
    // the previous tile's epilogue overlaps these MMAs
    if (have_prev) store_prev();
    int done = 1;
    if (tid == 0) done = mbar_wait(bar_mma, ph_mma) ? 1 : 0;
    ph_mma ^= 1u;
    if (!__syncthreads_and(done)) { ok = 0; break; }
    tc_fence_after();
    for (int cb = 0; cb < (npad >> 1); cb += 8) {
      float v[8];
      tc_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(ac0 + cb), v);
      tc_wait_ld();
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        // acc index cb + e (cb is a multiple of 8 below 32)
#pragma unroll
        for (int z = 0; z < 4; ++z)
          if (cb == 8 * z) acc[8 * z + e] = v[e];
      }
    }
    tc_fence_before();
    __syncthreads();
    prev = tl;
    have_prev = true;
  }
  if (ok && have_prev) store_prev();
  if (!ok && tid == 0) atomicOr(status, kDevTimeout);
  // leave only with the copies and MMAs finished and the tensor memory freed
  if (tid == 0 && !ok) {
    mbar_wait(bar_b, 0);
    mbar_wait(bar_raw, ph_raw);
    mbar_wait(bar_mma, ph_mma);
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

bool m2l_tc_supported(int p, int pm) {
  return tc_npad(p) <= kTcTmemCols && tc_npad(p) / 2 <= 32 && tc_smem(p, pm).total <= 227 * 1024;
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
  if (l < 4 || l > d.L || nsig < 1 || !m2l_tc_supported(d.p, d.pm)) return NUFFT_EINVAL;
  const int npar = 1 << (l - 1);
  const int ntiles = ((npar + kTcParents - 1) / kTcParents) * nsig;
  const int nsm = g_num_sms > 0 ? g_num_sms : 1;
  const int grid = ntiles < nsm ? ntiles : nsm;
  const size_t smem = tc_smem(d.p, d.pm).total;
  launch_pdl(k_m2l_tc, grid, kTcThreads, smem, st, d, l, nsig, bops, mexp, lexp, status);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}
